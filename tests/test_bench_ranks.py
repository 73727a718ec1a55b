"""Replica aggregation of bench.py across ranks (world size 2, gloo on CPU):
the job time is the slowest rank's, the throughput counts every rank's cells,
and the reference arm runs on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [12.5, 20.0][rank]
    job_ms = bench.reduce_timed_ms(local_ms, dist, "cpu")
    value = bench.job_mlups(world * 1000, 10, job_ms)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, job_ms, value))


def test_two_rank_timing_takes_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, job_ms, value in res:
        assert job_ms == 20.0
        # 2 ranks x 1000 cells x 10 steps in 20 ms
        assert value == pytest.approx(2 * 1000 * 10 / 0.020 / 1e6)


def test_single_rank_reduction_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_timed_ms(7.25) == 7.25
    assert bench.job_mlups(262144, 200, 6.0) == pytest.approx(262144 * 200 / 6e-3 / 1e6)


def test_reference_arm_exits_without_work_on_other_ranks():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                          "--steps", "1", "--warmup", "3"], capture_output=True, text=True, env=env, cwd=ROOT,
                         timeout=120)
    assert out.returncode == 0
    assert out.stdout.strip() == ""
