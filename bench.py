#!/usr/bin/env python3
"""Throughput of the fused RLBM step on GB300 (MLUPS and fraction of the HBM roofline).

Default workload (the 2-d massless Taylor-Green configuration): 512 x 512
doubly periodic grid, order-2 massless quadrature (Q = 28), off-lattice
bilinear streaming with lambda = 1, tau = 1, u0 = 0.1 c, uniform n = T = 1,
FP32 populations with an FP32 Landau solve whose eigenvalue gets a
float-float (48-bit) Newton correction.  A bench step is one RLBM time
step (one fused kernel launch over the whole grid); the L2 cache is flushed
(a 256 MiB write) before every timed step, so each step reads its inputs
from HBM.  Each launch is timed with CUDA events on the stream it runs on.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (launched by torch.distributed.run) every rank runs an
independent replica on its own GPU (replicas only; the step has no exchange
on one grid per GPU); value = all ranks' cell updates / max-over-ranks time.
``--impl reference`` times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    "tg512": dict(workload="tg512_bilinear_fp32", L=512, stream="bilinear", lam=1.0, tau=1.0,
                  u0=0.1, precision="fp32", order=2, m=0.0, resident_steps=5000),
    "tg512_onlattice": dict(workload="tg512_onlattice_fp32", L=512, stream="onlattice", lam=0.0,
                            tau=1.0, u0=0.1, precision="fp32", order=2, m=0.0, resident_steps=5000),
    "tg2048": dict(workload="tg2048_bilinear_fp32", L=2048, stream="bilinear", lam=1.0, tau=1.0,
                   u0=0.1, precision="fp32", order=2, m=0.0, resident_steps=500),
    "tg512_fp64": dict(workload="tg512_bilinear_fp64", L=512, stream="bilinear", lam=1.0, tau=1.0,
                       u0=0.1, precision="fp64", order=2, m=0.0, resident_steps=200),
}

METRIC = "MLUPS"   # million lattice-cell updates per second (whole job)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _kernel_source_sha():
    h = hashlib.sha256()
    for name in ("step_impl.cuh", "kernels.cuh", "fpconv.cuh"):
        with open(os.path.join(ROOT, "paper_1909_04502_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _profiled_traffic(workload):
    """DRAM bytes per launch from the committed ncu summary of this workload,
    or None when the kernel source changed since the capture."""
    path = os.path.join(ROOT, "profiles", "step_%s.md" % workload)
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    s = re.search(r"kernel_source_sha:\s*([0-9a-f]+)", txt)
    if not m or not s or s.group(1) != _kernel_source_sha():
        return None
    return float(m.group(1))


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + q, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# Oracle timing (CPU; test infrastructure) -- run in a child process pinned to
# one thread so that the reported core count is exact.
# ---------------------------------------------------------------------------


def _oracle_worker(L, steps, warmup, stream, lam, tau, u0):
    import numpy as np
    from oracle import lattice as OL
    from oracle import scheme as OS
    from paper_1909_04502_gb300 import inputs
    q = OL.massless_quadrature(2)
    sim = OS.Simulation(q, OL.Expansion(q), L, L, tau=tau, stream=stream,
                        lam=lam if stream == "bilinear" else None)
    sim.init(*inputs.taylor_green(L, u0=u0))
    sim.step(warmup)
    times = []
    t_begin = time.time()
    for _ in range(steps):
        t0 = time.perf_counter()
        sim.step(1)
        times.append(time.perf_counter() - t0)
    t_end = time.time()
    print(json.dumps({"cells": L * L, "times": times, "t_begin": t_begin, "t_end": t_end,
                      "finite": bool(np.isfinite(sim.fs).all())}))


def host_cores():
    """Cores this process may run on (the affinity mask), else the CPU count."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def run_oracle(L, steps, warmup, wl, procs=1):
    """The unchanged oracle in `procs` single-threaded worker processes at
    once, each stepping its own copy of the L x L sample (independent
    replicas, one per core).  Returns the per-worker reports and the
    aggregate cell updates per second over the span from the first timed
    step to the last (every worker's timed loop lies inside it)."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    cmd = [sys.executable, os.path.abspath(__file__), "--_oracle_worker",
           json.dumps([L, steps, warmup, wl["stream"], wl["lam"], wl["tau"], wl["u0"]])]
    workers = [subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env, cwd=ROOT)
               for _ in range(procs)]
    reports = []
    for w in workers:
        out, err = w.communicate()
        if w.returncode != 0:
            raise RuntimeError("oracle worker failed: " + err[-2000:])
        reports.append(json.loads(out.strip().splitlines()[-1]))
    span = max(r["t_end"] for r in reports) - min(r["t_begin"] for r in reports)
    rate = sum(r["cells"] * len(r["times"]) for r in reports) / span
    return reports, rate


def oracle_sample_size(wl, budget_s, nsteps):
    """Largest square grid <= the workload's whose nsteps oracle steps fit the
    budget, and the probed oracle time per cell update."""
    probe = run_oracle(64, 2, 0, wl)[0][0]
    per_cell = statistics.median(probe["times"]) / probe["cells"]
    L = wl["L"]
    while L > 32 and per_cell * L * L * nsteps > budget_s:
        L //= 2
    return L, per_cell


def reduce_timed_ms(local_ms, dist=None, device="cuda"):
    """Job time of a replica run: the slowest rank's timed interval (MAX over
    ranks; the identity on one rank)."""
    if dist is None:
        return float(local_ms)
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(total_cells, steps, job_ms):
    """Whole-job throughput: cell updates of all ranks over the job time."""
    return total_cells * steps / (job_ms * 1e-3) / 1e6


# ---------------------------------------------------------------------------


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="tg512", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched and adjoint measurements")
    ap.add_argument("--only", default=None, choices=["batched", "adjoint", "paper", "kh", "d3", "forcing", "d1"],
                    help="run only this extra measurement and print its JSON object")
    ap.add_argument("--side", type=int, default=None,
                    help="grid side for --only kh / d3 (default 2048 / 192); smaller sides serve profiling")
    ap.add_argument("--_oracle_worker", default=None)
    args = ap.parse_args()
    if args._oracle_worker is not None:
        _oracle_worker(*json.loads(args._oracle_worker))
        return
    args.warmup = max(args.warmup, 3)
    wl = WORKLOADS[args.workload]

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        bench_reference(args, wl)
        return

    import numpy as np
    import torch

    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    from paper_1909_04502_gb300 import build as _build
    if rank == 0:
        _build.build()
    if dist:
        dist.barrier()
    from paper_1909_04502_gb300 import inputs, rlbm

    if args.only:
        stream = torch.cuda.current_stream()
        if args.only == "batched":
            res = {"batched": bench_batched(torch, rlbm, inputs, stream),
                   "batched_small": bench_batched(torch, rlbm, inputs, stream, steps=50, side_hi=256)}
        elif args.only == "paper":
            res = {"massive_order3_tg512": bench_massive_order3(torch, rlbm, inputs, stream),
                   "paper_stencil45_tg512": bench_massive_order3(torch, rlbm, inputs, stream, m=15.0,
                                                                 groups=PAPER_STENCIL_45)}
        elif args.only == "kh":
            res = {"kelvin_helmholtz": bench_kh(torch, rlbm, inputs, stream, L=args.side or 2048)}
        elif args.only == "d3":
            res = {"d3_taylor_green": bench_d3(torch, rlbm, inputs, stream, L=args.side or 192)}
        elif args.only == "forcing":
            res = {"forcing_walls": bench_forcing_walls(torch, rlbm, inputs, stream)}
        elif args.only == "d1":
            res = {"d1_wave": bench_d1(torch, rlbm, inputs, stream)}
        else:
            res = {"adjoint": bench_adjoint(torch, rlbm, inputs, stream)}
        if rank == 0:
            print(json.dumps(res))
        return

    L = wl["L"]
    ncell = L * L
    fields = [np.ascontiguousarray(a) for a in inputs.taylor_green(L, u0=wl["u0"])]
    stream = torch.cuda.current_stream()
    lat = rlbm.Lattice(L, L, m=wl["m"], order=wl["order"], tau=wl["tau"], stream=wl["stream"],
                       lam=wl["lam"], precision=wl["precision"], cuda_stream=stream.cuda_stream)
    Q = lat.Q
    elem = 4 if wl["precision"] == "fp32" else 8
    lat.init(*fields)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    # warm-up
    for _ in range(args.warmup):
        flush.zero_()
        lat.step(1)
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()
            starts[k].record(stream)
            lat.step(1)
            ends[k].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    kt = [s.elapsed_time(e) for s, e in zip(starts, ends)]   # ms per launch
    total_ms = reduce_timed_ms(sum(kt), dist, "cuda")
    status = lat.sync_status(raise_on_error=False)

    value = job_mlups(world * ncell, args.steps, total_ms)
    ms_per_step = total_ms / args.steps
    peak, peak_kind = _peaks()
    alg_bytes = 2 * Q * elem * ncell                     # read + write every population once
    achieved = alg_bytes / (ms_per_step * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": _profiled_traffic(wl["workload"]),
                "peak_kind": peak_kind, "algorithmic_bytes_per_launch": alg_bytes,
                "kernel": "k_step (fused stream+collide)"}

    # back-to-back run of the whole job (L2 not flushed between steps)
    lat.init(*fields)
    m0 = lat.moments(full=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lat.step(wl["resident_steps"])
    e1.record(stream)
    torch.cuda.synchronize()
    resident_ms = e0.elapsed_time(e1)
    m1 = lat.moments(full=True)
    N0, T00 = float(m0["N"][0].sum()), float(m0["Tab"][0].sum())
    resident = {"steps": wl["resident_steps"],
                "mlups": round(ncell * wl["resident_steps"] / (resident_ms * 1e-3) / 1e6, 1),
                "note": "whole run back to back; the 59 MB working set of 512^2 stays in the 129 MB L2",
                "drift_N0_rel": float(abs(m1["N"][0].sum() - N0) / N0),
                "drift_T0a_rel": [float(abs(m1["Tab"][j].sum() - m0["Tab"][j].sum()) / T00) for j in range(3)]}

    # end to end through the C ABI with pinned host buffers
    host_in = [torch.from_numpy(a).pin_memory() for a in fields]
    host_out = {k: torch.empty((L, L), dtype=torch.float64).pin_memory() for k in ("n", "ux", "uy", "T", "eps")}
    e2e_steps = 100
    e2e_iters = 5
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_iters):
        lat.init(*host_in)
        lat.step(e2e_steps)
        _moments_to_pinned(lat, host_out)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_iters
    h2d, d2h = 4 * 8 * ncell, 5 * 8 * ncell           # bytes copied per call
    e2e = {"value": round(ncell * e2e_steps / e2e_s / 1e6, 1), "unit": METRIC,
           "h2d_bytes_per_step": h2d // e2e_steps, "d2h_bytes_per_step": d2h // e2e_steps,
           "h2d_bytes_per_call": h2d, "d2h_bytes_per_call": d2h, "steps_per_call": e2e_steps,
           "call": "rlbm_init(host n,u,T) + rlbm_step(100) + rlbm_moments(host n,u,T,eps), pinned; "
                   "the per-step bytes are the call's copies over its 100 steps"}

    parity = None
    cpu = None
    extras = {}
    if rank == 0:
        parity = oracle_parity(lat, fields, wl)
        if world == 1 and not args.no_cpu_baseline:
            cpu = cpu_baseline(wl)
    if not args.no_extras:
        extras["batched"] = bench_batched(torch, rlbm, inputs, stream)
        extras["batched_small"] = bench_batched(torch, rlbm, inputs, stream, steps=50, side_hi=256)
        extras["adjoint"] = bench_adjoint(torch, rlbm, inputs, stream)
        extras["massive_order3_tg512"] = bench_massive_order3(torch, rlbm, inputs, stream)
        extras["paper_stencil45_tg512"] = bench_massive_order3(torch, rlbm, inputs, stream, m=15.0,
                                                               groups=PAPER_STENCIL_45)
        extras["kelvin_helmholtz_2048"] = bench_kh(torch, rlbm, inputs, stream)
        extras["d3_taylor_green_192"] = bench_d3(torch, rlbm, inputs, stream)
        extras["forcing_walls"] = bench_forcing_walls(torch, rlbm, inputs, stream)
        extras["d1_wave"] = bench_d1(torch, rlbm, inputs, stream)
        if wl["workload"] == "tg512_bilinear_fp32":
            extras["viscosity"] = bench_tg_viscosity(rlbm, inputs)

    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": METRIC, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32" if elem == 4 else "f64",
        "data": "synthetic",
        "config": {"workload": wl["workload"], "nx": L, "ny": L, "Q": Q, "order": wl["order"],
                   "quadrature": "App. H massless order 2", "stream": wl["stream"], "lambda": wl["lam"],
                   "tau": wl["tau"], "u0": wl["u0"],
                   "landau": "FP32 Newton, float-float (48-bit) residual correction of the eigenvalue" if elem == 4 else "FP64",
                   "l2": "flushed before every timed step (256 MiB write)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": args.steps,
        "clocks": clocks, "resident": resident, "parity": parity, **extras,
        "status": {"nonphysical_cells": status[1]}, "wall_s_timed_region": round(wall, 4),
    }
    if rank == 0:
        print(json.dumps(line))
    lat.close()
    if dist:
        dist.destroy_process_group()


def _moments_to_pinned(lat, host_out):
    import ctypes
    from paper_1909_04502_gb300 import rlbm
    ptr = [host_out[k].data_ptr() for k in ("n", "ux", "uy", "T", "eps")]
    rc = rlbm.lib().rlbm_moments(lat.h, *ptr, None, None, 0)
    if rc != 0:
        raise RuntimeError(rlbm.lib().rlbm_last_error(lat.h).decode())


def oracle_parity(lat, fields, wl):
    """Two steps of the bench workload against the FP64 oracle, element by element."""
    import numpy as np
    from tests.cases import oracle_quadrature, oracle_sim, permutation, rel_linf
    L = wl["L"]
    if L > 1024:
        return None
    quad = oracle_quadrature(wl["m"], wl["order"])
    sim = oracle_sim(quad, L, L, tau=wl["tau"], stream=wl["stream"],
                     lam=wl["lam"] if wl["stream"] == "bilinear" else None)
    sim.init(*fields)
    lat.init(*fields)
    lat.step(2)
    sim.step(2)
    idx = permutation(lat.n, lat.p, quad)
    m = lat.moments()
    return {"steps": 2, "rel_linf_f": rel_linf(lat.populations()[idx], sim.fs),
            "rel_linf_ux": float(np.abs(m["ux"] - sim.fields.ux).max() / np.abs(sim.fields.ux).max()),
            "bar": 1e-5 if wl["precision"] == "fp32" else 1e-12}


def cpu_baseline(wl, budget_s=12.0):
    """The oracle on all host cores: one single-threaded worker per core,
    each stepping its own copy of the workload's grid (halved until three
    steps fit the budget) for as many steps as fill about budget_s seconds;
    the value is the aggregate over the workers."""
    L, per_cell = oracle_sample_size(wl, budget_s, 3)
    nsteps = int(max(3, min(200, budget_s / (per_cell * L * L))))
    cores = host_cores()
    reports, rate = run_oracle(L, nsteps, 1, wl, procs=cores)
    return {"value": round(rate / 1e6, 4), "unit": METRIC, "cores": cores, "kind": "oracle",
            "sample": "%d oracle steps of the same Taylor-Green configuration on a %dx%d grid in each of %d "
                      "single-threaded worker processes at once (numpy FP64, one per host core)"
                      % (nsteps, L, L, cores)}


def bench_batched(torch, rlbm, inputs, stream, steps=10, count=64, seed=1909, side_lo=64, side_hi=1024,
                  zetas=(0.0, 1.0, 10.0)):
    """Batched tau-sweep: `count` shear-wave runs, side ~ U{side_lo..side_hi},
    tau ~ U[0.6, 2.0], zeta round-robin over {0, 1, 10}, amplitude 0.05 c,
    FP32 storage (float-float Landau correction), on-lattice order-2 stencils.  One
    graph launch per call (the tuner's choice of persistent cooperative
    kernels, one per stencil kind, or independent per-instance chains of
    step kernels) against the same instances stepped one handle at a time
    (back-to-back launches).  The working set of all instances exceeds L2 for
    both sweeps the bench runs (about 5 GB and 0.4 GB), so L2 is not flushed."""
    import numpy as np
    runs = inputs.sweep(count=count, seed=seed, side_lo=side_lo, side_hi=side_hi, zetas=zetas)
    cfgs = [dict(nx=r["side"], ny=r["side"], tau=r["tau"], m=r["zeta"], precision="fp32") for r in runs]
    batch = rlbm.Batch(cfgs, cuda_stream=stream.cuda_stream)
    shape, grid, _ = batch.tune(trial_steps=4)
    cells = 0
    for i, r in enumerate(runs):
        f = [np.ascontiguousarray(a) for a in inputs.shear_wave(r["side"], r["side"], amp=0.05)]
        batch[i].init(*f)
        cells += r["side"] ** 2
    Qs = [batch[i].Q for i in range(len(batch))]
    alg_bytes = sum(2 * Q * 4 * r["side"] ** 2 for Q, r in zip(Qs, runs))
    batch.step(steps)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    batch.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    tb = e0.elapsed_time(e1) / steps
    # the same instances, one handle at a time (each call launches `steps` kernels)
    for lat in batch.instances:
        lat.step(1)
    torch.cuda.synchronize()
    e0.record(stream)
    for lat in batch.instances:
        lat.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    tp = e0.elapsed_time(e1) / steps
    rc, nonphys = batch.sync_status(raise_on_error=False)
    peak, _ = _peaks()
    out = {"workload": "tau_sweep_%d_shear_waves_side_%d_%d" % (count, side_lo, side_hi), "instances": count,
           "cells": cells, "seed": seed, "zetas": list(zetas),
           "steps_timed": steps, "ms_per_step_batched": round(tb, 4), "ms_per_step_plain_loop": round(tp, 4),
           "mlups_batched": round(cells / (tb * 1e-3) / 1e6, 1), "mlups_plain_loop": round(cells / (tp * 1e-3) / 1e6, 1),
           "speedup_vs_plain_loop": round(tp / tb, 3),
           "roofline": {"bound": "hbm", "achieved": round(alg_bytes / (tb * 1e-3) / 1e9, 1), "peak": peak,
                        "unit": "GB/s", "frac": round(alg_bytes / (tb * 1e-3) / 1e9 / peak, 4)},
           "tuned": {"schedule": ["persistent 32x8", "persistent 32x4", "per-instance chains"][shape],
                     "grid": grid}, "status": rc,
           "nonphysical": nonphys}
    batch.close()
    return out


def bench_adjoint(torch, rlbm, inputs, stream, L=512, nsteps=2000, K=100):
    """Differentiable calibration run: L x L massless shear flow u_y = 0.05
    sin(2 pi x / L), hidden tau field, nsteps steps; forward with checkpoints
    every K steps, then the adjoint backward pass with recomputation."""
    import numpy as np
    n, ux, uy, T = [np.ascontiguousarray(a) for a in inputs.shear_wave(L, L, amp=0.05)]
    tau = np.ascontiguousarray(inputs.smooth_tau(L, L))
    lat = rlbm.Lattice(L, L, tau_mode="field", precision="fp32", cuda_stream=stream.cuda_stream)
    lat.set_tau_field(tau)
    adj = rlbm.Adjoint(lat, nsteps, K)
    dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    n_d, ux_d, uy_d, T_d = dev(n), dev(ux), dev(uy), dev(T)
    tgt_x, tgt_y = dev(np.zeros_like(ux)), dev(0.9 * uy)
    out = {"loss": torch.zeros(1, dtype=torch.float64, device="cuda"), "tau": torch.empty_like(n_d),
           "ux0": torch.empty_like(n_d), "uy0": torch.empty_like(n_d)}
    adj.forward(n_d, ux_d, uy_d, T_d)                 # warm-up
    adj.backward(tgt_x, tgt_y, out=out)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    adj.forward(n_d, ux_d, uy_d, T_d)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    adj.backward(tgt_x, tgt_y, out=out)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    cells = L * L * nsteps
    Q = lat.Q
    # algorithmic bytes per cell and step (FP32 storage, per-cell tau):
    # forward: populations read and written, tau read; backward: the
    # recomputing forward step (the same plus the 32-byte macroscopic state
    # written) and the adjoint step (x(t-1) and a(t+1) read, a(t) written,
    # tau and the state read, the FP64 tau gradient read and written)
    fwd_b = 2 * Q * 4 + 4
    bwd_b = (2 * Q * 4 + 4 + 32) + (3 * Q * 4 + 4 + 32 + 16)
    peak, _ = _peaks()
    fwd_gbs = fwd_b * cells / (t1 - t0) / 1e9
    bwd_gbs = bwd_b * cells / (t2 - t1) / 1e9
    res = {"workload": "calibration_shear_%d_%dsteps_ckpt%d" % (L, nsteps, K), "forward_s": round(t1 - t0, 4),
           "backward_s": round(t2 - t1, 4), "backward_over_forward": round((t2 - t1) / (t1 - t0), 3),
           "mlups_forward": round(cells / (t1 - t0) / 1e6, 1),
           "mlups_adjoint_incl_recompute": round(cells / (t2 - t1) / 1e6, 1),
           "roofline": {"bound": "hbm", "unit": "GB/s", "peak": peak,
                        "forward": {"bytes_per_cell": fwd_b, "achieved": round(fwd_gbs, 1),
                                    "frac": round(fwd_gbs / peak, 4)},
                        "backward": {"bytes_per_cell": bwd_b, "achieved": round(bwd_gbs, 1),
                                     "frac": round(bwd_gbs / peak, 4)}},
           "loss": float(out["loss"].item()), "grad_tau_norm": float(out["tau"].norm().item())}
    adj.close()
    lat.close()
    return res


# Sec. 6.3: the 2-d stencil of the paper's performance table (45 vectors)
PAPER_STENCIL_45 = [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2), (3, 0), (3, 2), (3, 3), (4, 0)]


def bench_massive_order3(torch, rlbm, inputs, stream, L=512, m=5.0, steps=50, warmup=5, groups=None):
    """The fused step on the setup of the paper's only performance table
    (Taylor-Green, 512^2 periodic, third-order on-lattice massive stencil),
    in FP64 (the paper's precision) and with FP32 storage.  Without groups:
    the built-in zeta = 5 stencil (App. H column C, 49 vectors).  With the
    paper's own 45-vector stencil (groups = PAPER_STENCIL_45): it has
    non-negative order-3 weights only from m~ = 14.75 on (none at m~ = 5), so
    it runs at m~ = 15, T~ = 1; the cost of a site does not depend on the
    mass, except that FP32 storage at m~ >= 6 runs the extended-precision
    equilibrium (float-float moments, compensated contraction), which the
    1e-5 parity bar needs there.  The paper times its collide kernel alone
    on a P100 (55 MLUPS): context, not a target.  L2 is flushed before every
    timed step."""
    name = "paper_stencil45" if groups is not None else "builtin"
    out = {"workload": f"tg{L}_m{m:g}_order3_onlattice_{name}", "paper_collide_only_p100_mlups": 55.0}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    fields = [__import__("numpy").ascontiguousarray(a) for a in inputs.taylor_green(L, u0=0.1)]
    peak, _ = _peaks()
    for prec, elem in (("fp64", 8), ("fp32", 4)):
        lat = rlbm.Lattice(L, L, m=m, order=3, tau=1.0, stream="onlattice", precision=prec,
                           cuda_stream=stream.cuda_stream, groups=groups)
        lat.init(*fields)
        for _ in range(warmup):
            flush.zero_()
            lat.step(1)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            lat.step(1)
            b.record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / steps
        st = lat.sync_status(raise_on_error=False)
        gbs = 2 * lat.Q * elem * L * L / (ms * 1e-3) / 1e9
        out[prec] = {"Q": lat.Q, "ms_per_step": round(ms, 5), "mlups": round(L * L / (ms * 1e-3) / 1e6, 1),
                     "algorithmic_gbs": round(gbs, 1), "frac_of_hbm": round(gbs / peak, 4),
                     "nonphysical": st[1]}
        if prec == "fp32":
            out[prec]["equilibrium"] = "float-float moments, compensated contraction" if m >= 6.0 else "FP32"
        lat.close()
    return out


def bench_kh(torch, rlbm, inputs, stream, L=2048, steps=20, warmup=5):
    """The zeta = 1, order-3 Kelvin-Helmholtz shear layer (2048^2, +-0.3c,
    tanh width 20 cells, 1e-3 seeded perturbation, FP32 storage): zeta = m~/T~
    with m~ = T~ = 1.5, the smallest mass with a built-in order-3 stencil
    (Q = 65), tau = 0.85.  Each buffer holds 1.09 GB, more than L2, so no
    flush is needed; every step is timed with its own events."""
    m = T0 = 1.5
    fields = [__import__("numpy").ascontiguousarray(a) for a in inputs.kelvin_helmholtz(L, T0=T0)]
    lat = rlbm.Lattice(L, L, m=m, order=3, tau=0.85, precision="fp32", n_ref=1.0, T_ref=T0,
                       cuda_stream=stream.cuda_stream)
    lat.init(*fields)
    for _ in range(warmup):
        lat.step(1)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for a, b in ev:
        a.record(stream)
        lat.step(1)
        b.record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / steps
    st = lat.sync_status(raise_on_error=False)
    peak, _ = _peaks()
    gbs = 2 * lat.Q * 4 * L * L / (ms * 1e-3) / 1e9
    out = {"workload": f"kh{L}_zeta1_order3_fp32", "m": m, "T": T0, "Q": lat.Q, "ms_per_step": round(ms, 4),
           "mlups": round(L * L / (ms * 1e-3) / 1e6, 1), "algorithmic_gbs": round(gbs, 1),
           "frac_of_hbm": round(gbs / peak, 4), "full_run_s_estimate": round(10000 * ms / 1e3, 2),
           "nonphysical": st[1]}
    lat.close()
    return out


def bench_d3(torch, rlbm, inputs, stream, L=192, steps=10, warmup=3):
    """The (3+1)-d massless step, order 2 (Q = 78) and order 3 (Q = 288), in
    FP64 and with FP32 storage on the Taylor-Green flow uniform along z,
    192^3 cells (the paper's 3-d performance figure is for 192^3, zeta = 5,
    143 vectors, its collide kernel alone on a P100: 14 MLUPS; context only).
    Each buffer holds 4.1-16.3 GB, far more than L2."""
    fields = [__import__("numpy").ascontiguousarray(a) for a in inputs.taylor_green3(L, L, u0=0.2)]
    peak, _ = _peaks()
    out = {"workload": f"tg{L}^3_massless", "paper_3d_collide_only_p100_mlups": 14.0}
    for order, prec, elem in ((2, "fp64", 8), (2, "fp32", 4), (3, "fp64", 8), (3, "fp32", 4)):
        key = prec if order == 2 else f"order3_{prec}"
        lat = rlbm.Lattice3(L, L, L, tau=0.8, precision=prec, cuda_stream=stream.cuda_stream, order=order)
        lat.init(*fields)
        lat.step(warmup)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        for a, b in ev:
            a.record(stream)
            lat.step(1)
            b.record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / steps
        rc, bad = lat.sync_status()
        gbs = 2 * lat.Q * elem * L ** 3 / (ms * 1e-3) / 1e9
        out[key] = {"Q": lat.Q, "ms_per_step": round(ms, 3), "mlups": round(L ** 3 / (ms * 1e-3) / 1e6, 1),
                     "algorithmic_gbs": round(gbs, 1), "frac_of_hbm": round(gbs / peak, 4), "nonphysical": bad}
        lat.close()
    return out


def _time_steps(torch, lat, stream, steps, warmup):
    """Mean CUDA-event time of one step (ms), each step timed on its own."""
    lat.step(warmup)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for a, b in ev:
        a.record(stream)
        lat.step(1)
        b.record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev) / steps


def bench_forcing_walls(torch, rlbm, inputs, stream, nx=4096, ny=1024, m=5.0, steps=10, warmup=3):
    """The forcing-validation setup of Sec. 8.1 at a size that exercises the
    bandwidth: a massive gas (m~ = 5, order 2, Q = 29) between equilibrium
    walls at the first and last column, periodic in y, driven by the
    gravity-like force g = (0, 1e-8) (forcing scheme B), FP64 and FP32
    storage, on the orbit-symmetric kernel with the force and wall terms.
    Each buffer holds 3.9 (FP64) or 1.9 GB (FP32), more than L2."""
    import numpy as np
    peak, _ = _peaks()
    out = {"workload": f"channel{nx}x{ny}_m{m:g}_eqwalls_force"}
    one = np.ones((ny, nx))
    z = np.zeros((ny, nx))
    for prec, elem in (("fp64", 8), ("fp32", 4)):
        lat = rlbm.Lattice(nx, ny, m=m, tau=1.0, boundary="eqwall_x", precision=prec, g=(0.0, 1e-8),
                           cuda_stream=stream.cuda_stream)
        lat.init(one, z, z.copy(), one)
        ms = _time_steps(torch, lat, stream, steps, warmup)
        rc, bad = lat.sync_status(raise_on_error=False)
        gbs = 2 * lat.Q * elem * nx * ny / (ms * 1e-3) / 1e9
        out[prec] = {"Q": lat.Q, "ms_per_step": round(ms, 4), "mlups": round(nx * ny / (ms * 1e-3) / 1e6, 1),
                     "algorithmic_gbs": round(gbs, 1), "frac_of_hbm": round(gbs / peak, 4), "nonphysical": bad}
        lat.close()
    return out


def bench_d1(torch, rlbm, inputs, stream, nx=1 << 24, order=3, steps=10, warmup=3):
    """The native (1+1)-d massless gas (App. H (1+1)-d table, order 3,
    Q = 6) on 2^24 cells with a smooth density and temperature wave and a
    flow of 0.2c, FP64 and FP32 storage.  Each buffer holds 0.8 (FP64) or
    0.4 GB (FP32), more than L2."""
    import numpy as np
    peak, _ = _peaks()
    x = 2 * np.pi * np.arange(nx) / nx
    fields = [np.ascontiguousarray(a) for a in (1 + 0.1 * np.sin(x), 0.2 * np.cos(x), 1 + 0.1 * np.cos(x))]
    out = {"workload": f"d1_wave_{nx}_order{order}"}
    Q = 2 * order
    for prec, elem in (("fp64", 8), ("fp32", 4)):
        lat = rlbm.Lattice1(nx, order=order, tau=0.9, precision=prec, cuda_stream=stream.cuda_stream)
        lat.init(*fields)
        ms = _time_steps(torch, lat, stream, steps, warmup)
        rc, bad = lat.sync_status()
        gbs = 2 * Q * elem * nx / (ms * 1e-3) / 1e9
        out[prec] = {"Q": Q, "ms_per_step": round(ms, 4), "mlups": round(nx / (ms * 1e-3) / 1e6, 1),
                     "algorithmic_gbs": round(gbs, 1), "frac_of_hbm": round(gbs / peak, 4), "nonphysical": bad}
        lat.close()
    return out


def bench_tg_viscosity(rlbm, inputs, L=512, tau=1.0, u0=0.1, steps=5000, every=100):
    """Config-2 viscosity fit: the 512^2 Taylor-Green vortex (order 2, FP32
    storage) run for `steps` steps with the amplitude of the initial pattern
    sampled every `every` steps; a vortex decays at 2 eta k^2 / (eps + P),
    eps + P = 3 P (massless).  Bilinear lambda = 1 has delta x = 1
    (k = 2 pi / L), on-lattice delta x = 1/5 (k = 10 pi / L; fitted over its
    first 1.5 e-folds).  eta / P is compared with the CE value (3/4)(tau - 1/2)
    (App. C with the half-step lattice shift): a measurement, not a pin --
    order 2 and bilinear interpolation both move it."""
    import numpy as np
    n, ux, uy, T = [np.ascontiguousarray(a) for a in inputs.taylor_green(L, u0=u0)]
    px, py = ux / u0, uy / u0
    out = {}
    for mode, lam, k in (("bilinear", 1.0, 2 * np.pi / L), ("onlattice", 0.0, 10 * np.pi / L)):
        lat = rlbm.Lattice(L, L, tau=tau, stream=mode, lam=lam, precision="fp32")
        lat.init(n, ux, uy, T)
        guess = (tau - 0.5) * k * k / 2
        t_hi = min(steps, int(1.5 / guess))
        ts, amps, t = [], [], 0
        while t < t_hi:
            lat.step(every)
            t += every
            m = lat.moments()
            ts.append(t)
            amps.append(float(np.sum(m["ux"] * px + m["uy"] * py) / np.sum(px * px + py * py)))
        lat.close()
        sel = [i for i, tt in enumerate(ts) if tt >= 0.1 * t_hi]
        rate = -np.polyfit(np.array(ts)[sel], np.log(np.array(amps)[sel]), 1)[0]
        eta = 3 * rate / (2 * k * k)
        out[mode] = {"steps": t_hi, "decay_rate_per_step": float(rate), "eta_over_P": round(float(eta), 5),
                     "ce_eta_over_P": 0.75 * (tau - 0.5), "ratio_to_ce": round(float(eta / (0.75 * (tau - 0.5))), 4),
                     "amplitude_final_over_initial": round(amps[-1], 5)}
    out["note"] = ("order-2 stencil, whose shear viscosity is anisotropic: the first-order coefficient is "
                   "0.98 (tau - 1/2) P along the lattice axes and 0.52 (tau - 1/2) P along the diagonals, "
                   "where the Taylor-Green wavevectors lie (their mean is the CE 3/4); the on-lattice fit "
                   "measures the diagonal value, the bilinear fit adds the interpolation's diffusion")
    return out


def bench_reference(args, wl):
    """The FP64 CPU oracle as the reference arm, on the host cores."""
    budget = 150.0
    L, _ = oracle_sample_size(wl, budget, args.steps + args.warmup)
    cores = host_cores()
    reports, rate = run_oracle(L, args.steps, args.warmup, wl, procs=cores)
    value = rate / 1e6
    t = max(sum(r["times"]) for r in reports)
    cpu = {"value": round(value, 4), "unit": METRIC, "cores": cores, "kind": "oracle",
           "sample": "each step one oracle time step of the Taylor-Green configuration on a %dx%d grid, in "
                     "each of %d single-threaded worker processes at once (one per host core)" % (L, L, cores)}
    line = {"metric": METRIC, "value": round(value, 4), "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": wl["workload"], "nx": L, "ny": L, "sample_of": [wl["L"], wl["L"]]},
            "cpu_baseline": cpu, "e2e": {"value": round(value, 4), "unit": METRIC, "h2d_bytes_per_step": 0,
                                         "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
