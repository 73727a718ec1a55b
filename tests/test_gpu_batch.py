"""Batched steps (rlbm_batch_*), persistent kernels and per-instance chains:
bitwise equality with the plain step on every instance, bounded grid-barrier
timeout, autotuner."""
import numpy as np
import pytest

from paper_1909_04502_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rl():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_04502_gb300 import build, rlbm
    build.build()
    return rlbm


INSTANCES = [
    dict(nx=37, ny=23, tau=0.7),
    dict(nx=64, ny=64, tau=1.3, m=1.0),
    dict(nx=50, ny=70, tau=1.9, m=10.0),
    dict(nx=96, ny=40, tau=0.9),
    dict(nx=33, ny=33, tau=1.1, m=1.0),
    dict(nx=70, ny=21, tau=0.65, m=10.0),
    dict(nx=1, ny=40, tau=1.0),
    dict(nx=45, ny=30, tau=0.8, stream="bilinear", lam=1.0),
    dict(nx=20, ny=52, tau=1.2, stream="bilinear", lam=1.0),
]


def _fields(c, seed):
    return [np.ascontiguousarray(a) for a in inputs.random_smooth(c["nx"], c["ny"], seed=seed, umax=0.2)]


def test_batched_step_is_bitwise_equal_to_plain(rl):
    batch = rl.Batch([dict(c, precision="fp32") for c in INSTANCES])
    plain = []
    for i, c in enumerate(INSTANCES):
        c = dict(c)
        nx, ny = c.pop("nx"), c.pop("ny")
        lat = rl.Lattice(nx, ny, precision="fp32", **c)
        f = _fields(INSTANCES[i], seed=100 + i)
        lat.init(*f)
        batch[i].init(*f)
        plain.append(lat)
    for shape in (0, 1, 2, 0):
        gmax = batch.info()["grid_max"][shape] if shape < 2 else 0
        batch.config(shape, max(1, gmax // 3))
        batch.step(7)
        for lat in plain:
            lat.step(7)
        rc, nonphys = batch.sync_status()
        assert rc == 0 and nonphys == 0
        for i, lat in enumerate(plain):
            a = batch[i].populations()
            b = lat.populations()
            assert np.array_equal(a, b), (shape, i, np.abs(a - b).max())
            assert batch[i].t == lat.t
    # the fields of every instance agree too
    for i, lat in enumerate(plain):
        ma, mb = batch[i].moments(), lat.moments()
        for k in ("n", "ux", "uy", "T"):
            assert np.array_equal(ma[k], mb[k])
    batch.close()


@pytest.mark.parametrize("shape", [0, 2])
def test_mixed_batch_and_handle_steps_stay_consistent(rl, shape):
    """An instance stepped through its own handle between batched steps: the
    persistent kernels read its buffer parity from the descriptors, the
    chains take a graph captured for the new parities."""
    batch = rl.Batch([dict(c, precision="fp32") for c in INSTANCES[:3]])
    batch.config(shape, max(1, batch.info()["grid_max"][0] // 2))
    ref = []
    for i, c in enumerate(INSTANCES[:3]):
        f = _fields(c, seed=7 + i)
        batch[i].init(*f)
        cc = dict(c)
        nx, ny = cc.pop("nx"), cc.pop("ny")
        lat = rl.Lattice(nx, ny, precision="fp32", **cc)
        lat.init(*f)
        ref.append(lat)
    batch.step(2)
    batch[1].step(1)          # one instance stepped through its own handle
    batch.step(3)
    batch.step(3)
    for i, lat in enumerate(ref):
        lat.step(8 + (1 if i == 1 else 0))
        assert np.array_equal(batch[i].populations(), lat.populations())
    batch.close()


def test_barrier_timeout_is_reported_not_hung(rl):
    """A wait limit of one poll makes the grid barrier give up: the kernel
    leaves, the host reads RLBM_ERR_TIMEOUT, and the context stays usable."""
    batch = rl.Batch([dict(nx=256, ny=256, precision="fp32"), dict(nx=128, ny=96, precision="fp32", m=1.0)])
    for i in range(len(batch)):
        batch[i].init(*_fields(dict(nx=batch[i].nx, ny=batch[i].ny), seed=i))
    batch.config(0, batch.info()["grid_max"][0])
    batch.set_spin_limit(1)
    batch.step(4)
    rc, _ = batch.sync_status(raise_on_error=False)
    assert rc == -5
    # recovery: a normal limit works again and the device is healthy
    batch.set_spin_limit(1 << 24)
    batch[0].init(*_fields(dict(nx=256, ny=256), seed=0))
    batch.step(2)
    rc, _ = batch.sync_status(raise_on_error=False)
    assert rc == 0
    lat = rl.Lattice(32, 32, precision="fp32")
    lat.init(*_fields(dict(nx=32, ny=32), seed=3))
    lat.step(2)
    assert lat.sync_status()[0] == 0
    batch.close()


def test_autotuner_picks_a_valid_configuration(rl):
    batch = rl.Batch([dict(c, precision="fp32") for c in INSTANCES])
    shape, grid, ms = batch.tune(trial_steps=2)
    info = batch.info()
    assert shape in (0, 1, 2) and ms > 0
    assert (0 < grid <= info["grid_max"][shape]) if shape < 2 else grid == 0
    assert info["tile_shape"] == shape and info["grid"] == grid
    batch.close()


def test_unsupported_batch_configurations_are_rejected(rl):
    with pytest.raises(rl.RLBMError):
        rl.Batch([dict(nx=32, ny=32, precision="fp64")])
    with pytest.raises(rl.RLBMError):
        rl.Batch([dict(nx=32, ny=32, precision="fp32", order=3)])
