"""Parity at full size on sampled cells: the oracle recomputes single cells
(one pull step and one collision on the patch of post-collision populations
around the cell, read from device memory) where running it on the whole grid
would take too long.  Covers the largest grid the 32-bit layout accepts and
the full 64-instance tau-sweep through the batched kernels."""
import numpy as np
import pytest

from paper_1909_04502_gb300 import inputs
from tests.cases import device_patch, oracle_center_update, oracle_quadrature, permutation

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rl():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_04502_gb300 import build, rlbm
    build.build()
    return rlbm


def _sampled_parity(rl, lat, quad, idx, cells, tau, step, R, tol=1e-5, stream="onlattice", lam=None):
    patches = [device_patch(lat, cx, cy, R, quad, idx) for cx, cy in cells]
    step()
    for (cx, cy), fp in zip(cells, patches):
        want = oracle_center_update(quad, fp, tau, stream, lam)
        got = device_patch(lat, cx, cy, 0, quad, idx)[:, 0, 0]
        err = np.abs(got - want).max() / np.abs(want).max()
        assert err <= tol, (cx, cy, err)


def test_largest_grid_sampled_cells(rl):
    """8192^2, FP32 storage, massless order 2 on-lattice: Q * plane = 1.88e9
    elements, just under the 2^31 the layout's 32-bit offsets allow (the last
    plane starts at 1.8e9).  A 9000^2 grid is refused before any allocation."""
    import torch
    with pytest.raises(rl.RLBMError) as exc:
        rl.Lattice(9000, 9000, precision="fp32")
    assert exc.value.code == -2
    L = 8192
    lat = rl.Lattice(L, L, precision="fp32", tau=0.8)
    _, _, _, plane, _ = lat.buffers()
    assert lat.Q * plane < 2 ** 31 and (lat.Q - 1) * plane > 1.7e9
    lat.init(*[np.ascontiguousarray(a) for a in inputs.random_smooth(L, L, seed=41, umax=0.3)])
    torch.cuda.synchronize()
    quad = oracle_quadrature(0.0, 2)
    idx = permutation(lat.n, lat.p, quad)
    cells = [(0, 0), (L - 1, L - 1), (L - 1, 0), (0, L - 1), (4097, 123), (31, 8190), (5000, 6000)]
    _sampled_parity(rl, lat, quad, idx, cells, 0.8, lambda: lat.step(1), R=5)
    assert lat.sync_status()[0] == 0
    lat.close()


def test_tau_sweep_batch_sampled_cells(rl):
    """The 64-run tau-sweep (sides 64..1024, seed 1909, zeta round-robin over
    0, 1, 10) advanced one step by the batched kernels; sampled cells of runs
    of every mass against the oracle."""
    import torch
    runs = inputs.sweep(count=64, seed=1909)
    cfgs = [dict(nx=r["side"], ny=r["side"], tau=r["tau"], m=r["zeta"], precision="fp32") for r in runs]
    batch = rl.Batch(cfgs)
    for i, r in enumerate(runs):
        batch[i].init(*[np.ascontiguousarray(a) for a in inputs.shear_wave(r["side"], r["side"], amp=0.05)])
    torch.cuda.synchronize()
    rng = np.random.default_rng(7)
    checks = []
    for i in range(6):                      # zeta 0, 1, 10, 0, 1, 10
        lat, r = batch[i], runs[i]
        d = rl.plan(nx=r["side"], ny=r["side"], m=r["zeta"])
        quad = oracle_quadrature(r["zeta"], 2, d["n"], d["v0"])
        idx = permutation(lat.n, lat.p, quad)
        R = int(np.ceil(np.abs(quad.n).max())) + 1
        cells = [(0, 0), tuple(int(v) for v in rng.integers(0, r["side"], 2))]
        checks.append((lat, quad, idx, cells, r["tau"], R, [device_patch(lat, cx, cy, R, quad, idx)
                                                            for cx, cy in cells]))
    batch.step(1)
    rc, _ = batch.sync_status()
    assert rc == 0
    for lat, quad, idx, cells, tau, R, patches in checks:
        for (cx, cy), fp in zip(cells, patches):
            want = oracle_center_update(quad, fp, tau)
            got = device_patch(lat, cx, cy, 0, quad, idx)[:, 0, 0]
            assert np.abs(got - want).max() / np.abs(want).max() <= 1e-5, (lat.Q, cx, cy)
    batch.close()
