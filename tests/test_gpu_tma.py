"""The TMA-staged step kernels against the direct-load kernel: both evaluate
the same expressions in the same order, so populations must agree bit for
bit after several steps, on grids with ragged tiles and at full size."""
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


@pytest.mark.parametrize("stream,lam", [("onlattice", 0.0), ("bilinear", 1.0)])
@pytest.mark.parametrize("nx,ny", [(512, 512), (100, 37), (40, 24), (64, 9)])
def test_tma_kernels_match_direct_kernel_bitwise(rl, stream, lam, nx, ny):
    fields = [np.ascontiguousarray(a) for a in inputs.random_smooth(nx, ny, seed=nx + ny, umax=0.3)]
    out = {}
    for k in ("direct", "tma_32x8", "tma_32x4"):
        lat = rl.Lattice(nx, ny, stream=stream, lam=lam, tau=0.8, precision="fp32")
        lat.set_step_kernel(k)
        assert lat.step_kernel == k
        lat.init(*fields)
        lat.step(7)
        assert lat.sync_status()[0] == 0
        out[k] = lat.populations()
        lat.close()
    for k in ("tma_32x8", "tma_32x4"):
        assert np.array_equal(out[k], out["direct"]), (k, np.abs(out[k] - out["direct"]).max())


def test_kernel_selection(rl):
    lat = rl.Lattice(512, 512, stream="bilinear", lam=1.0, precision="fp32")
    assert lat.step_kernel == "direct"
    lat.set_step_kernel("tma_32x4")
    assert lat.step_kernel == "tma_32x4"
    lat.close()
    for kw in (dict(nx=3, ny=2, precision="fp32"), dict(nx=64, ny=64, precision="fp64"),
               dict(nx=64, ny=64, precision="fp32", m=1.0)):
        lat = rl.Lattice(**kw)
        assert lat.step_kernel == "direct"
        with pytest.raises(rl.RLBMError):
            lat.set_step_kernel("tma_32x8")
        lat.close()
