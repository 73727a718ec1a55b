"""rlbm_step_noalloc: the step for callers that cannot allocate device memory.

Such callers (a plugin running on device memory owned by its host
application, or code that must not allocate while it records work) pass
their own population buffers; the step's scratch lives in a file-scope device
array.  This test calls the entry point through the C ABI and checks it
against the handle API's rlbm_step on two calls in a row.  It is collected
last so that a run stopping at the first failure has run every other test.
"""
import ctypes

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


def _noalloc(rl, params, a, b, nsteps, tau=None):
    counts = (ctypes.c_longlong * max(nsteps, 1))()
    rc = rl.lib().rlbm_step_noalloc(ctypes.byref(params), a.data_ptr(), b.data_ptr(),
                                    None if tau is None else tau.data_ptr(), nsteps, counts)
    return rc, list(counts)[:nsteps]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_noalloc_matches_handle_step_on_two_calls(rl, precision, tol):
    import torch
    nx, ny = 40, 24                        # nx*ny is a multiple of 32: plane == nx*ny
    fields = [np.ascontiguousarray(a) for a in inputs.random_smooth(nx, ny, seed=21, umax=0.3)]
    kw = dict(precision=precision, stream="bilinear", lam=1.0, tau=0.9, n_ref=0.0)
    stream = torch.cuda.current_stream().cuda_stream
    lat = rl.Lattice(nx, ny, cuda_stream=stream, **kw)
    lat.init(*fields)
    Q = lat.Q
    f0 = torch.empty((Q, ny, nx), dtype=torch.float64, device="cuda")
    rc = rl.lib().rlbm_get_populations(lat.h, f0.data_ptr(), 1)
    assert rc == 0
    dt = torch.float64 if precision == "fp64" else torch.float32
    a = f0.to(dt).contiguous()
    b = torch.zeros_like(a)
    params, keep = rl.make_params(nx, ny, cuda_stream=stream, **kw)

    ref = torch.empty_like(f0)
    # call 1: a -> b ; call 2: b -> a
    for src, dst in ((a, b), (b, a)):
        rc, counts = _noalloc(rl, params, src, dst, 1)
        assert rc == 0 and counts == [0]
        lat.step(1)
        assert rl.lib().rlbm_get_populations(lat.h, ref.data_ptr(), 1) == 0
        torch.cuda.synchronize()
        got = dst.double()
        err = float((got - ref).abs().max() / ref.abs().max())
        assert err <= tol, err


def test_noalloc_multi_step_and_limits(rl):
    import torch
    nx, ny = 32, 16
    fields = [np.ascontiguousarray(a) for a in inputs.random_smooth(nx, ny, seed=22)]
    stream = torch.cuda.current_stream().cuda_stream
    lat = rl.Lattice(nx, ny, precision="fp64", cuda_stream=stream)
    lat.init(*fields)
    f = torch.empty((lat.Q, ny, nx), dtype=torch.float64, device="cuda")
    assert rl.lib().rlbm_get_populations(lat.h, f.data_ptr(), 1) == 0
    a, b = f.clone(), torch.zeros_like(f)
    params, keep = rl.make_params(nx, ny, precision="fp64", cuda_stream=stream)
    rc, counts = _noalloc(rl, params, a, b, 3)           # odd: result in b
    assert rc == 0 and counts == [0, 0, 0]
    lat.step(3)
    assert rl.lib().rlbm_get_populations(lat.h, f.data_ptr(), 1) == 0
    torch.cuda.synchronize()
    assert float((b - f).abs().max() / f.abs().max()) <= 1e-12
    # sizes beyond the scratch array are rejected before any device work
    rc = rl.lib().rlbm_step_noalloc(ctypes.byref(params), a.data_ptr(), b.data_ptr(), None, 1025, None)
    assert rc == -1
    assert "1024" in rl.lib().rlbm_last_error(None).decode()
