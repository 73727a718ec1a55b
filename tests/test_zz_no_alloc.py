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


class _DeviceView:
    """Exposes a raw device buffer (borrowed) to torch via __cuda_array_interface__."""

    def __init__(self, ptr, nbytes):
        self.__cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (ptr, False),
                                         "version": 3, "strides": None}


def _copy_of_handle_buffer(lat):
    """A caller-owned copy (halo included) of the handle's current f*(t) buffer."""
    import torch
    cur, prev, elem, plane, layout = lat.buffers()
    nbytes = lat.Q * plane * elem
    view = torch.as_tensor(_DeviceView(cur, nbytes), device="cuda")
    return view.clone(), elem


def _noalloc(rl, params, a, b, nsteps, tau=None):
    counts = (ctypes.c_longlong * max(nsteps, 1))()
    rc = rl.lib().rlbm_step_noalloc(ctypes.byref(params), a.data_ptr(), b.data_ptr(),
                                    None if tau is None else tau.data_ptr(), nsteps, counts)
    return rc, list(counts)[:nsteps]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_noalloc_matches_handle_step_on_two_calls(rl, precision, tol):
    import torch
    nx, ny = 40, 24
    fields = [np.ascontiguousarray(a) for a in inputs.random_smooth(nx, ny, seed=21, umax=0.3)]
    kw = dict(precision=precision, stream="bilinear", lam=1.0, tau=0.9)
    stream = torch.cuda.current_stream().cuda_stream
    lat = rl.Lattice(nx, ny, cuda_stream=stream, **kw)
    lat.init(*fields)
    torch.cuda.synchronize()
    a, elem = _copy_of_handle_buffer(lat)
    b = torch.zeros_like(a)
    params, keep = rl.make_params(nx, ny, cuda_stream=stream, **kw)
    ref = np.empty(1)
    # call 1: a -> b ; call 2: b -> a.  Compare with rlbm_step through the
    # handle, element by element over the whole buffer (halo included).
    for src, dst in ((a, b), (b, a)):
        rc, counts = _noalloc(rl, params, src, dst, 1)
        assert rc == 0 and counts == [0]
        lat.step(1)
        torch.cuda.synchronize()
        ref, _ = _copy_of_handle_buffer(lat)
        dt = torch.float64 if elem == 8 else torch.float32
        got, want = dst.view(dt).double(), ref.view(dt).double()
        err = float((got - want).abs().max() / want.abs().max())
        assert err <= tol, err


def test_noalloc_multi_step_and_limits(rl):
    import torch
    nx, ny = 32, 16
    fields = [np.ascontiguousarray(a) for a in inputs.random_smooth(nx, ny, seed=22)]
    stream = torch.cuda.current_stream().cuda_stream
    lat = rl.Lattice(nx, ny, precision="fp64", cuda_stream=stream)
    lat.init(*fields)
    torch.cuda.synchronize()
    a, elem = _copy_of_handle_buffer(lat)
    b = torch.zeros_like(a)
    params, keep = rl.make_params(nx, ny, precision="fp64", cuda_stream=stream)
    rc, counts = _noalloc(rl, params, a, b, 3)           # odd: result in b
    assert rc == 0 and counts == [0, 0, 0]
    lat.step(3)
    torch.cuda.synchronize()
    ref, _ = _copy_of_handle_buffer(lat)
    got, want = b.view(torch.float64), ref.view(torch.float64)
    assert float((got - want).abs().max() / want.abs().max()) <= 1e-12
    # sizes beyond the scratch array are rejected before any device work
    rc = rl.lib().rlbm_step_noalloc(ctypes.byref(params), a.data_ptr(), b.data_ptr(), None, 1025, None)
    assert rc == -1
    assert "1024" in rl.lib().rlbm_last_error(None).decode()
