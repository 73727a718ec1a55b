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


def _noalloc_vs_handle(rl, nx, ny, fields, kw, nsteps=2, tau=None):
    """Relative L-inf gap between rlbm_step_noalloc and rlbm_step of a handle
    created with the same parameters, over the whole buffer (halo included),
    after nsteps steps from the handle's initial state."""
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    lat = rl.Lattice(nx, ny, cuda_stream=stream, **kw)
    lat.init(*fields)
    if tau is not None:
        lat.set_tau_field(tau)
    torch.cuda.synchronize()
    a, elem = _copy_of_handle_buffer(lat)
    b = torch.zeros_like(a)
    params, keep = rl.make_params(nx, ny, cuda_stream=stream, **kw)
    dt = torch.float64 if elem == 8 else torch.float32
    tau_dev = None
    if tau is not None:
        tau_dev = torch.as_tensor(tau, device="cuda", dtype=dt).contiguous()
    rc, counts = _noalloc(rl, params, a, b, nsteps, tau_dev)
    assert rc == 0 and counts == [0] * nsteps
    lat.step(nsteps)
    torch.cuda.synchronize()
    ref, _ = _copy_of_handle_buffer(lat)
    got = (b if nsteps % 2 else a).view(dt).double()
    want = ref.view(dt).double()
    lat.close()
    return float((got - want).abs().max() / want.abs().max())


def test_noalloc_tables_follow_force_and_wall_temperatures(rl):
    """Calls in one process whose parameters differ only in the force or in
    the wall temperatures must each run with their own tables: every call is
    compared with a handle created with the same parameters."""
    nx, ny = 36, 20
    fields = [np.ascontiguousarray(a) for a in inputs.random_smooth(nx, ny, seed=23, umax=0.2)]
    base = dict(m=5.0, order=2, precision="fp64", tau=0.9)
    for extra in (dict(),
                  dict(g=(0.0, 1e-6)),
                  dict(g=(2e-6, -1e-6)),
                  dict(boundary="eqwall_x", wall_T=(1.01, 0.99)),
                  dict(boundary="eqwall_x", wall_T=(1.03, 0.97)),
                  dict()):
        err = _noalloc_vs_handle(rl, nx, ny, fields, dict(base, **extra))
        assert err <= 1e-12, (extra, err)


def test_noalloc_order3_tau_field(rl):
    """Order-3 massless stencil (Q = 44) with a per-cell relaxation time, in
    both precisions, against the handle path."""
    nx, ny = 30, 18
    fields = [np.ascontiguousarray(a) for a in inputs.random_smooth(nx, ny, seed=24, umax=0.2)]
    rng = np.random.default_rng(24)
    tau = np.ascontiguousarray(0.7 + 0.6 * rng.random((ny, nx)))
    for precision, tol in (("fp64", 1e-12), ("fp32", 1e-5)):
        kw = dict(order=3, precision=precision, tau_mode="field")
        err = _noalloc_vs_handle(rl, nx, ny, fields, kw, nsteps=3, tau=tau)
        assert err <= tol, (precision, err)


def test_noalloc_high_mass_order3_extended_equilibrium(rl):
    """Order 3, FP32 storage, m~ = 10: both paths run the extended-precision
    equilibrium and agree bit for bit."""
    nx, ny = 34, 22
    fields = [np.ascontiguousarray(a) for a in inputs.random_smooth(nx, ny, seed=25, umax=0.2)]
    err = _noalloc_vs_handle(rl, nx, ny, fields, dict(m=10.0, order=3, precision="fp32"), nsteps=3)
    assert err == 0.0, err
