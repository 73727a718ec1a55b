"""Thin Python binding of the C ABI in include/rlbm.h (argument marshalling only).

Every step of the RLBM update runs in the CUDA library ``librlbm.so`` built
in-tree by ``paper_1909_04502_gb300.build``.  There is no CPU fallback: if the
library is missing or cannot be loaded, every call raises.  PyTorch supplies
device memory and the CUDA stream; numpy arrays are accepted for host data.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "librlbm.so")

RLBM_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "UNSUPPORTED", -3: "CUDA", -4: "NONPHYSICAL", -5: "TIMEOUT",
          -6: "OOM", -7: "QUADRATURE"}
QUAD = {"massless": 0, "massive": 1, "custom": 2}
BC = {"periodic": 0, "freeflow_x": 1, "eqwall_x": 2}
PREC = {"fp64": 0, "fp32": 1}
STREAM = {"onlattice": 0, "bilinear": 1}
TAU = {"const": 0, "field": 1, "eta_over_s": 2}


class RLBMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int), ("m", ctypes.c_double), ("order", ctypes.c_int),
        ("quadrature", ctypes.c_int), ("groups", ctypes.POINTER(ctypes.c_int)),
        ("n_groups", ctypes.c_int), ("v0", ctypes.c_double),
        ("custom_table", ctypes.POINTER(ctypes.c_double)), ("custom_Q", ctypes.c_int),
        ("tau_mode", ctypes.c_int), ("tau", ctypes.c_double), ("eta_over_s", ctypes.c_double),
        ("kappa", ctypes.c_double), ("boundary", ctypes.c_int), ("nx", ctypes.c_int),
        ("ny", ctypes.c_int), ("precision", ctypes.c_int), ("stream_mode", ctypes.c_int),
        ("lam", ctypes.c_double), ("n_ref", ctypes.c_double), ("T_ref", ctypes.c_double),
        ("stream", ctypes.c_void_p), ("gx", ctypes.c_double), ("gy", ctypes.c_double),
        ("wall_T", ctypes.c_double * 2),
    ]


_LIB = None
_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int)
_VP = ctypes.c_void_p
_H = ctypes.c_void_p

SIGNATURES = {
    "rlbm_default_params": (None, [ctypes.POINTER(Params)]),
    "rlbm_create": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.POINTER(_H)]),
    "rlbm_plan": (ctypes.c_int, [ctypes.POINTER(Params), _IP, _IP, _IP, _DP, _DP, _DP, _DP]),
    "rlbm3_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                    ctypes.c_int, _VP, ctypes.POINTER(_H)]),
    "rlbm3_destroy": (None, [_H]),
    "rlbm3_plan": (ctypes.c_int, [ctypes.c_int, _IP, _IP, _IP, _DP, _DP, _DP]),
    "rlbm3_stencil": (ctypes.c_int, [_H, _IP, _IP, _DP, _DP]),
    "rlbm3_init": (ctypes.c_int, [_H, _VP, _VP, _VP, _VP, _VP, ctypes.c_int]),
    "rlbm3_step": (ctypes.c_int, [_H, ctypes.c_int]),
    "rlbm3_moments": (ctypes.c_int, [_H, _VP, ctypes.c_int]),
    "rlbm3_get_populations": (ctypes.c_int, [_H, _DP]),
    "rlbm3_sync_status": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_longlong)]),
    "rlbm3_last_error": (ctypes.c_char_p, [_H]),
    "rlbm1_plan": (ctypes.c_int, [ctypes.c_int, _IP, _IP, _DP, _DP, _DP]),
    "rlbm1_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, _DP, ctypes.c_int,
                                    _VP, ctypes.POINTER(_H)]),
    "rlbm1_destroy": (None, [_H]),
    "rlbm1_stencil": (ctypes.c_int, [_H, _IP, _IP, _DP, _DP]),
    "rlbm1_init": (ctypes.c_int, [_H, _VP, _VP, _VP, ctypes.c_int]),
    "rlbm1_step": (ctypes.c_int, [_H, ctypes.c_int]),
    "rlbm1_moments": (ctypes.c_int, [_H, _VP, ctypes.c_int]),
    "rlbm1_get_populations": (ctypes.c_int, [_H, _DP]),
    "rlbm1_sync_status": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_longlong)]),
    "rlbm1_last_error": (ctypes.c_char_p, [_H]),
    "rlbm_destroy": (None, [_H]),
    "rlbm_init": (ctypes.c_int, [_H, _VP, _VP, _VP, _VP, ctypes.c_int]),
    "rlbm_set_tau_field": (ctypes.c_int, [_H, _VP, ctypes.c_int]),
    "rlbm_step": (ctypes.c_int, [_H, ctypes.c_int]),
    "rlbm_set_step_kernel": (ctypes.c_int, [_H, ctypes.c_int]),
    "rlbm_adjoint_step": (ctypes.c_int, [_H, _VP, _VP, _VP, _VP]),
    "rlbm_step_kernel": (ctypes.c_int, [_H]),
    "rlbm_moments": (ctypes.c_int, [_H, _VP, _VP, _VP, _VP, _VP, _VP, _VP, ctypes.c_int]),
    "rlbm_get_populations": (ctypes.c_int, [_H, _VP, ctypes.c_int]),
    "rlbm_set_populations": (ctypes.c_int, [_H, _VP, ctypes.c_int]),
    "rlbm_stencil": (ctypes.c_int, [_H, _IP, _IP, _DP, _DP]),
    "rlbm_time": (ctypes.c_longlong, [_H]),
    "rlbm_sync_status": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_longlong)]),
    "rlbm_set_stream": (ctypes.c_int, [_H, _VP]),
    "rlbm_buffers": (ctypes.c_int, [_H, ctypes.POINTER(_VP), ctypes.POINTER(_VP), _IP,
                                    ctypes.POINTER(ctypes.c_longlong), _IP]),
    "rlbm_step_noalloc": (ctypes.c_int, [ctypes.POINTER(Params), _VP, _VP, _VP, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_longlong)]),
    "rlbm_batch_create": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.c_int, ctypes.POINTER(_VP)]),
    "rlbm_batch_destroy": (None, [_VP]),
    "rlbm_batch_size": (ctypes.c_int, [_VP]),
    "rlbm_batch_handle": (_VP, [_VP, ctypes.c_int]),
    "rlbm_batch_step": (ctypes.c_int, [_VP, ctypes.c_int]),
    "rlbm_batch_config": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int]),
    "rlbm_batch_tune": (ctypes.c_int, [_VP, ctypes.c_int, _IP, _IP, ctypes.POINTER(ctypes.c_float)]),
    "rlbm_batch_info": (ctypes.c_int, [_VP, _IP, _IP, _IP, ctypes.POINTER(ctypes.c_longlong)]),
    "rlbm_batch_set_spin_limit": (ctypes.c_int, [_VP, ctypes.c_longlong]),
    "rlbm_batch_sync_status": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_longlong)]),
    "rlbm_batch_last_error": (ctypes.c_char_p, [_VP]),
    "rlbm_adjoint_create": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_VP)]),
    "rlbm_adjoint_destroy": (None, [_VP]),
    "rlbm_adjoint_forward": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, ctypes.c_int]),
    "rlbm_adjoint_backward": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, _VP, _VP, _VP, _VP, ctypes.c_int]),
    "rlbm_adjoint_last_error": (ctypes.c_char_p, [_VP]),
    "rlbm_convert_f32_f64": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP, _VP, ctypes.c_int, _VP]),
    "rlbm_last_error": (ctypes.c_char_p, [_H]),
    "rlbm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
}


def lib():
    """Load librlbm.so (built in-tree).  Raises if it is absent: the library
    has no fallback path."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIBPATH):
            raise RuntimeError("librlbm.so is not built; run paper_1909_04502_gb300.build.build()")
        L = ctypes.CDLL(LIBPATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name, None)
            if fn is None:
                continue
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def _check(rc, handle=None):
    if rc != RLBM_OK:
        msg = lib().rlbm_last_error(handle).decode()
        raise RLBMError(rc, msg)


def make_params(nx, ny, m=0.0, order=2, quadrature=None, groups=None, v0=0.0, custom=None,
                tau=1.0, tau_mode="const", eta_over_s=0.0, kappa=0.0, boundary="periodic",
                precision="fp32", stream="onlattice", lam=0.0, n_ref=1.0, T_ref=1.0,
                cuda_stream=None, g=(0.0, 0.0), wall_T=(0.0, 0.0), d=2):
    """Fill an rlbm_params struct; returns (params, keepalive) -- the second
    item holds arrays the struct points to.  d = 1 runs a one-dimensional
    problem on the d = 2 stencil over an nx x 1 grid (ny must be 1)."""
    p = Params()
    lib().rlbm_default_params(ctypes.byref(p))
    p.d = int(d)
    p.m = float(m)
    p.order = int(order)
    if quadrature is None:
        quadrature = "massless" if m == 0 else "massive"
    p.quadrature = QUAD[quadrature]
    keep = []
    if groups is not None:
        g = np.ascontiguousarray(np.asarray(groups, dtype=np.int32).reshape(-1))
        keep.append(g)
        p.groups = g.ctypes.data_as(_IP)
        p.n_groups = len(g) // 2
    p.v0 = float(v0)
    if custom is not None:
        c = np.ascontiguousarray(np.asarray(custom, dtype=np.float64).reshape(-1, 6))
        keep.append(c)
        p.custom_table = c.ctypes.data_as(_DP)
        p.custom_Q = c.shape[0]
    p.tau_mode = TAU[tau_mode]
    p.tau = float(tau)
    p.eta_over_s = float(eta_over_s)
    p.kappa = float(kappa)
    p.boundary = BC[boundary]
    p.nx, p.ny = int(nx), int(ny)
    p.precision = PREC[precision]
    p.stream_mode = STREAM[stream]
    p.lam = float(lam)
    p.n_ref, p.T_ref = float(n_ref), float(T_ref)
    p.stream = cuda_stream
    p.gx, p.gy = float(g[0]), float(g[1])
    p.wall_T[0], p.wall_T[1] = float(wall_T[0]), float(wall_T[1])
    return p, keep


def plan(**kw):
    """Host-only tables (no GPU): dict with Q, K, n (Q,2), p (Q,3), w, H (Q,K), v0."""
    p, keep = make_params(kw.pop("nx", 1), kw.pop("ny", 1), **kw)
    Q, K = ctypes.c_int(), ctypes.c_int()
    nvec = np.zeros(144, dtype=np.int32)
    pm = np.zeros(216)
    w = np.zeros(72)
    H = np.zeros(72 * 16)
    v0 = ctypes.c_double()
    _check(lib().rlbm_plan(ctypes.byref(p), ctypes.byref(Q), ctypes.byref(K),
                           nvec.ctypes.data_as(_IP), pm.ctypes.data_as(_DP), w.ctypes.data_as(_DP),
                           H.ctypes.data_as(_DP), ctypes.byref(v0)))
    q, k = Q.value, K.value
    return dict(Q=q, K=k, n=nvec[:2 * q].reshape(q, 2).copy(), p=pm[:3 * q].reshape(q, 3).copy(),
                w=w[:q].copy(), H=H[:q * k].reshape(q, k).copy(), v0=v0.value)


def _ptr(a):
    """(pointer, on_device) for a numpy array or a torch tensor."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous float64")
        return a.ctypes.data, 0
    import torch
    if not isinstance(a, torch.Tensor) or a.dtype != torch.float64 or not a.is_contiguous():
        raise ValueError("tensors must be contiguous float64")
    return a.data_ptr(), 1 if a.is_cuda else 0


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


class Lattice:
    """One RLBM simulation on the current CUDA device (see include/rlbm.h).

    Keyword arguments are those of ``make_params``.  Work is issued on the
    torch current stream at construction unless ``cuda_stream`` is given.
    """

    def __init__(self, nx, ny, **kw):
        if "cuda_stream" not in kw:
            kw["cuda_stream"] = _current_stream()
        self.nx, self.ny = int(nx), int(ny)
        self._params, self._keep = make_params(nx, ny, **kw)
        h = _H()
        _check(lib().rlbm_create(ctypes.byref(self._params), ctypes.byref(h)))
        self.h = h
        Q = ctypes.c_int()
        _check(lib().rlbm_stencil(self.h, ctypes.byref(Q), None, None, None), self.h)
        self.Q = Q.value
        self.n = np.zeros((self.Q, 2), dtype=np.int32)
        self.p = np.zeros((self.Q, 3))
        self.w = np.zeros(self.Q)
        _check(lib().rlbm_stencil(self.h, ctypes.byref(Q), self.n.ctypes.data_as(_IP),
                                  self.p.ctypes.data_as(_DP), self.w.ctypes.data_as(_DP)), self.h)

    def close(self):
        if getattr(self, "h", None):
            lib().rlbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def ncell(self):
        return self.nx * self.ny

    @property
    def t(self):
        return lib().rlbm_time(self.h)

    def set_stream(self, stream):
        _check(lib().rlbm_set_stream(self.h, stream), self.h)

    def init(self, n, ux, uy, T):
        ptrs = [_ptr(a) for a in (n, ux, uy, T)]
        dev = {d for _, d in ptrs}
        if len(dev) != 1:
            raise ValueError("all init fields must live on the same side")
        for a in (n, ux, uy, T):
            size = a.size if isinstance(a, np.ndarray) else a.numel()
            if size != self.ncell:
                raise ValueError("field size must be nx*ny")
        _check(lib().rlbm_init(self.h, ptrs[0][0], ptrs[1][0], ptrs[2][0], ptrs[3][0], dev.pop()), self.h)

    def set_tau_field(self, tau):
        ptr, dev = _ptr(tau)
        _check(lib().rlbm_set_tau_field(self.h, ptr, dev), self.h)

    def step(self, nsteps=1):
        _check(lib().rlbm_step(self.h, int(nsteps)), self.h)

    KERNELS = {"auto": 0, "direct": 1, "tma_32x8": 2, "tma_32x4": 3}

    def set_step_kernel(self, kernel):
        """'auto', 'direct', 'tma_32x8' or 'tma_32x4' (rlbm_set_step_kernel)."""
        _check(lib().rlbm_set_step_kernel(self.h, self.KERNELS[kernel]), self.h)

    @property
    def step_kernel(self):
        k = lib().rlbm_step_kernel(self.h)
        return {v: n for n, v in self.KERNELS.items()}[k]

    def moments(self, full=False, out=None):
        """Fields of f(t) as numpy arrays (ny, nx) (host copy), or written into
        the given dict of float64 CUDA tensors ``out``."""
        names = ["n", "ux", "uy", "T", "eps"]
        if out is None:
            res = {k: np.empty((self.ny, self.nx)) for k in names}
            if full:
                res["N"] = np.empty((3, self.ny, self.nx))
                res["Tab"] = np.empty((6, self.ny, self.nx))
        else:
            res = out
        ptrs = [_ptr(res.get(k))[0] for k in names + ["N", "Tab"]]
        on_dev = 0 if out is None else 1
        _check(lib().rlbm_moments(self.h, *ptrs, on_dev), self.h)
        return res

    def populations(self):
        """Post-collision populations f*(t), float64 (Q, ny, nx)."""
        f = np.empty((self.Q, self.ny, self.nx))
        _check(lib().rlbm_get_populations(self.h, f.ctypes.data, 0), self.h)
        return f

    def set_populations(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        _check(lib().rlbm_set_populations(self.h, f.ctypes.data, 0), self.h)

    def sync_status(self, raise_on_error=True):
        cnt = ctypes.c_longlong()
        rc = lib().rlbm_sync_status(self.h, ctypes.byref(cnt))
        if rc != RLBM_OK and raise_on_error:
            _check(rc, self.h)
        return rc, cnt.value

    def buffers(self):
        """(cur, prev, elem_size, plane, (pitch, hx, hy, px)) of the device buffers."""
        cur, prev = _VP(), _VP()
        es = ctypes.c_int()
        plane = ctypes.c_longlong()
        lay = (ctypes.c_int * 4)()
        _check(lib().rlbm_buffers(self.h, ctypes.byref(cur), ctypes.byref(prev), ctypes.byref(es),
                                  ctypes.byref(plane), lay), self.h)
        return cur.value, prev.value, es.value, plane.value, tuple(lay)


class _BorrowedLattice(Lattice):
    """A Lattice view of a handle owned by a Batch (never destroyed here)."""

    def __init__(self, h, nx, ny):
        self.h = h
        self.nx, self.ny = nx, ny
        Q = ctypes.c_int()
        _check(lib().rlbm_stencil(self.h, ctypes.byref(Q), None, None, None), self.h)
        self.Q = Q.value
        self.n = np.zeros((self.Q, 2), dtype=np.int32)
        self.p = np.zeros((self.Q, 3))
        self.w = np.zeros(self.Q)
        _check(lib().rlbm_stencil(self.h, ctypes.byref(Q), self.n.ctypes.data_as(_IP),
                                  self.p.ctypes.data_as(_DP), self.w.ctypes.data_as(_DP)), self.h)

    def close(self):
        self.h = None


class Batch:
    """Many independent simulations stepped together from a CUDA graph, by
    persistent kernels (one per stencil kind; tile_shape 0 or 1) or by
    independent per-instance chains of step kernels (tile_shape 2)
    (rlbm_batch_* in include/rlbm.h).  ``configs`` is a list of keyword dicts
    for ``make_params`` (each with nx and ny)."""

    def __init__(self, configs, cuda_stream=None):
        if cuda_stream is None:
            cuda_stream = _current_stream()
        arr = (Params * len(configs))()
        self._keep = []
        dims = []
        for i, c in enumerate(configs):
            c = dict(c)
            nx, ny = c.pop("nx"), c.pop("ny")
            p, keep = make_params(nx, ny, cuda_stream=cuda_stream, **c)
            arr[i] = p
            self._keep.append(keep)
            dims.append((nx, ny))
        b = _VP()
        rc = lib().rlbm_batch_create(arr, len(configs), ctypes.byref(b))
        if rc != RLBM_OK:
            raise RLBMError(rc, lib().rlbm_last_error(None).decode())
        self.b = b
        self.instances = [_BorrowedLattice(lib().rlbm_batch_handle(self.b, i), nx, ny)
                          for i, (nx, ny) in enumerate(dims)]

    def _chk(self, rc):
        if rc != RLBM_OK:
            raise RLBMError(rc, lib().rlbm_batch_last_error(self.b).decode())

    def __len__(self):
        return len(self.instances)

    def __getitem__(self, i):
        return self.instances[i]

    def step(self, nsteps=1):
        self._chk(lib().rlbm_batch_step(self.b, int(nsteps)))

    def config(self, tile_shape, grid):
        self._chk(lib().rlbm_batch_config(self.b, int(tile_shape), int(grid)))

    def tune(self, trial_steps=3):
        shape, grid = ctypes.c_int(), ctypes.c_int()
        ms = ctypes.c_float()
        self._chk(lib().rlbm_batch_tune(self.b, int(trial_steps), ctypes.byref(shape), ctypes.byref(grid),
                                        ctypes.byref(ms)))
        return shape.value, grid.value, ms.value

    def info(self):
        shape, grid = ctypes.c_int(), ctypes.c_int()
        gmax = (ctypes.c_int * 2)()
        tiles = ctypes.c_longlong()
        self._chk(lib().rlbm_batch_info(self.b, ctypes.byref(shape), ctypes.byref(grid), gmax, ctypes.byref(tiles)))
        return dict(tile_shape=shape.value, grid=grid.value, grid_max=tuple(gmax), tiles=tiles.value)

    def set_spin_limit(self, limit):
        self._chk(lib().rlbm_batch_set_spin_limit(self.b, int(limit)))

    def sync_status(self, raise_on_error=True):
        cnt = ctypes.c_longlong()
        rc = lib().rlbm_batch_sync_status(self.b, ctypes.byref(cnt))
        if rc != RLBM_OK and raise_on_error:
            self._chk(rc)
        return rc, cnt.value

    def close(self):
        if getattr(self, "b", None):
            lib().rlbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Adjoint:
    """Checkpointed forward run and hand-written adjoint (rlbm_adjoint_* in
    include/rlbm.h) on a Lattice: gradients of L = 1/2 sum |u(T) - u_target|^2
    with respect to the per-cell tau field and the initial velocity."""

    def __init__(self, lattice, nsteps, checkpoint_every=100):
        self.lat = lattice
        self.nsteps = int(nsteps)
        a = _VP()
        rc = lib().rlbm_adjoint_create(lattice.h, self.nsteps, int(checkpoint_every), ctypes.byref(a))
        if rc != RLBM_OK:
            raise RLBMError(rc, "adjoint setup failed (periodic, order 2, constant or field tau)")
        self.a = a

    def _chk(self, rc):
        if rc != RLBM_OK:
            raise RLBMError(rc, lib().rlbm_adjoint_last_error(self.a).decode())

    def forward(self, n, ux, uy, T):
        ptrs = [_ptr(x) for x in (n, ux, uy, T)]
        dev = {d for _, d in ptrs}
        if len(dev) != 1:
            raise ValueError("all fields must live on the same side")
        self._chk(lib().rlbm_adjoint_forward(self.a, *[p for p, _ in ptrs], dev.pop()))

    def backward(self, ux_target, uy_target, out=None):
        """Returns (loss, grad_tau, grad_ux0, grad_uy0): numpy (host) or, with
        ``out`` a dict of CUDA float64 tensors {'tau','ux0','uy0','loss'}, device."""
        (pu, d1), (pv, d2) = _ptr(ux_target), _ptr(uy_target)
        if d1 != d2:
            raise ValueError("targets must live on the same side")
        ny, nx = self.lat.ny, self.lat.nx
        if out is None:
            res = {"loss": np.zeros(1), "tau": np.zeros((ny, nx)), "ux0": np.zeros((ny, nx)),
                   "uy0": np.zeros((ny, nx))}
            od = 0
        else:
            res, od = out, 1
        self._chk(lib().rlbm_adjoint_backward(self.a, pu, pv, d1, _ptr(res["loss"])[0], _ptr(res["tau"])[0],
                                              _ptr(res["ux0"])[0], _ptr(res["uy0"])[0], od))
        if out is None:
            return float(res["loss"][0]), res["tau"], res["ux0"], res["uy0"]
        return res

    def close(self):
        if getattr(self, "a", None):
            lib().rlbm_adjoint_destroy(self.a)
            self.a = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def plan3(order=2):
    """Host-only (3+1)-d tables of expansion order 2 or 3: dict with Q, K,
    n (Q,3), p (Q,4), w, H (Q,K)."""
    Q, K = ctypes.c_int(), ctypes.c_int()
    cap = 288
    nvec = np.zeros(3 * cap, dtype=np.int32)
    pm, w, H = np.zeros(4 * cap), np.zeros(cap), np.zeros(30 * cap)
    rc = lib().rlbm3_plan(int(order), ctypes.byref(Q), ctypes.byref(K), nvec.ctypes.data_as(_IP),
                          pm.ctypes.data_as(_DP), w.ctypes.data_as(_DP), H.ctypes.data_as(_DP))
    if rc != RLBM_OK:
        raise RLBMError(rc, lib().rlbm3_last_error(None).decode())
    q, k = Q.value, K.value
    return dict(Q=q, K=k, n=nvec[:3 * q].reshape(q, 3).copy(), p=pm[:4 * q].reshape(q, 4).copy(),
                w=w[:q].copy(), H=H[:k * q].reshape(q, k).copy())


class Lattice3:
    """A (3+1)-d massless periodic lattice (expansion order 2 or 3; FP64 or
    FP32 storage) behind the rlbm3_* calls; fields are numpy (nz, ny, nx)
    arrays or CUDA float64 tensors."""

    def __init__(self, nx, ny, nz, tau=1.0, precision="fp64", cuda_stream=None, order=2):
        if cuda_stream is None:
            cuda_stream = _current_stream()
        self.nx, self.ny, self.nz = nx, ny, nz
        h = _H()
        rc = lib().rlbm3_create(nx, ny, nz, tau, int(order), PREC[precision], cuda_stream, ctypes.byref(h))
        if rc != RLBM_OK:
            raise RLBMError(rc, lib().rlbm3_last_error(None).decode())
        self.h = h
        Q = ctypes.c_int()
        nvec = np.zeros(3 * 288, dtype=np.int32)
        pm = np.zeros(4 * 288)
        w = np.zeros(288)
        self._chk(lib().rlbm3_stencil(self.h, ctypes.byref(Q), nvec.ctypes.data_as(_IP), pm.ctypes.data_as(_DP),
                                      w.ctypes.data_as(_DP)))
        self.Q = Q.value
        self.n = nvec[:3 * self.Q].reshape(self.Q, 3).copy()
        self.p = pm[:4 * self.Q].reshape(self.Q, 4).copy()
        self.w = w[:self.Q].copy()

    def _chk(self, rc):
        if rc != RLBM_OK:
            raise RLBMError(rc, lib().rlbm3_last_error(self.h).decode())

    def init(self, n, ux, uy, uz, T):
        ptrs = [_ptr(a) for a in (n, ux, uy, uz, T)]
        dev = {d for _, d in ptrs}
        if len(dev) != 1:
            raise ValueError("fields must all live on the host or all on the device")
        self._chk(lib().rlbm3_init(self.h, *[p for p, _ in ptrs], dev.pop()))

    def step(self, k=1):
        self._chk(lib().rlbm3_step(self.h, int(k)))

    def moments(self):
        """dict n, ux, uy, uz, T, eps of f(t) as (nz, ny, nx) host arrays."""
        out = np.empty((6, self.nz, self.ny, self.nx))
        self._chk(lib().rlbm3_moments(self.h, out.ctypes.data, 0))
        return dict(zip(("n", "ux", "uy", "uz", "T", "eps"), out))

    def populations(self):
        f = np.empty((self.Q, self.nz, self.ny, self.nx))
        self._chk(lib().rlbm3_get_populations(self.h, f.ctypes.data_as(_DP)))
        return f

    def sync_status(self):
        c = ctypes.c_longlong()
        rc = lib().rlbm3_sync_status(self.h, ctypes.byref(c))
        if rc not in (RLBM_OK, -4):             # -4: NONPHYSICAL, reported with the count
            self._chk(rc)
        return rc, c.value

    def close(self):
        if getattr(self, "h", None):
            lib().rlbm3_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def plan1(order=2):
    """Host-only (1+1)-d tables (no GPU): dict with Q, n (Q,), p (Q, 2), w, H (Q, Q)."""
    Q = ctypes.c_int()
    nvec = np.zeros(10, dtype=np.int32)
    pm = np.zeros(20)
    w = np.zeros(10)
    H = np.zeros(100)
    rc = lib().rlbm1_plan(int(order), ctypes.byref(Q), nvec.ctypes.data_as(_IP), pm.ctypes.data_as(_DP),
                          w.ctypes.data_as(_DP), H.ctypes.data_as(_DP))
    if rc != RLBM_OK:
        raise RLBMError(rc, lib().rlbm1_last_error(None).decode())
    q = Q.value
    return dict(Q=q, n=nvec[:q].copy(), p=pm[:2 * q].reshape(q, 2).copy(), w=w[:q].copy(),
                H=H[:q * q].reshape(q, q).copy())


class Lattice1:
    """A (1+1)-d massless gas (App. H (1+1)-d table of expansion order 2 ... 5;
    FP64 or FP32 storage) behind the rlbm1_* calls; fields are numpy (nx,)
    arrays or CUDA float64 tensors."""

    FIELDS = ("n", "ux", "T", "eps", "N0", "Nx", "T00", "T0x")

    def __init__(self, nx, order=2, tau=1.0, boundary="periodic", wall_T=None, precision="fp64",
                 cuda_stream=None):
        if cuda_stream is None:
            cuda_stream = _current_stream()
        self.nx = int(nx)
        h = _H()
        wt = None
        if wall_T is not None:
            self._wall = np.ascontiguousarray(wall_T, dtype=np.float64)
            wt = self._wall.ctypes.data_as(_DP)
        rc = lib().rlbm1_create(self.nx, int(order), float(tau), BC[boundary], wt, PREC[precision], cuda_stream,
                                ctypes.byref(h))
        if rc != RLBM_OK:
            raise RLBMError(rc, lib().rlbm1_last_error(None).decode())
        self.h = h
        Q = ctypes.c_int()
        nvec = np.zeros(10, dtype=np.int32)
        pm = np.zeros(20)
        w = np.zeros(10)
        self._chk(lib().rlbm1_stencil(self.h, ctypes.byref(Q), nvec.ctypes.data_as(_IP), pm.ctypes.data_as(_DP),
                                      w.ctypes.data_as(_DP)))
        self.Q = Q.value
        self.n = nvec[:self.Q].copy()
        self.p = pm[:2 * self.Q].reshape(self.Q, 2).copy()
        self.w = w[:self.Q].copy()

    def _chk(self, rc):
        if rc != RLBM_OK:
            raise RLBMError(rc, lib().rlbm1_last_error(self.h).decode())

    def init(self, n, ux, T):
        ptrs = [_ptr(a) for a in (n, ux, T)]
        dev = {d for _, d in ptrs}
        if len(dev) != 1:
            raise ValueError("fields must all live on the host or all on the device")
        self._chk(lib().rlbm1_init(self.h, *[p for p, _ in ptrs], dev.pop()))

    def step(self, k=1):
        self._chk(lib().rlbm1_step(self.h, int(k)))

    def moments(self):
        """dict n, ux, T, eps, N0, Nx, T00, T0x of f(t) as (nx,) host arrays."""
        out = np.empty((8, self.nx))
        self._chk(lib().rlbm1_moments(self.h, out.ctypes.data, 0))
        return dict(zip(self.FIELDS, out))

    def populations(self):
        f = np.empty((self.Q, self.nx))
        self._chk(lib().rlbm1_get_populations(self.h, f.ctypes.data_as(_DP)))
        return f

    def sync_status(self):
        c = ctypes.c_longlong()
        rc = lib().rlbm1_sync_status(self.h, ctypes.byref(c))
        if rc not in (RLBM_OK, -4):             # -4: NONPHYSICAL, reported with the count
            self._chk(rc)
        return rc, c.value

    def close(self):
        if getattr(self, "h", None):
            lib().rlbm1_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
