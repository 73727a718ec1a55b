"""Shared test helpers: build oracle counterparts of product configurations
and match population orderings.  The oracle side never receives a value
computed by the product: only the configuration (stencil generators, v0,
grid, tau, boundary) and the seeded initial fields are shared."""
from __future__ import annotations

import numpy as np

from oracle import lattice as OL
from oracle import scheme as OS


def generators(nvec):
    """FS generator vectors of a stencil (one per group)."""
    gens = sorted({tuple(sorted((abs(int(a)), abs(int(b))), reverse=True)) for a, b in nvec},
                  key=lambda g: (g[0] ** 2 + g[1] ** 2, g))
    return gens


def oracle_quadrature(m, order, nvec=None, v0=None):
    """The oracle's quadrature for the same configuration: the App. H table
    (m = 0) or the oracle's own solve of the orthonormality conditions on the
    same FS stencil and v0 (m > 0)."""
    if m == 0:
        return OL.massless_quadrature(order)
    q, res = OL.massive_quadrature(generators(nvec), m, v0, order)
    assert res < 1e-9
    return q


def key(n, p0):
    return (int(n[0]), int(n[1]), round(float(p0), 9))


def permutation(prod_n, prod_p, quad):
    """idx such that product population idx[j] is oracle population j."""
    pos = {key(prod_n[i], prod_p[i, 0]): i for i in range(len(prod_n))}
    return np.array([pos[key(quad.n[j], quad.p[j, 0])] for j in range(quad.Q)])


def oracle_sim(quad, nx, ny, tau=1.0, boundary="periodic", stream="onlattice", lam=None, g=None,
               wall_T=(0.0, 0.0)):
    return OS.Simulation(quad, OL.Expansion(quad), nx, ny, tau=tau, boundary=boundary,
                         stream=stream, lam=lam, g=g, wall_T=wall_T)


def rel_linf(a, b):
    """max |a - b| / max |b| (relative L-infinity, normalised by the reference)."""
    return float(np.abs(a - b).max() / np.abs(b).max())


class _DeviceView:
    """A raw device buffer (borrowed) seen by torch through __cuda_array_interface__."""

    def __init__(self, ptr, nbytes):
        self.__cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (ptr, False),
                                         "version": 3, "strides": None}


def device_patch(lat, cx, cy, R, quad, idx, ref=(1.0, 1.0)):
    """Post-collision populations f*(t) of the (2R+1)^2 cells around (cx, cy)
    (periodic), read from the handle's current device buffer, as FP64 in the
    oracle's population order [Q][2R+1][2R+1].  FP32 storage holds
    f - f_ref; f_ref is the oracle's rest-frame equilibrium at the handle's
    (n_ref, T_ref) = ref, which equals the library's to rounding."""
    import torch
    cur, _, elem, plane, (pitch, hx, hy, px) = lat.buffers()
    Q = lat.Q
    raw = torch.as_tensor(_DeviceView(cur, Q * plane * elem), device="cuda")
    vals = raw.view(torch.float32 if elem == 4 else torch.float64)
    xs = (cx + np.arange(-R, R + 1)) % lat.nx
    ys = (cy + np.arange(-R, R + 1)) % lat.ny
    sidx = (ys[:, None] + hy) * pitch + (xs[None, :] + px)
    index = (np.arange(Q)[:, None, None] * plane + sidx[None]).reshape(-1)
    f = vals[torch.as_tensor(index, device="cuda")].double().cpu().numpy().reshape(Q, 2 * R + 1, 2 * R + 1)
    f = f[idx]                                  # oracle order
    if elem == 4:
        one = np.ones((1, 1))
        f = f + OL.Expansion(quad).feq(ref[0] * one, np.array([1.0, 0.0, 0.0]).reshape(3, 1, 1),
                                       ref[1] * one)[:, :1, :1]
    return f


def oracle_center_update(quad, fpatch, tau, stream="onlattice", lam=None):
    """One oracle step (pull streaming, collision) of a patch; returns the
    centre cell's f*(t+1) [Q].  The centre's pull stays inside the patch when
    R is at least the largest shift (+1 for the bilinear taps)."""
    R = fpatch.shape[1] // 2
    if stream == "onlattice":
        f = OS.stream_onlattice(fpatch, quad.n, "periodic")
    else:
        f = OS.stream_bilinear(fpatch, lam * quad.velocity(), "periodic")
    fs, _ = OS.collide(f, quad, OL.Expansion(quad), tau)
    return fs[:, R, R]
