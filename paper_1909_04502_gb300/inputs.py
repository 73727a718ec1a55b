"""Seeded synthetic workloads (initial macroscopic fields n, u, T and tau fields).

This module holds no arithmetic of the method: it only generates the initial
conditions the paper's benchmarks prescribe (Sec. 7.1 Taylor-Green vortex,
Eq. tg-initial-conditions; Sec. 8.1 Riemann problem), shear waves, a shear
layer and smooth random states for parity tests.  Fields are float64 arrays
of shape (ny, nx); u is the 3-velocity in units of c.
"""
from __future__ import annotations

import numpy as np


def taylor_green(L, u0=0.1, n0=1.0, T0=1.0):
    """Eq. tg-initial-conditions on x_i = 2 pi i / L (i = 0..L-1), uniform n, T."""
    x = 2 * np.pi * np.arange(L) / L
    X, Y = np.meshgrid(x, x)            # X varies along axis 1 (x), Y along axis 0 (y)
    ux = u0 * np.cos(X) * np.sin(Y)
    uy = -u0 * np.cos(Y) * np.sin(X)
    one = np.ones((L, L))
    return n0 * one, ux, uy, T0 * one


def shear_wave(nx, ny, amp=0.05, n0=1.0, T0=1.0):
    """u_y = amp sin(2 pi x / nx), u_x = 0, uniform n and T."""
    x = np.arange(nx)
    uy = np.tile(amp * np.sin(2 * np.pi * x / nx), (ny, 1))
    z = np.zeros((ny, nx))
    return n0 + z, z.copy(), uy, T0 + z


def sod(nx=1024, ny=1, nL=1.0, TL=1.0, nR=0.5, TR=0.8):
    """Riemann problem at rest: left state for x < nx/2, right state after.
    Defaults give P_L/P_R = 2.5 and T_L/T_R = 1.25."""
    left = np.arange(nx) < nx // 2
    n = np.where(left, nL, nR) * np.ones((ny, 1))
    T = np.where(left, TL, TR) * np.ones((ny, 1))
    z = np.zeros((ny, nx))
    return n, z, z.copy(), T


def kelvin_helmholtz(L, u=0.3, width=20.0, eps=1e-3, seed=1909, T0=1.0):
    """Doubly periodic shear layer: u_x = u [tanh((y - L/4)/w) - tanh((y - 3L/4)/w) - 1],
    u_y = eps * U[-1, 1] seeded."""
    y = np.arange(L)[:, None] + np.zeros((1, L))
    ux = u * (np.tanh((y - L / 4) / width) - np.tanh((y - 3 * L / 4) / width) - 1.0)
    rng = np.random.default_rng(seed)
    uy = eps * rng.uniform(-1.0, 1.0, (L, L))
    one = np.ones((L, L))
    return one.copy(), ux, uy, T0 * one


def random_smooth(nx, ny, seed=0, umax=0.3, dn=0.2, dT=0.2, modes=3):
    """Smooth periodic random fields (a few low Fourier modes) for parity tests."""
    rng = np.random.default_rng(seed)
    x = 2 * np.pi * np.arange(nx) / nx
    y = 2 * np.pi * np.arange(ny) / ny
    X, Y = np.meshgrid(x, y)

    def field():
        f = np.zeros((ny, nx))
        for _ in range(modes):
            kx, ky = rng.integers(0, 3, 2)
            ph = rng.uniform(0, 2 * np.pi)
            f += rng.uniform(-1, 1) * np.cos(kx * X + ky * Y + ph)
        return f / modes

    n = 1.0 + dn * field()
    T = 1.0 + dT * field()
    ux = umax * field()
    uy = umax * field()
    return n, ux, uy, T


def random_smooth3(nx, ny, nz, seed=0, umax=0.2, dn=0.2, dT=0.2, modes=3):
    """Smooth periodic random fields on an (nz, ny, nx) grid (a few low
    Fourier modes each): n, ux, uy, uz, T for three-dimensional parity tests."""
    rng = np.random.default_rng(seed)
    Z, Y, X = np.meshgrid(2 * np.pi * np.arange(nz) / nz, 2 * np.pi * np.arange(ny) / ny,
                          2 * np.pi * np.arange(nx) / nx, indexing="ij")

    def field():
        f = np.zeros((nz, ny, nx))
        for _ in range(modes):
            kx, ky, kz = rng.integers(0, 3, 3)
            f += rng.uniform(-1, 1) * np.cos(kx * X + ky * Y + kz * Z + rng.uniform(0, 2 * np.pi))
        return f / modes

    n = 1.0 + dn * field()
    T = 1.0 + dT * field()
    return n, umax * field(), umax * field(), umax * field(), T


def taylor_green3(L, nz, u0=0.2, n0=1.0, T0=1.0):
    """The Taylor-Green flow of ``taylor_green`` (u_x = u0 cos x sin y,
    u_y = -u0 cos y sin x on x_i = 2 pi i / L), uniform along z (nz cells),
    u_z = 0: the setup the paper runs with its (3+1)-dimensional solver."""
    n, ux, uy, T = taylor_green(L, u0=u0, n0=n0, T0=T0)
    rep = lambda a: np.ascontiguousarray(np.broadcast_to(a, (nz,) + a.shape))
    return rep(n), rep(ux), rep(uy), np.zeros((nz, L, L)), rep(T)


def smooth_tau(nx, ny, seed=5, lo=0.6, hi=2.0):
    """Hidden relaxation-time field: 1 + 0.3 * (four random low-k cosines),
    clipped to [lo, hi]."""
    rng = np.random.default_rng(seed)
    x = 2 * np.pi * np.arange(nx) / nx
    y = 2 * np.pi * np.arange(ny) / ny
    X, Y = np.meshgrid(x, y)
    f = np.zeros((ny, nx))
    for _ in range(4):
        kx, ky = rng.integers(1, 4, 2)
        f += rng.uniform(-1, 1) * np.cos(kx * X + ky * Y + rng.uniform(0, 2 * np.pi))
    return np.clip(1.0 + 0.3 * f / 4 * 2, lo, hi)


def sweep(count=64, seed=1909, side_lo=64, side_hi=1024, tau_lo=0.6, tau_hi=2.0,
          zetas=(0.0, 1.0, 10.0)):
    """Batched tau-sweep: per run a square side ~ U{side_lo..side_hi}, tau ~
    U[tau_lo, tau_hi], zeta assigned round-robin (PCG64 via numpy, seeded)."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(side_lo, side_hi + 1, count)
    taus = rng.uniform(tau_lo, tau_hi, count)
    return [dict(side=int(sides[i]), tau=float(taus[i]), zeta=float(zetas[i % len(zetas)]))
            for i in range(count)]
