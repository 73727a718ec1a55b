"""Continuum relations used by the RLBM oracle, FP64 (test infrastructure only).

Lattice units c = k_B = T0 = 1 (Sec. 5.1, Sec. 6.1).
"""
from __future__ import annotations

import numpy as np
from scipy import special

ETA = np.diag([1.0, -1.0, -1.0])   # Minkowski metric, Sec. 3


def G_d(zeta, d=2):
    """Eq. defG: G_d = (eps + P)/P = zeta K_{(d+3)/2}(zeta) / K_{(d+1)/2}(zeta);
    zeta -> 0 limit d + 1 (Eq. ultra-relativistic-eos)."""
    zeta = np.asarray(zeta, dtype=np.float64)
    out = np.full(zeta.shape, float(d + 1))
    nz = zeta > 0
    z = zeta[nz]
    out[nz] = z * special.kve((d + 3) / 2.0, z) / special.kve((d + 1) / 2.0, z)
    return out


def energy_per_particle(T, m, d=2):
    """Eq. eos-ddim: eps/n = T (G_d(m/T) - 1)."""
    T = np.asarray(T, dtype=np.float64)
    return T * (G_d(m / T, d) - 1.0)


def pressure(n, T):
    """Eq. eos-ddim: P = n T."""
    return n * T


def temperature_from_energy(e, m, d=2, iters=100):
    """Invert eps/n = T (G_d(m/T) - 1) for T (step 4 of Sec. 6.2).

    Massless: T = e/d exactly.  Massive: bisection on the monotone function
    T -> T (G_d(m/T) - 1), vectorised over cells, 100 halvings.  The bracket
    (0, e] holds the root: the function tends to m as T -> 0, equals at least
    e at T = e (G_d - 1 >= 1 for d >= 2), and eps/n >= m for a physical
    state."""
    e = np.asarray(e, dtype=np.float64)
    if m == 0.0:
        return e / d
    lo = np.full(e.shape, 1e-12)
    hi = np.maximum(e, 1e-12) * 1.0
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        f = energy_per_particle(mid, m, d) - e
        lo = np.where(f < 0, mid, lo)
        hi = np.where(f < 0, hi, mid)
    return 0.5 * (lo + hi)


def landau(Nvec, Tmat):
    """Steps 2-3 of Sec. 6.2 (Landau frame, Sec. 4): eps U^a = T^{ab} U_b.

    Solved as the eigenproblem of the mixed tensor A^a_b = T^{ac} eta_{cb}
    with LAPACK ``eig``; eps is the largest real eigenvalue and U its
    eigenvector normalised to U^a U_a = 1, U^0 > 0.  n = U_a N^a.
    Nvec: (3, ...), Tmat: (3, 3, ...).  Returns eps, U (3, ...), n, ok mask
    (ok = eigenvector timelike and eigenvalue real and positive).
    """
    shp = Nvec.shape[1:]
    A = np.moveaxis(Tmat.reshape(3, 3, -1), -1, 0) @ ETA       # (C, 3, 3)
    lam, vec = np.linalg.eig(A)
    lam_r = lam.real
    idx = np.argmax(lam_r, axis=1)
    C = A.shape[0]
    eps = lam_r[np.arange(C), idx]
    v = vec[np.arange(C), :, idx].real                         # (C, 3)
    norm2 = v[:, 0] ** 2 - v[:, 1] ** 2 - v[:, 2] ** 2
    ok = (norm2 > 0) & (eps > 0) & (np.abs(lam[np.arange(C), idx].imag) == 0)
    U = v / np.sqrt(np.abs(norm2))[:, None]
    U = U * np.sign(U[:, :1])
    U = U.T.reshape((3,) + shp)
    eps = eps.reshape(shp)
    Ul = ETA @ U.reshape(3, -1)
    n = np.sum(Ul * Nvec.reshape(3, -1), axis=0).reshape(shp)
    return eps, U, n, ok.reshape(shp)


def four_velocity(ux, uy):
    """U^mu = gamma (1, u) from the 3-velocity u (fraction of c)."""
    g = 1.0 / np.sqrt(1.0 - ux * ux - uy * uy)
    return np.stack([g, g * ux, g * uy], axis=0)


def ce_shear_viscosity_coeff(zeta, d=2):
    """f(zeta) in eta = f(zeta) P tau, Chapman-Enskog (App. C, "To give a few
    examples"): d = 2: (2 G_2 - zeta^2 + e^zeta zeta^4 Gamma(0, zeta)/(zeta + 1))/8.
    Gamma(0, z) = E_1(z); e^z E_1(z) is evaluated as Tricomi's U(1, 1, z).
    UR limit (d+1)/(d+2) (Eq. ce-ur-limit)."""
    if d != 2:
        raise NotImplementedError
    z = np.asarray(zeta, dtype=np.float64)
    g = G_d(z, 2)
    zz = np.where(z > 0, z, 1.0)
    tail = np.where(z > 0, z ** 4 * special.hyperu(1.0, 1.0, zz) / (z + 1.0), 0.0)
    return (2.0 * g - z * z + tail) / 8.0
