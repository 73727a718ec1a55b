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
    (ok = finite moments, eigenvector timelike, eigenvalue real and positive).
    """
    shp = Nvec.shape[1:]
    A = np.moveaxis(Tmat.reshape(3, 3, -1), -1, 0) @ ETA       # (C, 3, 3)
    # a cell with non-finite moments is non-physical (no eigenpair); it is
    # solved as the identity so that LAPACK sees finite input, and flagged
    finite = np.all(np.isfinite(A), axis=(1, 2)) & np.all(np.isfinite(Nvec.reshape(3, -1)), axis=0)
    A = np.where(finite[:, None, None], A, np.eye(3))
    lam, vec = np.linalg.eig(A)
    lam_r = lam.real
    idx = np.argmax(lam_r, axis=1)
    C = A.shape[0]
    eps = lam_r[np.arange(C), idx]
    v = vec[np.arange(C), :, idx].real                         # (C, 3)
    norm2 = v[:, 0] ** 2 - v[:, 1] ** 2 - v[:, 2] ** 2
    ok = (norm2 > 0) & (eps > 0) & (np.abs(lam[np.arange(C), idx].imag) == 0) & finite
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


def _exp_e1(z):
    """e^z Gamma(0, z) = e^z E_1(z) for z > 0: scipy's exp1 times exp(z) up to
    z = 500 (relative error ~1e-15), Tricomi's U(1, 1, z) beyond (the
    exponential would overflow)."""
    z = np.asarray(z, dtype=np.float64)
    small = np.minimum(z, 500.0)
    return np.where(z <= 500.0, special.exp1(small) * np.exp(small), special.hyperu(1.0, 1.0, z))


def bickley_ki1(z):
    """Ki_1(z) = int_z^inf K_0(t) dt (the Bickley function of App. C), by
    adaptive quadrature."""
    from scipy import integrate
    z = np.atleast_1d(np.asarray(z, dtype=np.float64))
    return np.array([integrate.quad(lambda t: special.k0(t), v, np.inf, epsabs=0, epsrel=1e-13, limit=200)[0]
                     for v in z])


def ce_shear_viscosity_coeff(zeta, d=2):
    """f(zeta) in eta = f(zeta) P tau, Chapman-Enskog (App. C, "To give a few
    examples"): d = 2: (2 G_2 - zeta^2 + e^zeta zeta^4 Gamma(0, zeta)/(zeta + 1))/8;
    d = 3: (3 G_3 - 5 zeta^2 + G_3 zeta^2 - zeta^3 Ki_1(zeta)/K_2(zeta))/15.
    Gamma(0, z) = E_1(z) (e^z E_1(z) by _exp_e1).  UR limit (d+1)/(d+2)
    (Eq. ce-ur-limit)."""
    if d == 3:
        z = np.atleast_1d(np.asarray(zeta, dtype=np.float64))
        g = G_d(z, 3)
        out = np.full(z.shape, 4.0 / 5.0)
        nz = z > 0
        if np.any(nz):
            zn = z[nz]
            out[nz] = (3 * g[nz] - 5 * zn * zn + g[nz] * zn * zn - zn ** 3 * bickley_ki1(zn) / special.kv(2, zn)) / 15
        return out if np.ndim(zeta) else float(out[0])
    if d != 2:
        raise NotImplementedError
    z = np.asarray(zeta, dtype=np.float64)
    g = G_d(z, 2)
    zz = np.where(z > 0, z, 1.0)
    tail = np.where(z > 0, z ** 4 * _exp_e1(zz) / (z + 1.0), 0.0)
    return (2.0 * g - z * z + tail) / 8.0


def ce_thermal_conductivity_coeff(zeta, d=2):
    """g(zeta) in lambda = g(zeta) n tau (k_B = c = 1), Chapman-Enskog with
    the Anderson-Witting collision, d = 2 (App. C, thermal conductivity):
    G (G/2 - 1 - G zeta^2 e^zeta Gamma(0, zeta) / (2 (zeta + 1))), G = G_2.
    UR limit (d+1)/d = 3/2.  The heat flux is q^a = lambda nabla^a T."""
    if d != 2:
        raise NotImplementedError
    z = np.asarray(zeta, dtype=np.float64)
    g = G_d(z, 2)
    zz = np.where(z > 0, z, 1.0)
    tail = np.where(z > 0, z * z * _exp_e1(zz) / (2.0 * (z + 1.0)), 0.0)
    return g * (g / 2.0 - 1.0 - g * tail)


def ce_bulk_viscosity_coeff(zeta, d=2):
    """h(zeta) in mu = h(zeta) P tau, Chapman-Enskog with the Anderson-Witting
    collision, d = 2 (App. C, bulk viscosity):
    (zeta^4 + 3 zeta^2 + 2 G^3 - 12 G^2 + 18 G - zeta^2 G^2 + 2 zeta^2 G)
      / (4 (G^2 - 4 G + 1 - zeta^2))  +  e^zeta zeta^4 Gamma(0, zeta) / (4 (zeta + 1)).
    Zero in the UR limit.  The dynamic pressure is varpi = -mu nabla_a U^a."""
    if d != 2:
        raise NotImplementedError
    z = np.asarray(zeta, dtype=np.float64)
    g = G_d(z, 2)
    zz = np.where(z > 0, z, 1.0)
    num = z ** 4 + 3 * z * z + 2 * g ** 3 - 12 * g * g + 18 * g - z * z * g * g + 2 * z * z * g
    den = 4.0 * (g * g - 4.0 * g + 1.0 - z * z)
    tail = np.where(z > 0, z ** 4 * _exp_e1(zz) / (4.0 * (z + 1.0)), 0.0)
    return np.where(z > 0, num / np.where(z > 0, den, 1.0) + tail, 0.0)


def riemann_ur(nL, PL, nR, PR, d=2, c=1.0):
    """Inviscid ultra-relativistic Riemann problem with the fluid at rest on
    both sides of a membrane at x = 0 and PL > PR (App. D): a rarefaction
    moving left, a contact discontinuity and a shock moving right.

    The EOS is eps = d P, P = n T, so the sound speed is c/sqrt(d) and the
    adiabatic index (d+1)/d.  Along the left-moving rarefaction the Riemann
    invariants P R^a and n R^b are those of the left state, with
    R = (1+beta)/(1-beta), a = (d+1)/(2 sqrt d), b = sqrt(d)/2.  Across the
    shock the Rankine-Hugoniot conditions in the shock frame give the shock
    speed, the post-shock velocity and n_II.  P_C is the root (by bisection
    on (PR, PL)) of: the velocity reached at the tail of the rarefaction at
    pressure P_C equals the post-shock velocity at P_C.

    Returns a dict with P_C, beta_C, beta_s, n_I, n_II and the self-similar
    speeds of the head, tail, contact and shock (in units of c)."""
    sd = np.sqrt(d)
    cs = 1.0 / sd

    def beta_shock(P):
        return np.sqrt(d * (P - PR) ** 2 / ((PR + d * P) * (P + d * PR)))

    def beta_rare(P):
        # (1 - beta)/(1 + beta) = (P/PL)^(1/a) on the fan
        q = (P / PL) ** (2.0 * sd / (d + 1))
        return (1.0 - q) / (1.0 + q)

    lo, hi = PR, PL
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if beta_rare(mid) - beta_shock(mid) > 0.0:
            lo = mid            # rarefaction still faster: P_C is higher
        else:
            hi = mid
    PC = 0.5 * (lo + hi)
    bC = beta_shock(PC)
    bs = np.sqrt((PR + d * PC) / (d * (PC + d * PR)))
    nII = nR * np.sqrt(PC * (PR + d * PC) / (PR * (PC + d * PR)))
    nI = nL * (PC / PL) ** (d / (d + 1.0))
    return {"P_C": PC, "beta_C": bC, "beta_s": bs, "n_I": nI, "n_II": nII,
            "w_H": -cs * c, "w_T": c * (bC - cs) / (1.0 - bC * cs), "w_C": bC * c, "w_S": bs * c,
            "nL": nL, "PL": PL, "nR": nR, "PR": PR, "d": d, "c": c}


def riemann_ur_profile(sol, w):
    """n, P, beta of the App. D solution at self-similar coordinates w = x/t."""
    w = np.asarray(w, dtype=np.float64)
    d, c = sol["d"], sol["c"]
    sd = np.sqrt(d)
    n = np.empty_like(w)
    P = np.empty_like(w)
    beta = np.zeros_like(w)
    L = w < sol["w_H"]
    fan = (w >= sol["w_H"]) & (w < sol["w_T"])
    I = (w >= sol["w_T"]) & (w < sol["w_C"])
    II = (w >= sol["w_C"]) & (w < sol["w_S"])
    R = w >= sol["w_S"]
    n[L], P[L] = sol["nL"], sol["PL"]
    # on the fan the characteristic (beta - cs)/(1 - beta cs) equals w/c
    x = w[fan] / c
    b = (x + 1.0 / sd) / (1.0 + x / sd)
    beta[fan] = b
    ratio = (1.0 - b) / (1.0 + b)
    n[fan] = sol["nL"] * ratio ** (sd / 2.0)
    P[fan] = sol["PL"] * ratio ** ((d + 1) / (2.0 * sd))
    n[I], P[I], beta[I] = sol["n_I"], sol["P_C"], sol["beta_C"]
    n[II], P[II], beta[II] = sol["n_II"], sol["P_C"], sol["beta_C"]
    n[R], P[R] = sol["nR"], sol["PR"]
    return n, P, beta
