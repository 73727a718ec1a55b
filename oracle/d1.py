"""(1+1)-dimensional massless RLBM step, FP64 (oracle; test infrastructure only).

Covers the d = 1 massless case of Sec. 5 and Sec. 6.2 (lattice units
c = k_B = T0 = 1):
- the App. H "(1+1) dimensions" quadratures: populations p_{j,s} =
  p0_j (1, s), s = +-1, on the shells p0_j of the table, moving one cell per
  step in direction s;
- the equilibrium of the massless limit of Sec. 5.2 (Eq.
  mj-expanded-1D-massless): the weight omega of the massive expansion is
  normalised with C = 1/(2 m K_1(m)) -> 1/2, so omega = exp(-p0)/2 on the
  measure dp/p0, under which the constant polynomial has no finite norm;
- the Landau frame of Sec. 4 (2 x 2 mixed tensor), the massless EOS
  eps = P = n T (d = 1), Anderson-Witting relaxation and pull streaming.

Readings (the paper is silent or garbled here):
- App. H prints the order-4 table with its two columns exchanged: the
  printed weights are the shells (the roots of L_4) and the printed shells
  the weights.  They are read exchanged back.
- The massless limit of the expansion.  The order-N massive basis in d = 1 is
  {1} and phi_{a,s} = (p0)^a sign(p^x)^s, 1 <= a <= N, s = 0, 1 ((p^x)^2 is
  tied to (p0)^2 on the mass shell).  As m -> 0 the norm of the constant and
  its overlap with f_MJ / omega diverge alike (logarithmically, from
  p0 -> 0), so the projection tends to
      F(p) = c0 + sum_jk (G^-1)_jk r_k phi_j(p),
      c0 = lim_{p -> 0} f_MJ / omega = n / T,
      G_jk = int omega phi_j phi_k dp/p0,  r_k = int (f_MJ - c0 omega) phi_k dp/p0,
  and f^eq_i = w_i F(p_i).  At N = 1 this is the printed first-order formula
  f^eq = n omega ((1 - p0)/T + p0 U^0 + p^x U^x).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

ETA2 = np.diag([1.0, -1.0])

# App. H, (1+1) dimensions: shells p0_j and weights w_j as printed (per
# direction), orders 2 ... 5.  Order 4 is stored as printed; the reading
# exchanges its columns (module docstring).
MASSLESS_D1_PRINTED = {
    2: ([3.414213562373095048, 0.585786437626904951],
        [0.042893218813452475, 1.457106781186547524]),
    3: ([6.289945082937479196, 0.415774556783479083, 2.294280360279041719],
        [0.001651724516604877, 1.710285053107483686, 0.121396555709244769]),
    4: ([1.869968763544262523, 0.008571999852268322, 0.000057401877068880, 0.204735168059733606],
        [0.322547689619392311, 4.536620296921127983, 9.395070912301133129, 1.745761101158346575]),
    5: ([0.26356031971814091020, 3.59642577104072208122, 1.41340305910651679221, 7.08581000585883755692,
         12.6408008442757826594],
        [1.97964401902679930651, 0.02111608983931054815, 0.28206165857260368669, 0.00050971712153383997,
         0.00000184877308595198]),
}


def massless_table_1d(order):
    """(shells, weights per direction) of App. H, order-4 columns exchanged."""
    p0, w = MASSLESS_D1_PRINTED[order]
    if order == 4:
        p0, w = w, p0
    return list(p0), list(w)


@dataclass
class Quadrature1:
    n: np.ndarray        # (Q,) integer displacement per step (+-1)
    p: np.ndarray        # (Q, 2) momenta (p0, px)
    w: np.ndarray        # (Q,) weights of omega dp/p0 (half the printed per-direction value)
    order: int

    @property
    def Q(self):
        return len(self.w)


def massless_quadrature_1d(order=2):
    """Populations (shell j in table order, then direction s = +1, -1):
    p = p0_j (1, s), weight w_j / 2 (omega = exp(-p0)/2 spread over the two
    directions of the line)."""
    shells, wts = massless_table_1d(order)
    n, p, w = [], [], []
    for x, wj in zip(shells, wts):
        for s in (1, -1):
            n.append(s)
            p.append((x, s * x))
            w.append(0.5 * wj)
    return Quadrature1(np.array(n), np.array(p, dtype=np.float64), np.array(w), order)


def basis_1d(order):
    """(a, s) of phi_{a,s} = (p0)^a sign(p^x)^s, a = 1 ... N, s = 0, 1."""
    return [(a, s) for a in range(1, order + 1) for s in (0, 1)]


def omega_integral(a, s):
    """int omega (p0)^a sign(p^x)^s dp/p0 over the line, omega = exp(-p0)/2:
    (a - 1)! for even s, 0 for odd s (a >= 1)."""
    return float(math.factorial(a - 1)) if s % 2 == 0 else 0.0


def mj_moment_1d(a, s, n, U0, Ux, T):
    """int f_MJ (p0)^a sign(p^x)^s dp/p0 of the massless Maxwell-Juttner
    distribution f = (n/(2T)) exp(-p.U/T) (normalised so that N^0 = n U^0):
    with U = (cosh th, sinh th) and p.U = p0 (U^0 - s U^x) = p0 exp(-s th),
    the integral over p0 on each half-line is (a - 1)! (T exp(s th))^a, so
        n (a - 1)! T^(a-1) cosh(a th)   (s even),
        n (a - 1)! T^(a-1) sinh(a th)   (s odd)."""
    U0, Ux = np.asarray(U0), np.asarray(Ux)
    E = U0 + Ux                                  # exp(th)
    c = n * math.factorial(a - 1) * T ** (a - 1)
    Ea, Eia = E ** a, E ** (-a)
    return c * ((Ea + Eia) / 2 if s % 2 == 0 else (Ea - Eia) / 2)


class Expansion1:
    """Equilibrium of the massless d = 1 expansion (module docstring) on a
    quadrature of the given order.  The Gram matrix has integer entries
    (factorials); its inverse is taken in exact rational arithmetic, and the
    projection and its evaluation run in np.longdouble (at order 5 the
    members reach (p0)^5 ~ 3e5 and cancel: in double the equilibrium loses
    about 1e-13)."""

    def __init__(self, quad: Quadrature1):
        from fractions import Fraction
        self.quad = quad
        self.basis = basis_1d(quad.order)
        K = len(self.basis)
        G = [[Fraction(int(round(omega_integral(a + b, s + t)))) for (b, t) in self.basis] for (a, s) in self.basis]
        # Gauss-Jordan elimination over the rationals
        A = [row[:] + [Fraction(int(i == j)) for j in range(K)] for i, row in enumerate(G)]
        for c in range(K):
            piv = next(r for r in range(c, K) if A[r][c] != 0)
            A[c], A[piv] = A[piv], A[c]
            d = A[c][c]
            A[c] = [x / d for x in A[c]]
            for r in range(K):
                if r != c and A[r][c] != 0:
                    f = A[r][c]
                    A[r] = [x - f * y for x, y in zip(A[r], A[c])]
        self.Ginv = np.array([[np.longdouble(x.numerator) / np.longdouble(x.denominator) for x in row[K:]]
                              for row in A])

    def F(self, n, U, T, p):
        """F(p) = c0 + sum_jk (G^-1)_jk r_k phi_j(p) at momenta p (P, 2) on the
        light cone; n, T: (...) arrays, U: (2, ...).  Returns (P, ...)."""
        ld = np.longdouble
        n, T = np.asarray(n, dtype=ld), np.asarray(T, dtype=ld)
        U = np.asarray(U, dtype=ld)
        c0 = n / T
        r = np.array([mj_moment_1d(a, s, n, U[0], U[1], T) - c0 * ld(omega_integral(a, s))
                      for (a, s) in self.basis])                     # (K, ...)
        b = np.tensordot(self.Ginv, r, axes=1)                       # (K, ...)
        p = np.asarray(p, dtype=ld)
        sgn = np.sign(p[:, 1])
        phi = np.array([p[:, 0] ** a * sgn ** s for (a, s) in self.basis])      # (K, P)
        return (c0[None] + np.tensordot(phi.T, b, axes=1)).astype(np.float64)

    def feq(self, n, U, T):
        """f^eq_i = w_i F(p_i); n, T: (...) arrays, U: (2, ...)."""
        n = np.asarray(n, dtype=np.float64)
        return self.quad.w.reshape((-1,) + (1,) * n.ndim) * self.F(n, U, T, self.quad.p)


def landau2(Nvec, Tmat):
    """Sec. 4 in d = 1: the largest eigenvalue eps of A^a_b = T^{ag} eta_{gb}
    with a timelike eigenvector U (U.U = 1, U^0 > 0), n = U_a N^a.
    Nvec: (2, ...), Tmat: (2, 2, ...).  Returns eps, U, n, ok (LAPACK eig
    per cell; cells without a real timelike eigenvector are flagged)."""
    shp = Nvec.shape[1:]
    Nf = Nvec.reshape(2, -1)
    A = np.einsum("abc,bd->cad", Tmat.reshape(2, 2, -1), ETA2)        # (C, 2, 2)
    C = A.shape[0]
    eps = np.full(C, np.nan)
    U = np.full((2, C), np.nan)
    good = np.all(np.isfinite(A), axis=(1, 2))
    vals, vecs = np.linalg.eig(np.where(good[:, None, None], A, np.eye(2)))
    for k in range(2):
        v = np.real(vecs[:, :, k])                                     # (C, 2)
        lam = np.real(vals[:, k])
        real = np.abs(np.imag(vals[:, k])) <= 1e-12 * np.maximum(1.0, np.abs(lam))
        nrm = v[:, 0] ** 2 - v[:, 1] ** 2
        take = good & real & (nrm > 0) & ~(np.isfinite(eps) & (eps >= lam))
        sc = np.where(take, np.sign(v[:, 0]) / np.sqrt(np.where(nrm > 0, nrm, 1.0)), 0.0)
        eps = np.where(take, lam, eps)
        U = np.where(take[None], (v * sc[:, None]).T, U)
    n = U[0] * Nf[0] - U[1] * Nf[1]
    ok = np.isfinite(eps) & (eps > 0) & (n > 0)
    return eps.reshape(shp), U.reshape((2,) + shp), n.reshape(shp), ok.reshape(shp)


@dataclass
class Fields1:
    n: np.ndarray
    U: np.ndarray
    T: np.ndarray
    eps: np.ndarray
    N: np.ndarray
    Tab: np.ndarray
    ok: np.ndarray

    @property
    def ux(self):
        return self.U[1] / self.U[0]


def macroscopic1(f, quad: Quadrature1):
    """Steps 1-4: moments, the 2 x 2 Landau solve, n = U.N, T = eps / n."""
    N = np.tensordot(quad.p.T, f, axes=1)                               # (2, nx)
    Tab = np.einsum("ia,ib,i...->ab...", quad.p, quad.p, f)             # (2, 2, nx)
    eps, U, n, ok = landau2(N, Tab)
    return Fields1(n, U, eps / n, eps, N, Tab, ok)


def four_velocity1(ux):
    g = 1.0 / np.sqrt(1.0 - ux * ux)
    return np.array([g, g * ux])


def collide1(f, quad: Quadrature1, exp: Expansion1, tau, eqwall=False, wall_T=(0.0, 0.0)):
    """Steps 1-8 of Sec. 6.2 in d = 1; eqwall: the first and last cell hold
    f^eq(n, U = (1, 0), T_w) after the collision (T_w the prescribed wall
    temperature, or the cell's own T)."""
    fl = macroscopic1(f, quad)
    feq = exp.feq(fl.n, fl.U, fl.T)
    s = np.sign(quad.p[:, 1])[:, None]
    omega = (fl.U[0][None] - s * fl.U[1][None]) / tau                  # p.U / (p0 tau)
    fs = (1.0 - omega) * f + omega * feq
    if eqwall:
        for side, col in enumerate((0, f.shape[1] - 1)):
            T = wall_T[side] if wall_T[side] > 0 else fl.T[col]
            fs[:, col] = exp.feq(np.array([fl.n[col]]), np.array([[1.0], [0.0]]), np.array([T]))[:, 0]
    # a cell without a physical Landau frame is left unrelaxed
    with np.errstate(invalid="ignore"):
        good = fl.ok & (fl.n > 0) & (fl.T > 0) & np.isfinite(fl.T)
    return np.where(good[None], fs, f), fl


def stream1(fs, shifts, boundary="periodic"):
    """f_i(x) = f*_i(x - n_i); periodic or clamped (free-flow / wall) ends."""
    Q, nx = fs.shape
    xs = np.arange(nx)
    out = np.empty_like(fs)
    for i in range(Q):
        src = xs - int(shifts[i])
        src = src % nx if boundary == "periodic" else np.clip(src, 0, nx - 1)
        out[i] = fs[i][src]
    return out


class Simulation1:
    """State convention of scheme.Simulation (post-collision populations)."""

    def __init__(self, quad: Quadrature1, nx, tau=1.0, boundary="periodic", wall_T=(0.0, 0.0)):
        self.quad, self.exp = quad, Expansion1(quad)
        self.nx, self.tau, self.boundary, self.wall_T = nx, tau, boundary, wall_T
        self.fs = None
        self.fields = None

    def init(self, n, ux, T):
        U = four_velocity1(np.asarray(ux, dtype=np.float64))
        self.fs = self.exp.feq(np.asarray(n, dtype=np.float64), U, np.asarray(T, dtype=np.float64))
        self.fields = macroscopic1(self.fs, self.quad)

    def step(self, nsteps=1):
        for _ in range(nsteps):
            f = stream1(self.fs, self.quad.n, self.boundary)
            self.fs, self.fields = collide1(f, self.quad, self.exp, self.tau,
                                            self.boundary == "eqwall_x", self.wall_T)
        return self.fs
