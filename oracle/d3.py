"""(3+1)-dimensional massless RLBM step, FP64 (oracle; test infrastructure only).

Covers the d = 3 case of Sec. 5 and Sec. 6.2 for massless particles at
expansion orders N = 2 and 3 (lattice units c = k_B = T0 = 1):
- the App. H "(3+1) dimensions" quadratures, p_ij = p0_j (1, n_i/|n_i|);
- the Gram-Schmidt basis of Sec. 5.2 under the massless weight
  omega = e^{-p0} (d^3p / p0 = p0 dp0 dOmega on the light cone);
- the equilibrium of Eq. mj-discrete-feq with projections from the
  Maxwell-Juttner moments of App. B (d = 3, m = 0);
- on-lattice streaming, the Landau frame of Sec. 4 (4 x 4 mixed tensor),
  the massless EOS eps = 3 n T (Eq. ultra-relativistic-eos, d = 3) and the
  Anderson-Witting relaxation.

Population order: groups in the order of ``MASSLESS_D3`` (shell-major, see
``massless_quadrature_3d``), orbit members in ``fs_orbit3`` order.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass

import numpy as np

ETA4 = np.diag([1.0, -1.0, -1.0, -1.0])

# App. H, (3+1) dimensions, order 2: the three shell energies (roots of the
# generalized Laguerre polynomial L_3^(1)) and the six printed weights.
# Reading: the first printed group (+-2, +-1, +-1) cannot belong to a massless
# stencil, whose vectors must all have the length of (+-3, 0, 0); the group
# with that length is (+-2, +-2, +-1).  The weights are listed shell-major
# (shells in increasing energy, per shell the (2, 2, 1) group, then the
# (3, 0, 0) group), as the two-dimensional tables are; the other readings do
# not integrate the omega-moments.
MASSLESS_D3 = {
    2: dict(
        groups=[(2, 2, 1), (3, 0, 0)],
        shells=[0.9358222275240878, 3.3054072893322786, 7.7587704831436335],
        weights_printed=[0.0245283950433191, 0.0, 0.0163006691342629, 0.0,
                         0.0003891858228425, 0.0017936666649682],
    ),
    # order 3 (v0 = 1/sqrt(41)): the groups as printed, four shells (the nodes
    # of L_4^(1)), the twelve printed weights read shell-major like order 2
    3: dict(
        groups=[(4, 4, 3), (5, 4, 0), (6, 2, 1)],
        shells=[0.7432919279814314, 2.5716350076462784, 5.7311787516890996, 10.953894312683190],
        weights_printed=[0.0, 0.0, 0.0093098040253911, 0.0085195569675087, 0.0,
                         0.0056909667738262, 0.0013041770173120, 0.0, 0.0008932820065742,
                         0.0000029126213348, 0.0000338363537565, 0.0000090390475856],
    ),
}


def fs_orbit3(gen):
    """Full-symmetric orbit of a 3-vector (component permutations and sign
    flips), de-duplicated, sorted descending lexicographically."""
    out = set()
    for perm in itertools.permutations(gen):
        for signs in itertools.product((1, -1), repeat=3):
            out.add(tuple(s * c for s, c in zip(signs, perm)))
    return sorted(out, reverse=True)


@dataclass
class Quadrature3:
    n: np.ndarray        # (Q, 3) integer stencil vectors
    p: np.ndarray        # (Q, 4) momenta (p0, px, py, pz)
    w: np.ndarray        # (Q,) weights

    @property
    def Q(self):
        return len(self.w)


def massless_quadrature_3d(order=2):
    """Eq. ur-discrete-momentum-vectors in d = 3 with the App. H weights
    (readings above; per shell the groups in table order); zero-weight
    (group, shell) pairs are dropped."""
    tab = MASSLESS_D3[order]
    G, S, W = tab["groups"], tab["shells"], tab["weights_printed"]
    ns, ps, ws = [], [], []
    for j, p0 in enumerate(S):
        for g, gen in enumerate(G):
            w = W[j * len(G) + g]
            if w == 0.0:
                continue
            for v in fs_orbit3(gen):
                nv = np.array(v, dtype=np.float64)
                ns.append(v)
                ps.append(np.concatenate([[p0], p0 * nv / np.linalg.norm(nv)]))
                ws.append(w)
    return Quadrature3(np.array(ns, dtype=np.int64), np.array(ps), np.array(ws))


# --------------------------------------------------------------------------
# Sec. 5.2 in d = 3, m = 0.
# --------------------------------------------------------------------------


def _dfact(k):
    return 1 if k <= 0 else k * _dfact(k - 2)


def omega_moment_3d(c0, a, b, c):
    """E_omega[p0^c0 px^a py^b pz^c] = int d^3p/p0 e^{-p0} p0^c0 px^a py^b pz^c,
    normalised to 1 for the constant: on the light cone d^3p/p0 = p0 dp0 dOmega,
    the angular mean of nx^a ny^b nz^c is (a-1)!!(b-1)!!(c-1)!!/(a+b+c+1)!!
    (even a, b, c; zero otherwise) and int p0^(k+1) e^{-p0} dp0 = (k+1)!."""
    if a % 2 or b % 2 or c % 2:
        return 0.0
    ang = _dfact(a - 1) * _dfact(b - 1) * _dfact(c - 1) / _dfact(a + b + c + 1)
    return ang * math.factorial(c0 + a + b + c + 1)


def monomials_3d(order):
    """Generating set V of Sec. 5.2 up to ``order``: index tuples over
    (0, x, y, z), as exponent 4-tuples (c0, a, b, c)."""
    out = []
    for deg in range(order + 1):
        for idx in itertools.combinations_with_replacement(range(4), deg):
            out.append(tuple(idx.count(k) for k in range(4)))
    return out


def gram_schmidt_basis_3d(order, tol=1e-9):
    """Orthonormal polynomials J = C phi under omega (classical Gram-Schmidt on
    V in order, dropping members dependent on the light cone p0^2 = |p|^2)."""
    mons = monomials_3d(order)
    nm = len(mons)
    G = np.array([[omega_moment_3d(*(np.add(u, v))) for v in mons] for u in mons])
    rows = []
    for i in range(nm):
        v = np.zeros(nm)
        v[i] = 1.0
        for r in rows:
            v = v - (r @ G @ v) * r
        nrm2 = v @ G @ v
        if nrm2 <= tol * G[i, i]:
            continue
        rows.append(v / math.sqrt(nrm2))
    return np.array(rows), mons


def eval_monomials_3d(mons, p):
    return np.stack([p[..., 0] ** e0 * p[..., 1] ** a * p[..., 2] ** b * p[..., 3] ** c
                     for (e0, a, b, c) in mons], axis=0)


def mj_moment_3d(mon, n, U, T):
    """App. B moments of the massless MJ distribution in d = 3 up to rank 3:
    <1> = n / (2T), <p^a> = n U^a, <p^a p^b> = n (4 T U^a U^b - T eta^ab),
    <p^a p^b p^c> = n (24 T^2 U^a U^b U^c - 4 T^2 (eta^ab U^c + eta^ac U^b + eta^bc U^a))
    (traceless, as massless moments must be)."""
    idx = [k for k in range(4) for _ in range(mon[k])]
    if len(idx) == 0:
        return n / (2.0 * T)
    if len(idx) == 1:
        return n * U[idx[0]]
    if len(idx) == 2:
        a, b = idx
        return n * (4.0 * T * U[a] * U[b] - T * ETA4[a, b])
    if len(idx) == 3:
        a, b, c = idx
        return n * (24.0 * T * T * U[a] * U[b] * U[c]
                    - 4.0 * T * T * (ETA4[a, b] * U[c] + ETA4[a, c] * U[b] + ETA4[b, c] * U[a]))
    raise ValueError("moments above rank 3 are not needed up to order 3")


class Expansion3:
    """J^(k)(p_i) at the quadrature points and f^eq of Eq. mj-discrete-feq."""

    def __init__(self, quad: Quadrature3, order=2):
        self.quad = quad
        self.order = order
        self.C, self.mons = gram_schmidt_basis_3d(order)
        self.J = self.C @ eval_monomials_3d(self.mons, quad.p)      # (K, Q)

    def feq(self, n, U, T):
        """f^eq_i = w_i sum_k a^(k) J^(k)(p_i), a = C M(n, U, T); shape (Q, ...)."""
        M = np.stack([mj_moment_3d(mon, n, U, T) * np.ones_like(T) for mon in self.mons], axis=0)
        a = np.tensordot(self.C, M, axes=1)
        return self.quad.w.reshape((-1,) + (1,) * np.ndim(T)) * np.tensordot(self.J.T, a, axes=1)


# --------------------------------------------------------------------------
# Sec. 4 and Sec. 6.2 in d = 3.
# --------------------------------------------------------------------------


def landau4(Nvec, Tmat):
    """eps U^a = T^ab U_b: the largest real eigenvalue of A^a_b = T^ac eta_cb
    (LAPACK eig) and its eigenvector with U.U = 1, U^0 > 0; n = U_a N^a.
    Nvec (4, ...), Tmat (4, 4, ...).  Returns eps, U (4, ...), n, ok."""
    shp = Nvec.shape[1:]
    A = np.moveaxis(Tmat.reshape(4, 4, -1), -1, 0) @ ETA4
    finite = np.all(np.isfinite(A), axis=(1, 2)) & np.all(np.isfinite(Nvec.reshape(4, -1)), axis=0)
    A = np.where(finite[:, None, None], A, np.eye(4))
    lam, vec = np.linalg.eig(A)
    idx = np.argmax(lam.real, axis=1)
    C = A.shape[0]
    eps = lam.real[np.arange(C), idx]
    v = vec[np.arange(C), :, idx].real
    norm2 = v[:, 0] ** 2 - v[:, 1] ** 2 - v[:, 2] ** 2 - v[:, 3] ** 2
    ok = (norm2 > 0) & (eps > 0) & (np.abs(lam[np.arange(C), idx].imag) == 0) & finite
    U = v / np.sqrt(np.abs(norm2))[:, None]
    U = U * np.sign(U[:, :1])
    U = U.T.reshape((4,) + shp)
    n = np.sum((ETA4 @ U.reshape(4, -1)) * Nvec.reshape(4, -1), axis=0).reshape(shp)
    return eps.reshape(shp), U, n, ok.reshape(shp)


@dataclass
class Fields3:
    n: np.ndarray
    U: np.ndarray      # (4, ...)
    T: np.ndarray
    eps: np.ndarray
    N: np.ndarray      # (4, ...)
    Tab: np.ndarray    # (4, 4, ...)
    ok: np.ndarray

    def u(self, k):
        """3-velocity component k (1, 2, 3) in units of c."""
        return self.U[k] / self.U[0]


def macroscopic3(f, quad: Quadrature3):
    """Steps 2-5: N^a, T^ab, the Landau frame, n = U.N, T = eps / (3 n)."""
    p = quad.p
    N = np.tensordot(p.T, f, axes=1)
    Tab = np.einsum("qa,qb,q...->ab...", p, p, f)
    eps, U, n, ok = landau4(N, Tab)
    return Fields3(n, U, eps / (3.0 * n), eps, N, Tab, ok)


def collide3(f, quad: Quadrature3, exp: Expansion3, tau):
    """Steps 2-8 per cell: f* = f - (p.U / (p0 tau)) (f - f^eq); a cell
    without a Landau frame is left as it is."""
    fl = macroscopic3(f, quad)
    feq = exp.feq(fl.n, fl.U, fl.T)
    pU = np.tensordot(quad.p * np.array([1.0, -1.0, -1.0, -1.0]), fl.U, axes=([1], [0]))
    om = pU / (quad.p[:, 0].reshape((-1,) + (1,) * (f.ndim - 1)) * tau)
    with np.errstate(invalid="ignore"):
        good = fl.ok & (fl.n > 0) & (fl.T > 0) & np.isfinite(fl.n) & np.isfinite(fl.T)
    # (selected, not multiplied by zero: the frame of a bad cell may be NaN)
    return np.where(good[None], f - om * (f - feq), f), fl


def stream3(fs, shifts):
    """On-lattice pull with periodic wrap: f_i(x) = f*_i(x - n_i); arrays are
    (Q, nz, ny, nx), shifts (Q, 3) in (x, y, z) order."""
    out = np.empty_like(fs)
    for i, (sx, sy, sz) in enumerate(shifts):
        out[i] = np.roll(fs[i], shift=(int(sz), int(sy), int(sx)), axis=(0, 1, 2))
    return out


class Simulation3:
    """Periodic (3+1)-d run: f*(0) = f^eq(n0, U0, T0), then stream + collide.
    ``fs`` holds f* after the last step, ``fields`` the fields of the
    streamed f before that collision."""

    def __init__(self, quad: Quadrature3, exp: Expansion3, nx, ny, nz, tau=1.0):
        self.quad, self.exp, self.tau = quad, exp, tau
        self.shape = (nz, ny, nx)
        self.fs = None
        self.fields = None

    def init(self, n, ux, uy, uz, T):
        g = 1.0 / np.sqrt(1.0 - ux * ux - uy * uy - uz * uz)
        U = np.stack([g, g * ux, g * uy, g * uz])
        self.fs = self.exp.feq(n, U, T)
        self.fields = macroscopic3(self.fs, self.quad)

    def step(self, k=1):
        for _ in range(k):
            f = stream3(self.fs, self.quad.n)
            self.fs, self.fields = collide3(f, self.quad, self.exp, self.tau)
