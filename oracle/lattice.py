"""Velocity-space discretisation of the RLBM, FP64 (oracle; test infrastructure only).

Covers Sec. 5.2-5.3 and App. B, F, G, H of arXiv:1909.04502 for d = 2
(lattice units c = k_B = T0 = 1, so m~ = m and T~ = T).

Population order used throughout the oracle: the order returned by
``quadrature`` (groups in the order given, orbit members in ``fs_orbit``
order, shells innermost for massless tables).
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass
from decimal import Decimal, localcontext
from fractions import Fraction

import numpy as np
from scipy import special

# --------------------------------------------------------------------------
# Stencils (D1): full-symmetric orbits of generator vectors, Sec. 5.3.
# --------------------------------------------------------------------------


def fs_orbit(gen):
    """All vectors obtained from ``gen`` by permuting components and flipping
    signs ("full-symmetric" group, Sec. 5.3 worked example).  Deterministic
    order: sorted descending lexicographically after de-duplication."""
    out = set()
    for perm in itertools.permutations(gen):
        for signs in itertools.product((1, -1), repeat=len(gen)):
            out.add(tuple(s * c for s, c in zip(signs, perm)))
    return sorted(out, reverse=True)


# --------------------------------------------------------------------------
# Massless (m~ = 0) two-dimensional quadratures, App. H "(2+1) dimensions".
# Shell energies and weights are the paper's printed digits.  The weight
# column is stored exactly in the printed order.
# --------------------------------------------------------------------------

MASSLESS_D2 = {
    2: dict(
        groups=[(3, 4), (5, 0)],
        shells=[0.4157745567834790, 2.2942803602790417, 6.2899450829374791],
        weights_printed=[0.0, 0.0888866262411466, 0.0, 0.0348147166961551,
                         0.0017535654166088, 0.0004218743543938],
    ),
    3: dict(
        groups=[(3, 4), (5, 0)],
        shells=[0.3225476896193923, 1.7457611011583465, 4.5366202969211279,
                9.3950709123011331],
        weights_printed=[0.0, 0.0753942630427042, 0.0410206173754781,
                         0.0241670278669858, 0.0044457884155769,
                         0.0026380943565871, 0.0000616926157132,
                         0.0000365655303385],
    ),
}


def massless_weight_table(order, reading="shell_major"):
    """Map the printed weight column of App. H (2+1 dims) to w[group][shell].

    Reading (the paper's sentence about the column order does not fit its
    numbers for d = 2): ``shell_major`` -- for each shell j, the weight of the
    (+-5, 0) group comes first, then that of the (+-3, +-4) group.  Under this
    reading the weights sum to one and the App. F polynomials are orthonormal
    on the stencil.  ``literal`` -- all shells of the first listed group, then
    all shells of the second (the paper's sentence); kept only so that a test
    can show it fails the orthonormality conditions.
    Returns an array ``w[g, j]`` with g indexing ``MASSLESS_D2[order]['groups']``.
    """
    tab = MASSLESS_D2[order]
    ns = len(tab["shells"])
    col = np.asarray(tab["weights_printed"], dtype=np.float64)
    w = np.zeros((2, ns))
    if reading == "shell_major":
        for j in range(ns):
            w[1, j] = col[2 * j]       # (+-5, 0)
            w[0, j] = col[2 * j + 1]   # (+-3, +-4)
    elif reading == "literal":
        w[0, :] = col[:ns]
        w[1, :] = col[ns:]
    else:
        raise ValueError(reading)
    return w


@dataclass
class Quadrature:
    """A discrete momentum set {n_i, p_i^mu, w_i} (D1-D3)."""
    n: np.ndarray        # (Q, 2) integer stencil vectors
    p: np.ndarray        # (Q, 3) momenta p~^mu = (p0, px, py)
    w: np.ndarray        # (Q,) weights
    m: float             # rest mass m~ in units of T0
    order: int           # expansion order N
    v0: float | None = None   # massive parametrisation, Eq. discrete-momentum-vectors

    @property
    def Q(self):
        return len(self.w)

    def velocity(self):
        """Microscopic velocity v^i = p^i / p^0 (Eq. rbe-rta-lattice-friendly)."""
        return self.p[:, 1:] / self.p[:, :1]


def massless_quadrature(order=2, reading="shell_major", keep_zero=False):
    """Eq. ur-discrete-momentum-vectors: p_ij = p0_j (1, n_i/||n_i||), App. H."""
    tab = MASSLESS_D2[order]
    wt = massless_weight_table(order, reading)
    ns, ps, ws = [], [], []
    for g, gen in enumerate(tab["groups"]):
        for vec in fs_orbit(gen):
            norm = math.hypot(*vec)
            for j, p0 in enumerate(tab["shells"]):
                if wt[g, j] == 0.0 and not keep_zero:
                    continue
                ns.append(vec)
                ps.append((p0, p0 * vec[0] / norm, p0 * vec[1] / norm))
                ws.append(wt[g, j])
    return Quadrature(np.array(ns, dtype=np.int64), np.array(ps), np.array(ws), 0.0, order)


def massive_momenta(n, m, v0):
    """Eq. discrete-momentum-vectors / discrete-p0: p~_i = m~ gamma_i (1, v0 n_i)."""
    n = np.asarray(n, dtype=np.float64)
    v2 = v0 * v0 * np.sum(n * n, axis=1)
    gam = 1.0 / np.sqrt(1.0 - v2)
    p = np.empty((len(n), 3))
    p[:, 0] = m * gam
    p[:, 1:] = (m * gam * v0)[:, None] * n
    return p


def stencil_from_groups(groups):
    """Union of FS orbits; returns (vectors (Q,2), group index per vector)."""
    vecs, gidx = [], []
    for g, gen in enumerate(groups):
        for v in fs_orbit(gen):
            vecs.append(v)
            gidx.append(g)
    return np.array(vecs, dtype=np.int64), np.array(gidx)


# --------------------------------------------------------------------------
# Orthonormal polynomials, App. F "(2+1) dimensions" (any m~), order <= 2.
# Basis order: J0, J1_0, J1_x, J1_y, J2_00, J2_0x, J2_xx, J2_0y, J2_xy.
# --------------------------------------------------------------------------


def appF_polys_d2(p, m):
    """Evaluate the nine App. F (2+1)-d polynomials at momenta p (..., 3)."""
    p0, px, py = p[..., 0], p[..., 1], p[..., 2]
    Gt = m + 1.0
    s1 = math.sqrt((2.0 * m * (m + 3.0) + 3.0) / Gt)
    s2 = math.sqrt(3.0 * Gt + m * m)
    J = [
        np.ones_like(p0),
        p0 - Gt,
        px / math.sqrt(Gt),
        py / math.sqrt(Gt),
        p0 * (-m - 2.0) + 0.5 * m * (m + 4.0) + 0.5 * p0 * p0 + 1.0,
        p0 * px * (m + 1.0) / (Gt * s1) + px * (-m * (m + 3.0) - 3.0) / (Gt * s1),
        -p0 * p0 / (2.0 * s2) + px * px / s2 + m * m / (2.0 * s2),
        p0 * py * (m + 1.0) / (Gt * s1) + py * (-m * (m + 3.0) - 3.0) / (Gt * s1),
        px * py / s2,
    ]
    return np.stack(J, axis=0)


def appG_proj_d2(U, T, m):
    """App. G "(2+1) dimensions": b^(k)(U, T), with a^(k) = n b^(k) (T0 = 1).

    U has shape (3, ...) (contravariant U^mu), T has shape (...).  Returns
    (9, ...) in the basis order of ``appF_polys_d2``.
    G = zeta + 1 with zeta = m/T; G~ = m~ + 1.
    """
    U0, Ux, Uy = U[0], U[1], U[2]
    G = m / T + 1.0
    Gt = m + 1.0
    s1 = math.sqrt((2.0 * m * (m + 3.0) + 3.0) / Gt)
    s2 = math.sqrt(3.0 * Gt + m * m)
    b = [
        1.0 / (m + T),
        U0 - Gt / (m + T),
        Ux / math.sqrt(Gt),
        Uy / math.sqrt(Gt),
        0.5 * U0 * U0 * T * (m * m / (G * T * T) + 3.0)
        + 0.5 * ((m * (m + 4.0) + 2.0) / (m + T) - T) + U0 * (-m - 2.0),
        U0 * Ux * (m + 1.0) * T * (m * m / (T * T) + 3.0 * G) / (G * Gt * s1)
        - Ux * (m * (m + 3.0) + 3.0) / (Gt * s1),
        -U0 * U0 * (3.0 * G * T * T + m * m) / (2.0 * G * T * s2)
        + Ux * Ux * T * (m * m / (T * T) + 3.0 * G) / (G * s2)
        + (3.0 * G * T * T + m * m) / (2.0 * G * T * s2),
        U0 * Uy * (m + 1.0) * T * (m * m / (T * T) + 3.0 * G) / (G * Gt * s1)
        - Uy * (m * (m + 3.0) + 3.0) / (Gt * s1),
        Ux * Uy * T * (m * m / (T * T) + 3.0 * G) / (G * s2),
    ]
    return np.stack([np.broadcast_to(x, np.shape(T)) for x in b], axis=0)


# --------------------------------------------------------------------------
# Exact integrals against the weight omega (Sec. 5.2, normalisation Eq.
# numerical-normalization-cond; App. F (2+1)-d weight e^m/(2 pi) exp(-p0)).
# d^2p / p0 = dp0 dtheta on the mass shell, |p| = sqrt(p0^2 - m^2).
# --------------------------------------------------------------------------


def _angular(a, b):
    """int_0^{2 pi} cos^a sin^b dtheta / (2 pi)."""
    if a % 2 or b % 2:
        return 0.0
    num = 1.0
    for k in range(a - 1, 0, -2):
        num *= k
    for k in range(b - 1, 0, -2):
        num *= k
    den = 1.0
    for k in range(a + b, 0, -2):
        den *= k
    return num / den


def _radial(c, k2, m):
    """e^m int_m^inf e^{-p0} p0^c (p0^2 - m^2)^{k2} dp0 with p0 = m + s:
    int_0^inf e^{-s} (m+s)^c s^{k2} (2m+s)^{k2} ds, expanded with positive
    coefficients so no cancellation occurs."""
    poly = np.array([1.0])
    for _ in range(c):
        poly = np.convolve(poly, [m, 1.0])
    for _ in range(k2):
        poly = np.convolve(poly, [0.0, 2.0 * m, 1.0])
    return float(sum(coef * math.factorial(q) for q, coef in enumerate(poly)))


def omega_moment(c, a, b, m):
    """E_omega[p0^c px^a py^b] = int omega p0^c px^a py^b d^2p/p0, d = 2."""
    ang = _angular(a, b)
    if ang == 0.0:
        return 0.0
    return ang * _radial(c, (a + b) // 2, m)


# --------------------------------------------------------------------------
# Gram-Schmidt (Sec. 5.2) from V = {1, p^a, p^a p^b, p^a p^b p^c, ...}.
# Monomials are exponent triples (c, a, b) of p0^c px^a py^b.
# --------------------------------------------------------------------------


def monomials(order):
    """Generating set V of Sec. 5.2 up to ``order``: index tuples alpha_1 <=
    ... <= alpha_n over (0, x, y), returned as exponent triples."""
    out = []
    for deg in range(order + 1):
        for idx in itertools.combinations_with_replacement(range(3), deg):
            out.append((idx.count(0), idx.count(1), idx.count(2)))
    return out


def eval_monomials(mons, p):
    return np.stack([p[..., 0] ** c * p[..., 1] ** a * p[..., 2] ** b for (c, a, b) in mons], axis=0)


def gram_schmidt_basis(order, m, tol=1e-9):
    """Orthonormal polynomials J = C phi under omega (Eq. mj-orthogonal-conditions,
    continuum side), by classical Gram-Schmidt on V in order, dropping
    members that are linearly dependent on the mass shell p0^2 = m^2 + |p|^2.
    Returns (C, mons): C has shape (K, len(mons))."""
    mons = monomials(order)
    nm = len(mons)
    Gm = np.empty((nm, nm))
    for i, (c1, a1, b1) in enumerate(mons):
        for j, (c2, a2, b2) in enumerate(mons):
            Gm[i, j] = omega_moment(c1 + c2, a1 + a2, b1 + b2, m)
    rows = []
    for i in range(nm):
        v = np.zeros(nm)
        v[i] = 1.0
        for r in rows:
            v = v - (r @ Gm @ v) * r
        nrm2 = v @ Gm @ v
        if nrm2 <= tol * Gm[i, i]:
            continue
        rows.append(v / math.sqrt(nrm2))
    return np.array(rows), mons


# --------------------------------------------------------------------------
# Maxwell-Juttner moments from the Z-tensors of App. B.
# --------------------------------------------------------------------------


def A_ratio(j, zeta, d=2):
    """A_j / A_1 with A_n = 2^{(d+1)/2} pi^{(d-1)/2} zeta^{n+(d-1)/2} K_{n+(d-1)/2}(zeta)
    (App. B).  zeta = 0 uses the limit zeta^nu K_nu(zeta) -> 2^{nu-1} Gamma(nu)."""
    h = (d - 1) / 2.0
    zeta = np.asarray(zeta, dtype=np.float64)
    if np.all(zeta == 0.0):
        lim = lambda nu: 2.0 ** (nu - 1.0) * special.gamma(nu)
        return np.full(zeta.shape, lim(j + h) / lim(1 + h))
    # ratio of exponentially scaled Bessel functions (the e^{-zeta} cancels)
    return zeta ** (j - 1) * special.kve(j + h, zeta) / special.kve(1 + h, zeta)


def A_ratio_half_integer(j, zeta):
    """A_j / A_1 for d = 2 (Bessel orders j + 1/2 and 3/2), evaluated in
    whatever float type zeta carries: K_{n+1/2}(z) = sqrt(pi/(2z)) e^{-z}
    R_n(z) with the terminating series R_n(z) = sum_{k<=n} (n+k)!/(k!(n-k)!)
    (2z)^{-k} (textbook closed form of the half-integer modified Bessel
    function), so A_j/A_1 = zeta^{j-1} R_j(zeta) / R_1(zeta) without special
    functions.  zeta > 0."""
    def R(nu):
        tot = zeta * 0 + 1
        for k in range(1, nu + 1):
            c = math.factorial(nu + k) // (math.factorial(k) * math.factorial(nu - k))
            tot = tot + c / (2 * zeta) ** k
        return tot
    return zeta ** (j - 1) * R(j) / R(1)


def _pairings(idx):
    """All ways to choose k disjoint index pairs from positions, for every k.
    Yields (pairs, singles)."""
    idx = list(idx)
    if not idx:
        yield [], []
        return
    first, rest = idx[0], idx[1:]
    for pairs, singles in _pairings(rest):
        yield pairs, [first] + singles
    for j in range(len(rest)):
        partner = rest[j]
        others = rest[:j] + rest[j + 1:]
        for pairs, singles in _pairings(others):
            yield [(first, partner)] + pairs, singles


ETA = np.diag([1.0, -1.0, -1.0])


def mj_moment_ld(alphas, n, U, T, m):
    """mj_moment for d = 2 and m > 0 in np.longdouble (the same App. B
    formula, with A_j/A_1 from A_ratio_half_integer)."""
    r = len(alphas)
    T = np.asarray(T, dtype=np.longdouble)
    zeta = np.longdouble(m) / T
    total = np.longdouble(0)
    for pairs, singles in _pairings(range(r)):
        k = len(pairs)
        term = (-1) ** k * A_ratio_half_integer(r - k, zeta)
        for (i, j) in pairs:
            term = term * np.longdouble(ETA[alphas[i], alphas[j]])
        for s_ in singles:
            term = term * U[alphas[s_]]
        total = total + term
    return np.asarray(n, dtype=np.longdouble) * T ** (r - 1) * total


def mj_moment(alphas, n, U, T, m, d=2):
    """int f_MJ p^{alpha_1} ... p^{alpha_r} d^dp/p0 with f_MJ normalised so that
    N_E^alpha = n U^alpha (Eq. first-moment-eq, Eq. phys-normalization):
    B Z^{alpha...} = n T^{r-1} sum_k (-1)^k (A_{r-k}/A_1) <U_{r-2k} eta_k>
    (App. B).  ``alphas`` is a tuple of component indices in {0,1,2}.
    U: (3, ...), T, n: (...)."""
    r = len(alphas)
    zeta = m / np.asarray(T)
    total = 0.0
    for pairs, singles in _pairings(range(r)):
        k = len(pairs)
        term = (-1.0) ** k * A_ratio(r - k, zeta, d)
        for (i, j) in pairs:
            term = term * ETA[alphas[i], alphas[j]]
        for s in singles:
            term = term * U[alphas[s]]
        total = total + term
    return n * np.asarray(T) ** (r - 1) * total


def mj_monomial_moment(mon, n, U, T, m):
    """MJ moment of the monomial p0^c px^a py^b."""
    c, a, b = mon
    return mj_moment((0,) * c + (1,) * a + (2,) * b, n, U, T, m)


# --------------------------------------------------------------------------
# Basis + projections used by the equilibrium (Sec. 5.2, Eq. mj-discrete-feq).
# --------------------------------------------------------------------------


class Expansion:
    """J^(k)(p_i) at the quadrature points, and a^(k)(n, U, T).

    order <= 2: App. F polynomials and App. G projections (closed forms).
    order == 3: Gram-Schmidt basis and projections a_k = int f_MJ J_k d^2p/p0
    assembled from the App. B moments (the order-3 formulas are in the
    paper's missing supplement).  For m > 0 the projections and the sum
    f^eq = w sum_k a_k J_k run in np.longdouble: the Gram-Schmidt
    coefficients of p0 ~ m~ monomials are large and cancel, and in double
    the equilibrium loses 7.5e-13 of max |f| at m~ = 15.
    """

    def __init__(self, quad: Quadrature, order=None, source=None):
        self.quad = quad
        self.order = quad.order if order is None else order
        self.m = quad.m
        if source is None:
            source = "appFG" if self.order == 2 else "gram_schmidt"
        self.source = source
        self.extended = False
        if source == "appFG":
            if self.order != 2:
                raise ValueError("App. F/G closed forms are printed up to order 2")
            self.J = appF_polys_d2(quad.p, self.m)          # (9, Q)
        else:
            # the basis and its values at the quadrature points in 50-digit
            # decimal arithmetic, rounded once: in double the cancellation
            # between monomials of p0 ~ m~ costs up to 1e-10 at m~ = 20
            with localcontext() as ctx:
                ctx.prec = 50
                rows, self.mons = _gram_schmidt_decimal(self.order, self.m)
                self.C = np.array([[float(x) for x in r] for r in rows])
                self.C_ld = np.array([[np.longdouble(str(x)) for x in r] for r in rows])
                pw = lambda x, k: math.prod([x] * k, start=Decimal(1))
                J = []
                for p0, px, py in quad.p:
                    phi = [pw(Decimal(p0), c) * pw(Decimal(px), a) * pw(Decimal(py), b)
                           for (c, a, b) in self.mons]
                    J.append([sum(r[q] * phi[q] for q in range(len(phi))) for r in rows])
            self.J = np.array([[float(x) for x in row] for row in J]).T              # (K, Q)
            self.J_ld = np.array([[np.longdouble(str(x)) for x in row] for row in J]).T
        self.extended = source == "gram_schmidt" and self.m > 0.0

    def projections(self, n, U, T):
        """a^(k) = n b^(k), shape (K, ...)."""
        if self.source == "appFG":
            return n * appG_proj_d2(U, T, self.m)
        Mm = np.stack([mj_monomial_moment(mon, n, U, T, self.m) * np.ones_like(T)
                       for mon in self.mons], axis=0)
        return np.tensordot(self.C, Mm, axes=1)

    def feq(self, n, U, T):
        """Eq. mj-discrete-feq: f^eq_i = w_i sum_k a^(k) J^(k)(p_i), shape (Q, ...)."""
        if self.extended:
            ld = np.longdouble
            n_, T_ = np.asarray(n, dtype=ld), np.asarray(T, dtype=ld)
            U_ = np.asarray(U, dtype=ld)
            Mm = np.stack([mj_moment_ld((0,) * c + (1,) * a + (2,) * b, n_, U_, T_, self.m) * np.ones_like(T_)
                           for (c, a, b) in self.mons], axis=0)
            a_ = np.tensordot(self.C_ld, Mm, axes=1)
            w = np.asarray(self.quad.w, dtype=ld).reshape((-1,) + (1,) * np.ndim(T))
            return (w * np.tensordot(self.J_ld.T, a_, axes=1)).astype(np.float64)
        a = self.projections(n, U, T)
        return self.quad.w.reshape((-1,) + (1,) * np.ndim(T)) * np.tensordot(self.J.T, a, axes=1)


# --------------------------------------------------------------------------
# Quadrature search (Sec. 5.3, Eq. quadrature-problem).
# --------------------------------------------------------------------------


def orthonormality_system(groups, m, v0, order=2, basis="appF"):
    """A(v0) w = b from Eq. mj-orthogonal-conditions with one unknown weight per
    FS group: rows are the pairs (l <= k) of basis polynomials, b = delta_lk."""
    vecs, gidx = stencil_from_groups(groups)
    p = massive_momenta(vecs, m, v0)
    if basis == "appF":
        J = appF_polys_d2(p, m)
    else:
        C, mons = gram_schmidt_basis(order, m)
        J = C @ eval_monomials(mons, p)
    K = J.shape[0]
    rows, rhs = [], []
    for l in range(K):
        for k in range(l, K):
            prod = J[l] * J[k]
            rows.append([prod[gidx == g].sum() for g in range(len(groups))])
            rhs.append(1.0 if l == k else 0.0)
    return np.array(rows), np.array(rhs)


def solve_group_weights(groups, m, v0, order=2, basis="appF"):
    """Least-squares solution of A(v0) w = b (LAPACK); returns (w, residual)."""
    A, b = orthonormality_system(groups, m, v0, order, basis)
    w, *_ = np.linalg.lstsq(A, b, rcond=None)
    return w, float(np.max(np.abs(A @ w - b)))


def _omega_moment_fraction(c, a, b, m):
    """E_omega[p0^c px^a py^b] (d = 2) as an exact rational for a rational m:
    the angular factor (a-1)!!(b-1)!!/(a+b)!! and the radial integral
    int_0^inf e^{-s} (m+s)^c (s (2m+s))^{(a+b)/2} ds expanded into s^q e^{-s}
    terms (each q!), the same formulas as ``omega_moment``."""
    if a % 2 or b % 2:
        return Fraction(0)
    ang = Fraction(1)
    for k in range(a - 1, 0, -2):
        ang *= k
    for k in range(b - 1, 0, -2):
        ang *= k
    for k in range(a + b, 0, -2):
        ang /= k
    poly = [Fraction(1)]
    for _ in range(c):
        poly = [(poly[q] * m if q < len(poly) else 0) + (poly[q - 1] if q else 0) for q in range(len(poly) + 1)]
    for _ in range((a + b) // 2):
        nxt = [Fraction(0)] * (len(poly) + 2)
        for q, x in enumerate(poly):
            nxt[q + 1] += 2 * m * x
            nxt[q + 2] += x
        poly = nxt
    return ang * sum(x * math.factorial(q) for q, x in enumerate(poly))


def _gram_schmidt_decimal(order, m):
    """``gram_schmidt_basis`` in decimal arithmetic at the current context's
    precision, on exact omega-moments: rows of C as lists of Decimal."""
    mons = monomials(order)
    nm = len(mons)
    mf = Fraction(m)
    D = lambda fr: Decimal(fr.numerator) / Decimal(fr.denominator)
    G = [[D(_omega_moment_fraction(c1 + c2, a1 + a2, b1 + b2, mf)) for (c2, a2, b2) in mons]
         for (c1, a1, b1) in mons]
    Gdot = lambda u, v: sum(u[i] * sum(G[i][j] * v[j] for j in range(nm)) for i in range(nm))
    rows = []
    for i in range(nm):
        v = [Decimal(0)] * nm
        v[i] = Decimal(1)
        for r in rows:
            pr = Gdot(r, v)
            v = [v[k] - pr * r[k] for k in range(nm)]
        n2 = Gdot(v, v)
        if n2 <= Decimal("1e-9") * G[i][i]:
            continue
        nrm = n2.sqrt()
        rows.append([x / nrm for x in v])
    return rows, mons


def _basis_at_momenta_decimal(rows, mons, m, v0, vecs):
    """J = C phi at the momenta of Eq. discrete-momentum-vectors / discrete-p0
    for the stencil vectors ``vecs``, in decimal arithmetic (Q lists of K)."""
    pw = lambda x, k: math.prod([x] * k, start=Decimal(1))   # Decimal 0 ** 0 is an error
    dv0, dm = Decimal(v0), Decimal(Fraction(m).numerator) / Decimal(Fraction(m).denominator)
    out = []
    for nx, ny in vecs:
        vx, vy = dv0 * int(nx), dv0 * int(ny)
        gam = 1 / (1 - vx * vx - vy * vy).sqrt()
        p0, px, py = dm * gam, dm * gam * vx, dm * gam * vy
        phi = [pw(p0, c) * pw(px, a) * pw(py, b) for (c, a, b) in mons]
        out.append([sum(r[q] * phi[q] for q in range(len(mons))) for r in rows])
    return out


def solve_group_weights_exact(groups, m, v0, order=2, digits=50):
    """The group weights of Eq. mj-orthogonal-conditions in ``digits``-digit
    decimal arithmetic: Gram-Schmidt (Sec. 5.2) on the generating set V with
    exact omega-moments, J at the stencil momenta of Eq.
    discrete-momentum-vectors / discrete-p0, the conditions summed per FS
    group, and the least-squares solution through the normal equations
    (Gaussian elimination with partial pivoting).  The same steps as
    ``solve_group_weights`` with the GS basis; in double they lose up to 1e-8
    of a weight at order 3 (m~ = 20) to the conditioning of the monomial
    basis, here the result is limited by the final rounding.  Returns
    (w, residual) as floats."""
    with localcontext() as ctx:
        ctx.prec = digits
        rows, mons = _gram_schmidt_decimal(order, m)
        K = len(rows)
        vecs, gidx = stencil_from_groups(groups)
        ng = len(groups)
        A = [[Decimal(0)] * ng for _ in range(K * (K + 1) // 2)]
        bvec = []
        for l in range(K):
            for k in range(l, K):
                bvec.append(Decimal(1) if l == k else Decimal(0))
        for J, g in zip(_basis_at_momenta_decimal(rows, mons, m, v0, vecs), gidx):
            rr = 0
            for l in range(K):
                for k in range(l, K):
                    A[rr][g] += J[l] * J[k]
                    rr += 1
        # normal equations A^T A w = A^T b
        N = [[sum(A[r][i] * A[r][j] for r in range(len(A))) for j in range(ng)] for i in range(ng)]
        y = [sum(A[r][i] * bvec[r] for r in range(len(A))) for i in range(ng)]
        for c in range(ng):
            piv = max(range(c, ng), key=lambda r: abs(N[r][c]))
            N[c], N[piv], y[c], y[piv] = N[piv], N[c], y[piv], y[c]
            for r in range(c + 1, ng):
                f = N[r][c] / N[c][c]
                N[r] = [N[r][j] - f * N[c][j] for j in range(ng)]
                y[r] -= f * y[c]
        w = [Decimal(0)] * ng
        for c in range(ng - 1, -1, -1):
            w[c] = (y[c] - sum(N[c][j] * w[j] for j in range(c + 1, ng))) / N[c][c]
        res = max(abs(sum(A[r][g] * w[g] for g in range(ng)) - bvec[r]) for r in range(len(A)))
        return np.array([float(x) for x in w]), float(res)


def massive_quadrature(groups, m, v0, order=2, basis=None, drop_zero=1e-300, exact=True):
    """Quadrature on an FS stencil with the weights of
    ``solve_group_weights_exact`` (``exact``) or of ``solve_group_weights``
    in double with the given basis."""
    if basis is None:
        basis = "appF" if order == 2 else "gs"
    if exact:
        wg, res = solve_group_weights_exact(groups, m, v0, order)
    else:
        wg, res = solve_group_weights(groups, m, v0, order, basis)
    vecs, gidx = stencil_from_groups(groups)
    w = wg[gidx]
    keep = np.abs(w) > drop_zero
    p = massive_momenta(vecs, m, v0)
    return Quadrature(vecs[keep], p[keep], w[keep], m, order, v0), res


def search_v0(groups, m, order=2, basis=None, npts=2000, v0_lo=None, v0_hi=None):
    """Line search of Sec. 5.3: scan v0 in (0, 1/max||n||) and return the list
    of v0 values where the system is consistent and all weights are >= 0."""
    if basis is None:
        basis = "appF" if order == 2 else "gs"
    vmax = 1.0 / max(math.hypot(*g) for g in groups if any(g))
    lo = v0_lo if v0_lo is not None else vmax * 1e-3
    hi = v0_hi if v0_hi is not None else vmax * (1 - 1e-9)
    ok = []
    for v0 in np.linspace(lo, hi, npts):
        w, res = solve_group_weights(groups, m, v0, order, basis)
        if res < 1e-9 and np.all(w >= 0.0):
            ok.append(float(v0))
    return ok
