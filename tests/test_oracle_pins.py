"""Pins of the FP64 oracle against what arXiv:1909.04502 and mathematics fix.

None of these tests compares the oracle with itself: each check uses a value
printed in the paper (tests/golden/), a closed form, an independent numerical
integration, a textbook routine (Gauss-Laguerre nodes), or an invariant.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy import special

from oracle import lattice as L
from oracle import physics as P
from oracle import scheme as S

GOLD = os.path.join(os.path.dirname(__file__), "golden")
RNG = np.random.default_rng(1909)


def gold(name):
    with open(os.path.join(GOLD, name)) as fh:
        return json.load(fh)


# ---------------------------------------------------------------- quadratures


@pytest.mark.parametrize("order", [2, 3])
def test_massless_tables_match_printed(order):
    g = gold("massless_d2_tables.json")["order%d" % order]
    tab = L.MASSLESS_D2[order]
    assert [tuple(x) for x in g["groups"]] == tab["groups"]
    assert np.array_equal(np.array(g["shells"]), np.array(tab["shells"]))
    assert np.array_equal(np.array(g["weights_column"], dtype=float), np.array(tab["weights_printed"]))


def test_main_text_listing_agrees_with_shell_major_reading():
    g = gold("massless_d2_tables.json")["order2"]
    w = L.massless_weight_table(2, "shell_major")
    # main text (Sec. 5.3): group index 1 carries (0, 0, 0.00175...) -> (+-5, 0)
    assert np.allclose(w[1], g["main_text_w1j"], atol=1e-11)
    assert np.allclose(w[0], g["main_text_w2j"], atol=1e-11)


@pytest.mark.parametrize("order,Q", [(2, 28), (3, 44)])
def test_massless_weights_sum_to_one(order, Q):
    q = L.massless_quadrature(order)
    assert q.Q == Q
    assert abs(q.w.sum() - 1.0) < 5e-15
    # the literal reading of the column order fails the normalisation
    assert abs(L.massless_quadrature(order, reading="literal").w.sum() - 1.0) > 0.05


@pytest.mark.parametrize("order", [2, 3])
def test_massless_shells_are_gauss_laguerre_nodes(order):
    """d = 2 shell energies are the roots of the Laguerre polynomial L_{N+1}."""
    nodes, _ = np.polynomial.laguerre.laggauss(order + 1)
    assert np.allclose(np.sort(L.MASSLESS_D2[order]["shells"]), np.sort(nodes), rtol=0, atol=2e-15)


def _continuum_integral(func, m, ns=100, nth=64):
    """int omega F d^2p/p0 with omega = e^m/(2 pi) e^{-p0}: Gauss-Laguerre in
    s = p0 - m times the uniform rule in theta (exact for the polynomials used)."""
    s, ws = np.polynomial.laguerre.laggauss(ns)
    th = 2 * np.pi * np.arange(nth) / nth
    S_, TH = np.meshgrid(s, th, indexing="ij")
    p0 = m + S_
    pr = np.sqrt(S_ * (2 * m + S_))
    p = np.stack([p0, pr * np.cos(TH), pr * np.sin(TH)], axis=-1)
    vals = func(p)
    return np.tensordot(vals, ws, axes=([-2], [0])).mean(axis=-1)


@pytest.mark.parametrize("m", [0.0, 1.0, 5.0, 10.0])
def test_appF_polynomials_orthonormal_in_continuum(m):
    G = _continuum_integral(lambda p: np.einsum("k...,l...->kl...", L.appF_polys_d2(p, m), L.appF_polys_d2(p, m)), m)
    assert np.abs(G - np.eye(9)).max() < 1e-11


@pytest.mark.parametrize("m", [0.0, 1.0, 5.0])
def test_omega_moments_closed_form_vs_numeric(m):
    for (c, a, b) in [(0, 0, 0), (1, 0, 0), (2, 2, 0), (3, 2, 2), (1, 4, 0), (0, 0, 6), (2, 1, 1)]:
        num = _continuum_integral(lambda p: p[..., 0] ** c * p[..., 1] ** a * p[..., 2] ** b, m)
        assert abs(num - L.omega_moment(c, a, b, m)) < 1e-10 * max(1.0, abs(num))


@pytest.mark.parametrize("m", [0.0, 1.0, 5.0, 10.0])
def test_gram_schmidt_reproduces_appF(m):
    """Gram-Schmidt on V (Sec. 5.2) yields exactly the printed App. F polynomials
    (printed order: J2_00, J2_0x, J2_xx, J2_0y, J2_xy)."""
    C, mons = L.gram_schmidt_basis(2, m)
    assert C.shape[0] == 9
    p = RNG.uniform(-3, 3, (20, 3))
    p[:, 0] = np.sqrt(m * m + p[:, 1] ** 2 + p[:, 2] ** 2)
    gs = (C @ L.eval_monomials(mons, p))[[0, 1, 2, 3, 4, 5, 7, 6, 8]]
    assert np.abs(gs - L.appF_polys_d2(p, m)).max() < 1e-12


def test_order3_basis_has_sixteen_members():
    """On the mass shell the degree <= 3 polynomials in (p0, px, py) span
    16 dimensions (p0^2 is not independent)."""
    for m in (0.0, 1.2):
        C, _ = L.gram_schmidt_basis(3, m)
        assert C.shape[0] == 16


def test_appF_orthonormal_on_massless_order2_quadrature():
    q = L.massless_quadrature(2)
    J = L.appF_polys_d2(q.p, 0.0)
    assert np.abs((J * q.w) @ J.T - np.eye(9)).max() < 1e-13
    ql = L.massless_quadrature(2, reading="literal")
    Jl = L.appF_polys_d2(ql.p, 0.0)
    assert np.abs((Jl * ql.w) @ Jl.T - np.eye(9)).max() > 0.1


def test_order3_basis_orthonormal_on_massless_order3_quadrature():
    q = L.massless_quadrature(3)
    C, mons = L.gram_schmidt_basis(3, 0.0)
    J = C @ L.eval_monomials(mons, q.p)
    assert np.abs((J * q.w) @ J.T - np.eye(16)).max() < 5e-12


def test_mass5_worked_example_weights():
    g = gold("mass5_worked_example.json")
    groups = [tuple(x) for x in g["groups"]]
    w, res = L.solve_group_weights(groups, g["m"], g["v0"])
    assert res < 1e-12
    assert np.allclose(w, g["weights"], rtol=0, atol=5e-14)   # printed to ~16 decimals
    vecs, _ = L.stencil_from_groups(groups)
    assert len(vecs) == g["n_velocities_full"]
    w2, _ = L.solve_group_weights(groups, g["m"], g["v0_w2_zero"])
    w3, _ = L.solve_group_weights(groups, g["m"], g["v0_w3_zero"])
    assert abs(w2[1]) < 1e-7 and abs(w3[2]) < 1e-7
    assert len(vecs) - 4 == g["n_velocities_pruned"]
    # weights sum to one (Eq. numerical-normalization-cond)
    sizes = [len(L.fs_orbit(x)) for x in groups]
    assert abs(np.dot(sizes, w) - 1.0) < 1e-13


def test_exact_weights_match_printed_worked_example():
    """The decimal-arithmetic solve gives the printed Sec. 5.3 weights and
    leaves no residual above its working precision."""
    g = gold("mass5_worked_example.json")
    w, res = L.solve_group_weights_exact([tuple(x) for x in g["groups"]], g["m"], g["v0"])
    assert res < 1e-40
    assert np.allclose(w, g["weights"], rtol=0, atol=5e-14)


@pytest.mark.parametrize("m,v0", [(20.0, 0.175), (5.0, 0.2199)])
def test_exact_order3_weights_reproduce_omega_moments(m, v0):
    """App. H stencil G_D^(o3) (order 3) with the exact weights: the rule
    integrates every product of two members of V (degree <= 6) like the
    weight omega itself, i.e. Eq. mj-orthogonal-conditions written in the
    monomial basis (J = C phi with C invertible), checked against the exact
    rational omega-moments without any Gram-Schmidt step (the double-
    precision LAPACK solve misses them by 1e-11 to 1e-10)."""
    groups = [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (3, 1), (3, 2), (3, 3), (4, 0), (4, 2)]
    q, res = L.massive_quadrature(groups, m, v0, order=3)
    assert res < 1e-35
    mons = L.monomials(3)
    phi = L.eval_monomials(mons, q.p)
    worst = 0.0
    for i, (c1, a1, b1) in enumerate(mons):
        for j, (c2, a2, b2) in enumerate(mons):
            exact = float(L._omega_moment_fraction(c1 + c2, a1 + a2, b1 + b2, Fraction(m)))
            got = math.fsum(q.w * phi[i] * phi[j])
            scale = math.fsum(np.abs(q.w * phi[i] * phi[j]))
            worst = max(worst, abs(got - exact) / scale)
    assert worst < 1e-14


def test_mass5_search_finds_printed_window_and_failing_stencil():
    g = gold("mass5_worked_example.json")
    ok = L.search_v0([tuple(x) for x in g["groups"]], 5.0, npts=401, v0_lo=0.2720, v0_hi=0.2736)
    assert ok and min(ok) <= g["v0"] <= max(ok)
    # the window of non-negative weights is bounded by the two pruning values
    step = 0.0016 / 400
    assert abs(min(ok) - g["v0_w2_zero"]) < 1.01 * step
    assert abs(max(ok) - g["v0_w3_zero"]) < 1.01 * step
    bad = L.search_v0([tuple(x) for x in g["v0_failing_stencil_groups"]], 5.0, npts=300)
    assert bad == []


# ------------------------------------------------------------- equilibrium


def _mj_numeric(alphas, n, U, T, m, ns=100, nth=256):
    """int f_MJ p^a... d^2p/p0 for the analytic Maxwell-Juttner distribution
    (Eq. maxwell-juttner with B of Eq. phys-normalization, d = 2), by
    quadrature in (p0, theta).  Independent of App. B and of the lattice."""
    U = np.asarray(U, dtype=float)
    z = m / T
    zK = math.sqrt(2.0) * special.gamma(1.5) if m == 0 else z ** 1.5 * special.kv(1.5, z)
    B = n / (T * T * 2 ** 1.5 * math.sqrt(math.pi) * zK)
    a = (U[0] - math.hypot(U[1], U[2])) / T        # slowest exponential decay rate
    s, ws = np.polynomial.laguerre.laggauss(ns)
    th = 2 * np.pi * np.arange(nth) / nth
    S_, TH = np.meshgrid(s / a, th, indexing="ij")
    p0 = m + S_
    pr = np.sqrt(S_ * (2 * m + S_))
    p = [p0, pr * np.cos(TH), pr * np.sin(TH)]
    Up = U[0] * p0 - U[1] * p[1] - U[2] * p[2]
    integrand = B * np.exp(-Up / T + a * S_)
    for al in alphas:
        integrand = integrand * p[al]
    return float(np.tensordot(integrand, ws, axes=([0], [0])).mean() * 2 * np.pi / a)


def test_mj_numeric_integral_normalisation():
    n, T, m = 1.3, 0.9, 0.0
    U = P.four_velocity(np.array(0.3), np.array(-0.2))
    assert abs(_mj_numeric((0,), n, U, T, m) - n * U[0]) < 1e-10
    assert abs(_mj_numeric((2,), n, U, T, m) - n * U[2]) < 1e-10


@pytest.mark.parametrize("m", [0.0, 1.0, 5.0])
def test_z_tensor_moments_match_numeric_integrals(m):
    """App. B Z-tensor moments vs direct integration of f_MJ, orders 0-3."""
    n, T = 1.2, 0.8 if m == 0 else 1.1
    U = P.four_velocity(np.array(0.25), np.array(0.15))
    for alphas in [(), (0,), (1,), (0, 0), (0, 1), (1, 2), (2, 2), (0, 0, 0), (0, 1, 1), (1, 1, 2), (2, 2, 2)]:
        num = _mj_numeric(alphas, n, U, T, m)
        ana = float(L.mj_moment(alphas, n, U, np.array(T), m))
        assert abs(num - ana) < 1e-9 * max(1.0, abs(num)), (alphas, num, ana)


@pytest.mark.parametrize("m", [0.0, 1.0, 5.0])
def test_appG_projections_match_numeric_integrals(m):
    """App. G: a^(k) = n b^(k) = int f_MJ J^(k) d^2p/p0 (Eq. mj-projection-coefficients)."""
    n, T = 1.1, 1.25
    U = P.four_velocity(np.array(-0.3), np.array(0.2))
    b = L.appG_proj_d2(U, np.array(T), m) * n
    # J^(k) expressed through monomials via Gram-Schmidt (it reproduces App. F,
    # see test_gram_schmidt_reproduces_appF), integrated term by term
    C, mons = L.gram_schmidt_basis(2, m)
    C = C[[0, 1, 2, 3, 4, 5, 7, 6, 8]]
    num_m = np.array([_mj_numeric((0,) * c + (1,) * a + (2,) * bb, n, U, T, m) for (c, a, bb) in mons])
    assert np.abs(C @ num_m - b).max() < 1e-9


def _eos_energy_tensor(n, U, T, m):
    eps = n * P.energy_per_particle(T, m)
    Pp = n * T
    return (eps + Pp) * np.einsum("a...,b...->ab...", U, U) - Pp * P.ETA.reshape(3, 3, *([1] * np.ndim(T)))


def _random_state(shape, umax=0.6):
    n = RNG.uniform(0.5, 2.0, shape)
    T = RNG.uniform(0.6, 1.6, shape)
    r = RNG.uniform(0, umax, shape)
    th = RNG.uniform(0, 2 * np.pi, shape)
    return n, r * np.cos(th), r * np.sin(th), T


@pytest.mark.parametrize("case", ["massless2", "massless3", "mass5"])
def test_equilibrium_recovers_exact_first_and_second_moments(case):
    """Eq. first-moment-eq / second-moment-eq: sum f^eq p = n U and
    sum f^eq p p = (eps + P) U U - P eta, with eps/n from Bessel functions."""
    if case == "mass5":
        q, _ = L.massive_quadrature([(0, 0), (1, 0), (1, 1), (2, 1), (2, 2), (3, 1)], 5.0, 0.2726)
    else:
        q = L.massless_quadrature(int(case[-1]))
    e = L.Expansion(q)
    n, ux, uy, T = _random_state((6, 5))
    U = P.four_velocity(ux, uy)
    f = e.feq(n, U, T)
    N, Tab = S.moments(f, q.p)
    TE = _eos_energy_tensor(n, U, T, q.m)
    assert np.abs(N - n * U).max() < 1e-12 * np.abs(n * U).max()
    assert np.abs(Tab - TE).max() < 1e-12 * np.abs(TE).max()


def test_order3_equilibrium_recovers_third_moments():
    q = L.massless_quadrature(3)
    e = L.Expansion(q)
    n, ux, uy, T = (np.array(1.3), np.array(0.2), np.array(-0.35), np.array(1.1))
    U = P.four_velocity(ux, uy)
    f = e.feq(n, U, T)
    for al in [(0, 0, 0), (0, 1, 2), (1, 1, 1), (2, 2, 1), (0, 0, 2)]:
        disc = np.sum(f * np.prod(q.p[:, list(al)], axis=1))
        ref = _mj_numeric(al, float(n), U, float(T), 0.0)
        assert abs(disc - ref) < 1e-10 * abs(ref) + 1e-12


def test_order2_expansion_misses_third_moments():
    """Sanity of the previous pin: at N = 2 third moments are not recovered."""
    q = L.massless_quadrature(2)
    n, U, T = 1.0, P.four_velocity(np.array(0.3), np.array(0.0)), 1.2
    f = L.Expansion(q).feq(n, U, np.array(T))
    disc = np.sum(f * q.p[:, 1] ** 3)
    assert abs(disc - _mj_numeric((1, 1, 1), n, U, T, 0.0)) > 1e-3


def test_rest_frame_equilibrium_is_n_times_weight():
    """App. G at U = (1, 0, 0), T~ = 1, m = 0: only a^(0) = n survives."""
    for order in (2, 3):
        q = L.massless_quadrature(order)
        f = L.Expansion(q).feq(np.array(1.7), P.four_velocity(np.array(0.0), np.array(0.0)), np.array(1.0))
        assert np.abs(f - 1.7 * q.w).max() < 1e-14


def test_gram_schmidt_projection_route_matches_appG_route():
    """Two routes printed in the paper (App. G closed forms vs App. B moments
    contracted with the Gram-Schmidt basis) give the same f^eq."""
    for m, q in [(0.0, L.massless_quadrature(2)),
                 (5.0, L.massive_quadrature([(0, 0), (1, 0), (1, 1), (2, 1), (2, 2), (3, 1)], 5.0, 0.2726)[0])]:
        n, ux, uy, T = _random_state((4, 3))
        U = P.four_velocity(ux, uy)
        a = L.Expansion(q, source="appFG").feq(n, U, T)
        b = L.Expansion(q, order=2, source="gram_schmidt").feq(n, U, T)
        assert np.abs(a - b).max() < 1e-13 * np.abs(a).max()


# ---------------------------------------------------------- EOS and Landau


def test_G2_closed_form_from_half_integer_bessel():
    z = np.array([0.01, 0.5, 1.0, 5.0, 10.0, 40.0])
    assert np.allclose(P.G_d(z, 2), (z * z + 3 * z + 3) / (z + 1), rtol=1e-13)
    assert P.G_d(np.array([0.0]), 2)[0] == 3.0
    # d = 3: eps = P (3 + zeta K1/K2) (Eq. relativistic-eos-3D)
    assert np.allclose(P.G_d(z, 3) - 1, 3 + z * special.kv(1, z) / special.kv(2, z), rtol=1e-12)


@pytest.mark.parametrize("m", [0.0, 1.0, 5.0, 10.0])
def test_temperature_inversion(m):
    T = np.linspace(0.2, 3.0, 15)
    e = P.energy_per_particle(T, m)
    assert np.abs(P.temperature_from_energy(e, m) - T).max() < 1e-13
    # the d = 2 closed form of the inversion
    Tc = ((e - 2 * m) + np.sqrt(e * e + 4 * e * m - 4 * m * m)) / 4
    assert np.abs(Tc - T).max() < 1e-12


def test_ultrarelativistic_and_classical_eos_limits():
    assert abs(P.energy_per_particle(np.array(1.0), 0.0) - 2.0) < 1e-15   # eps = d P
    T = 1.0
    m = 2000.0
    ek = P.energy_per_particle(np.array(T), m) - m                   # eps_c = (d/2) P
    assert abs(ek - 1.0) < 2e-3


def _boost(beta_x, beta_y):
    b2 = beta_x ** 2 + beta_y ** 2
    g = 1 / math.sqrt(1 - b2)
    bx, by = beta_x, beta_y
    L_ = np.eye(3)
    L_[0, 0] = g
    L_[0, 1] = L_[1, 0] = g * bx
    L_[0, 2] = L_[2, 0] = g * by
    if b2 > 0:
        L_[1, 1] = 1 + (g - 1) * bx * bx / b2
        L_[2, 2] = 1 + (g - 1) * by * by / b2
        L_[1, 2] = L_[2, 1] = (g - 1) * bx * by / b2
    return L_


def test_landau_flags_non_finite_cells_instead_of_raising():
    """A cell whose moments are not finite has no Landau frame: it is flagged
    (reading of Sec. 4 for non-physical states), and the other cells of the
    same call are solved as usual."""
    N = np.zeros((3, 2))
    Tm = np.zeros((3, 3, 2))
    N[0] = 1.0
    Tm[0, 0], Tm[1, 1], Tm[2, 2] = 2.0, 1.0, 1.0            # rest frame, eps = 2, P = 1
    Tm[0, 0, 1] = np.nan
    eps, U, n, ok = P.landau(N, Tm)
    assert ok.tolist() == [True, False]
    assert abs(eps[0] - 2.0) < 1e-14 and abs(n[0] - 1.0) < 1e-14 and abs(U[0, 0] - 1.0) < 1e-14


@pytest.mark.parametrize("beta", [(0.0, 0.0), (0.3, 0.1), (-0.6, 0.5), (0.9, 0.0), (0.0, -0.9)])
def test_landau_solve_is_lorentz_consistent(beta):
    """Boost a rest-frame tensor (ideal part + a traceless shear part) and
    recover eps, n and U = Lambda e0 (Sec. 4, Landau frame)."""
    eps, Pp, n, pi = 2.4, 1.1, 0.9, 0.07
    Trest = np.diag([eps, Pp + pi, Pp - pi])
    Trest[1, 2] = Trest[2, 1] = 0.03
    Lb = _boost(*beta)
    Tlab = Lb @ Trest @ Lb.T
    Nlab = Lb @ np.array([n, 0.0, 0.0])
    e_, U, n_, ok = P.landau(Nlab.reshape(3, 1), Tlab.reshape(3, 3, 1))
    assert ok[0]
    assert abs(e_[0] - eps) < 1e-13 * eps / (1 - beta[0] ** 2 - beta[1] ** 2)
    assert abs(n_[0] - n) < 1e-13 * 10
    assert np.abs(U[:, 0] - Lb[:, 0]).max() < 1e-12
    # eigen-residual T^{ab} U_b = eps U^a
    assert np.abs(Tlab @ (P.ETA @ U[:, 0]) - e_[0] * U[:, 0]).max() < 1e-12 * np.abs(Tlab).max()


# ---------------------------------------------------------- collision, streaming


@pytest.mark.parametrize("case", ["massless2", "massless3", "mass5"])
def test_collision_conserves_N0_and_T0a(case):
    """Sec. 6.2 step 8 with n = U.N and the Landau condition: Delta N^0 = 0,
    Delta T^{0a} = 0 per cell; spatial N^i is not a collision invariant."""
    if case == "mass5":
        q, _ = L.massive_quadrature([(0, 0), (1, 0), (1, 1), (2, 1), (2, 2), (3, 1)], 5.0, 0.2726)
    else:
        q = L.massless_quadrature(int(case[-1]))
    e = L.Expansion(q)
    n, ux, uy, T = _random_state((5, 4), umax=0.5)
    f = e.feq(n, P.four_velocity(ux, uy), T) * (1 + 0.05 * RNG.standard_normal((q.Q, 5, 4)))
    tau = RNG.uniform(0.6, 2.0, (5, 4))
    fs, fl = S.collide(f, q, e, tau)
    N1, T1 = S.moments(fs, q.p)
    N0, T0 = S.moments(f, q.p)
    scale = np.abs(T0).max()
    # the printed weights carry ~16 decimals; the order-3 table reaches p0 = 9.4
    assert np.abs(N1[0] - N0[0]).max() < 1e-12 * scale
    assert np.abs(T1[0] - T0[0]).max() < 1e-12 * scale
    assert np.abs(N1[1] - N0[1]).max() > 1e-6


def test_collision_of_equilibrium_is_identity():
    q = L.massless_quadrature(2)
    e = L.Expansion(q)
    n, ux, uy, T = _random_state((3, 3))
    f = e.feq(n, P.four_velocity(ux, uy), T)
    fs, fl = S.collide(f, q, e, 0.7)
    assert np.abs(fs - f).max() < 1e-13 * np.abs(f).max()


def test_onlattice_streaming_is_a_permutation():
    q = L.massless_quadrature(2)
    fs = RNG.standard_normal((q.Q, 7, 11))
    f = S.stream_onlattice(fs, q.n)
    for i in range(q.Q):
        assert np.array_equal(np.sort(f[i].ravel()), np.sort(fs[i].ravel()))
    # a population moves by exactly n_i
    i = 3
    src = np.zeros((q.Q, 7, 11))
    src[i, 2, 4] = 1.0
    out = S.stream_onlattice(src, q.n)
    yy, xx = np.argwhere(out[i] == 1.0)[0]
    assert (xx - 4) % 11 == q.n[i, 0] % 11 and (yy - 2) % 7 == q.n[i, 1] % 7


def test_bilinear_at_integer_displacement_equals_onlattice():
    """lambda = 5 (massless, ||n_i|| = 5): displacement lambda v_i = n_i exactly."""
    q = L.massless_quadrature(2)
    fs = RNG.standard_normal((q.Q, 9, 13))
    a = S.stream_onlattice(fs, q.n)
    b = S.stream_bilinear(fs, 5.0 * q.velocity())
    assert np.abs(a - b).max() < 1e-15


def test_bilinear_streaming_conserves_global_sums():
    q = L.massless_quadrature(2)
    fs = RNG.uniform(0, 1, (q.Q, 12, 10))
    b = S.stream_bilinear(fs, 1.0 * q.velocity())
    assert np.abs(b.sum(axis=(1, 2)) - fs.sum(axis=(1, 2))).max() < 1e-12
    # a constant field is a fixed point (weights sum to one)
    c = np.ones((q.Q, 5, 6))
    assert np.abs(S.stream_bilinear(c, 1.0 * q.velocity()) - 1.0).max() < 1e-15


# Displacements lambda * v_i of the massless order-2 stencil (|v_i| = 1) at
# lambda = 0.5, 1 and 2.5, and two massive-like short vectors: fractional
# parts 0.1 ... 0.9 in both directions, none of them 1/2 in both axes (where
# phi and 1 - phi coincide).
def _fractional_displacements():
    q = L.massless_quadrature(2)
    out = [lam * v for lam in (0.5, 1.0, 2.5) for v in q.velocity()]
    out += [np.array([0.37, -1.71]), np.array([-2.26, 0.13])]
    return out


@pytest.mark.parametrize("k", range(0, 86, 5))
def test_bilinear_streaming_reproduces_linear_fields_exactly(k):
    """Bilinear interpolation is exact on fields linear in x and y: a field
    F = a + b x + c y streamed by a displacement d must equal F(x - d) at every
    cell whose two tap columns and rows lie inside the grid (no periodic
    wrap).  A swap of phi and 1 - phi, or a wrong rounding of the departure
    point, moves the result by a non-zero multiple of b or c."""
    d = _fractional_displacements()[k % len(_fractional_displacements())]
    ny, nx = 17, 23
    a, b, c = 0.7, 0.013, -0.021
    yy, xx = np.mgrid[0:ny, 0:nx].astype(np.float64)
    F = a + b * xx + c * yy
    out = S.stream_bilinear(F[None], d[None])[0]
    src = -d
    o = np.floor(src)
    lo_x, hi_x = max(0, -int(o[0])), min(nx, nx - int(o[0]) - 1)
    lo_y, hi_y = max(0, -int(o[1])), min(ny, ny - int(o[1]) - 1)
    assert hi_x - lo_x >= 5 and hi_y - lo_y >= 5
    want = a + b * (xx - d[0]) + c * (yy - d[1])
    sl = (slice(lo_y, hi_y), slice(lo_x, hi_x))
    assert np.abs(out[sl] - want[sl]).max() < 1e-14


@pytest.mark.parametrize("k", range(0, 86, 5))
def test_bilinear_streaming_moves_an_impulse_by_exactly_its_displacement(k):
    """A unit impulse streamed by d keeps its mass, its centre moves by exactly
    d, and its variance along each axis is phi (1 - phi) -- the numerical
    diffusion of one interpolation, phi the fractional part of the departure
    point x - d.  (Grid large enough that no tap wraps.)"""
    d = _fractional_displacements()[k % len(_fractional_displacements())]
    ny, nx = 15, 15
    y0, x0 = 7, 7
    f = np.zeros((1, ny, nx))
    f[0, y0, x0] = 1.0
    out = S.stream_bilinear(f, d[None])[0]
    yy, xx = np.mgrid[0:ny, 0:nx].astype(np.float64)
    mass = out.sum()
    assert abs(mass - 1.0) < 1e-15
    cx, cy = (out * xx).sum(), (out * yy).sum()
    assert abs(cx - (x0 + d[0])) < 1e-13 and abs(cy - (y0 + d[1])) < 1e-13
    phi = -d - np.floor(-d)
    vx, vy = (out * (xx - cx) ** 2).sum(), (out * (yy - cy) ** 2).sum()
    assert abs(vx - phi[0] * (1 - phi[0])) < 1e-13 and abs(vy - phi[1] * (1 - phi[1])) < 1e-13


def test_bilinear_taps_are_non_negative_and_bracket_the_departure_point():
    """All four weights lie in [0, 1] and sum to one, and the taps are the
    corners of the unit cell that contains x - d."""
    for d in _fractional_displacements():
        taps = S.bilinear_taps(d)
        w = np.array([t[2] for t in taps])
        assert (w >= 0).all() and (w <= 1).all() and abs(w.sum() - 1) < 1e-15
        xs = sorted({t[0] for t in taps})
        ys = sorted({t[1] for t in taps})
        # (a departure point within 1e-12 of a whole cell is that cell)
        assert xs[0] - 1e-12 <= -d[0] <= xs[-1] + 1e-12 and xs[-1] - xs[0] == 1
        assert ys[0] - 1e-12 <= -d[1] <= ys[-1] + 1e-12 and ys[-1] - ys[0] == 1


def test_tau_from_eta_over_s_reproduces_eta_over_s():
    """Step 7 with eta/s fixed.  With the independent App. C coefficient
    eta = c P tau (c = ce_shear_viscosity_coeff(0) = 3/4 for a massless d = 2
    gas), P = n T and the entropy density s = (d + 1) n, the ratio
    eta / s = c T tau / (d + 1) in lattice units, times 1/kappa to convert
    hbar/k_B units, must give back the prescribed eta/s for every (n, T)."""
    rng = np.random.default_rng(7)
    c = P.ce_shear_viscosity_coeff(0.0)
    for _ in range(20):
        n, T = rng.uniform(0.2, 3.0, 2)
        target, kappa = rng.uniform(0.01, 1.0), rng.uniform(1.0, 30.0)
        tau = S.tau_from_eta_over_s(T, target, kappa)
        eta = c * (n * T) * tau
        s = 3.0 * n
        assert abs(eta / s / kappa - target) < 1e-14 * target


def test_freeflow_streaming_clamps_sources():
    q = L.massless_quadrature(2)
    fs = np.zeros((q.Q, 1, 20))
    fs[:, 0, 0] = 1.0
    f = S.stream_onlattice(fs, q.n, "freeflow_x")
    for i in range(q.Q):
        sx = q.n[i, 0]
        # cells whose source x - sx falls at or left of 0 read the boundary cell
        expect = (np.arange(20) - sx <= 0).astype(float)
        assert np.array_equal(f[i, 0], expect)


def test_periodic_run_conserves_global_N0_and_T0a():
    q = L.massless_quadrature(2)
    e = L.Expansion(q)
    sim = S.Simulation(q, e, 24, 20, tau=0.8)
    n, ux, uy, T = _random_state((20, 24), umax=0.3)
    sim.init(n, ux, uy, T)
    N0, T0 = S.moments(sim.fs, q.p)
    sim.step(5)
    N1, T1 = S.moments(sim.fs, q.p)
    assert abs(N1[0].sum() - N0[0].sum()) < 1e-11 * N0[0].sum()
    assert np.abs(T1[0].sum(axis=(-1, -2)) - T0[0].sum(axis=(-1, -2))).max() < 1e-11 * T0[0, 0].sum()


# ---------------------------------------------------------- transport coefficients


def test_ce_shear_viscosity_limits():
    """App. C: d = 2 CE eta = P tau (2 G - zeta^2 + e^zeta zeta^4 Gamma(0,zeta)/(zeta+1))/8;
    UR limit (d+1)/(d+2) = 3/4 (Eq. ce-ur-limit); classical limit -> 1."""
    assert abs(P.ce_shear_viscosity_coeff(np.array(0.0)) - 0.75) < 1e-15
    assert abs(P.ce_shear_viscosity_coeff(np.array(1e-6)) - 0.75) < 1e-5
    assert abs(P.ce_shear_viscosity_coeff(np.array(2000.0)) - 1.0) < 2e-3
    z = np.linspace(0.1, 20, 30)
    assert np.all(np.diff(P.ce_shear_viscosity_coeff(z)) > 0)


@pytest.mark.parametrize("zeta", [0.0, 0.5, 1.0, 2.0, 5.0, 10.0, 50.0])
def test_ce_shear_viscosity_matches_the_chapman_enskog_integral(zeta):
    """App. C closed form against the first-order CE integral it comes from,
    evaluated by quadrature: in a shear flow u_x(y) the Anderson-Witting
    correction is df = -(tau / p0) f_eq p^x p^y du_x/dy / T (rest frame), so
    eta = (tau / T) int d^2p (p^x p^y)^2 f_eq / p0^2 and, with n = int d^2p f_eq
    and P = n T, eta / (P tau) = (pi/4) int p^5 e^{-p0/T}/p0^2 dp /
    (2 pi T^2 int p e^{-p0/T} dp).  Independent of the Gamma(0, zeta) form."""
    from scipy import integrate
    T = 1.0
    m = zeta * T

    def w(p, k):
        return p ** k * np.exp(-(np.sqrt(m * m + p * p) - m) / T)

    num = (np.pi / 4) * integrate.quad(lambda p: w(p, 5) / (m * m + p * p), 0, np.inf, epsabs=0,
                                       epsrel=1e-13, limit=500)[0]
    den = T * T * 2 * np.pi * integrate.quad(lambda p: w(p, 1), 0, np.inf, epsabs=0, epsrel=1e-13, limit=500)[0]
    assert abs(float(P.ce_shear_viscosity_coeff(np.array(zeta))) - num / den) < 1e-8


def _mj_radial(f, m, T=1.0):
    """int_0^inf f(p, p0) e^{-(p0 - m)/T} dp by quadrature (p0 = sqrt(m^2 + p^2))."""
    from scipy import integrate
    return integrate.quad(lambda p: f(p, np.sqrt(m * m + p * p)) * np.exp(-(np.sqrt(m * m + p * p) - m) / T),
                          0, np.inf, epsabs=0, epsrel=1e-12, limit=400)[0]


@pytest.mark.parametrize("zeta", [0.0, 0.5, 1.0, 2.0, 5.0, 10.0])
def test_ce_thermal_conductivity_matches_the_chapman_enskog_integral(zeta):
    """App. C closed form against the first-order Anderson-Witting correction
    integrated by quadrature.  A fluid at rest with a temperature gradient at
    uniform pressure (d_x n / n = -d_x T / T) has df = -(tau / p0) p^x d_x f_eq,
    d_x ln f_eq = d_x T ((p0 - <p0>) / T^2 - 1 / T); the diffusion current
    V^x = int d^2p / p0 p^x df and the heat flux q^x = -h_e V^x = -lambda d_x T
    (h_e = (eps + P) / n) give lambda = h_e V^x / d_x T."""
    T, m, n, tau = 1.0, zeta, 1.0, 1.0
    Z = 2 * np.pi * _mj_radial(lambda p, p0: p, m, T)
    p0m = 2 * np.pi * _mj_radial(lambda p, p0: p * p0, m, T) / Z
    # int d^2p (p_x^2 / p0^2) f_eq (...): angular average of p_x^2 is p^2 / 2
    I = np.pi * _mj_radial(lambda p, p0: p ** 3 / p0 ** 2 * ((p0 - p0m) / T ** 2 - 1 / T), m, T) * n / Z
    he = (n * p0m + n * T) / n
    lam = -he * tau * I
    assert abs(float(P.ce_thermal_conductivity_coeff(np.array(zeta))) - lam / (n * tau)) < 1e-10


@pytest.mark.parametrize("zeta", [0.0, 0.5, 1.0, 2.0, 5.0, 10.0])
def test_ce_bulk_viscosity_matches_the_chapman_enskog_integral(zeta):
    """App. C closed form against the first-order Anderson-Witting correction
    for a uniform expansion theta = d_x U^x of a fluid at rest with uniform
    n, T: the Euler equations give d_t n = -n theta and
    d_t T = -(T / e'(T)) theta (e = eps / n), so
    p^mu d_mu ln f_eq = p0 (-theta + (p0 - <p0>) d_t T / T^2) + (p^x)^2 theta / T,
    df = -(tau / p0) f_eq p^mu d_mu ln f_eq,
    varpi = -(1/d) (dT^00 - dT^xx - dT^yy), mu = -varpi / theta;
    the Landau matching dT^00 = 0 holds as well."""
    T, m, n, tau, th = 1.0, zeta, 1.0, 1.0, 1.0
    Z = 2 * np.pi * _mj_radial(lambda p, p0: p, m, T)
    p0m = 2 * np.pi * _mj_radial(lambda p, p0: p * p0, m, T) / Z
    p02 = 2 * np.pi * _mj_radial(lambda p, p0: p * p0 * p0, m, T) / Z
    dTdt = -(T / ((p02 - p0m ** 2) / T ** 2)) * th
    A = lambda p, p0: p0 * (-th + (p0 - p0m) / T ** 2 * dTdt) + p * p / 2 * th / T
    dT00 = -tau * 2 * np.pi * _mj_radial(lambda p, p0: p * A(p, p0), m, T) * n / Z
    dTii = -tau * 2 * np.pi * _mj_radial(lambda p, p0: p ** 3 / p0 ** 2 * A(p, p0), m, T) * n / Z
    varpi = -(dT00 - dTii) / 2
    assert abs(dT00) < 1e-12
    mu = -varpi / th / (n * T * tau)
    assert abs(float(P.ce_bulk_viscosity_coeff(np.array(zeta))) - mu) < 1e-10


def _mj_on_fine_rule(m, ns=120, nth=64):
    """The exact Maxwell-Juttner populations on a product rule for
    int d^2p / p0 = int dp0 dtheta: Gauss-Laguerre in s = p0 - m (textbook
    nodes) times the trapezoid rule in theta; f = n e^{-(p.U - m)/T} /
    (2 pi T (m + T)) normalises N^0 = n at rest (d = 2)."""
    s, ws = special.roots_laguerre(ns)
    th = 2 * np.pi * np.arange(nth) / nth
    S, TH = np.meshgrid(s, th, indexing="ij")
    pm = np.sqrt(S * (2 * m + S))
    p = np.stack([(m + S).ravel(), (pm * np.cos(TH)).ravel(), (pm * np.sin(TH)).ravel()], axis=1)
    W = (ws[:, None] * np.exp(s)[:, None] * np.full((1, nth), 2 * np.pi / nth)).ravel()

    def feq(n, ux, uy, T):
        g = 1 / np.sqrt(1 - ux * ux - uy * uy)
        pu = g * (p[:, 0] - p[:, 1] * ux - p[:, 2] * uy)
        return W * n / (2 * np.pi * T * (m + T)) * np.exp(-(pu - m) / T)
    return p, feq


@pytest.mark.parametrize("zeta", [0.0, 0.5, 1.0, 2.0, 5.0, 10.0, 20.0])
def test_first_order_coefficients_of_the_exact_distribution_are_app_c(zeta):
    """``transport.first_order`` fed the exact MJ distribution on a fine rule
    (instead of a lattice) gives the App. C closed forms of eta, lambda and mu,
    and mu = 0 for massless particles."""
    from oracle import transport as TR
    p, feq = _mj_on_fine_rule(zeta)
    assert abs(np.sum(feq(1.0, 0.0, 0.0, 1.0) * p[:, 0]) - 1.0) < 1e-13
    r = TR.first_order(p, feq, zeta)
    assert abs(r["eta"] - float(P.ce_shear_viscosity_coeff(np.array(zeta)))) < 1e-10
    assert abs(r["lam"] - float(P.ce_thermal_conductivity_coeff(np.array(zeta)))) < 1e-10
    assert abs(r["mu"] - float(P.ce_bulk_viscosity_coeff(np.array(zeta)))) < 2e-11
    if zeta == 0.0:
        assert abs(r["mu"]) < 1e-15


def test_first_order_shear_coefficient_explains_the_lattice_viscosities():
    """On the massless App. H tables the same routine gives eta / (P tau) =
    1.307 (order 2) and 1.0021 (order 3) of the UR value 3/4 (Eq.
    ce-ur-limit), the offsets the whole-scheme shear-wave pins measure as
    0.98 (tau - 1/2) and 0.7516 (tau - 1/2)."""
    from oracle import transport as TR
    got = {}
    for order in (2, 3):
        q = L.massless_quadrature(order)
        got[order] = TR.first_order(q.p, TR.lattice_feq(L.Expansion(q)), 0.0)["eta"]
    assert abs(got[2] - 0.980) < 2e-3
    assert abs(got[3] - 0.7516) < 2e-4


def test_order2_shear_viscosity_is_anisotropic_and_averages_to_ur():
    """The first-order shear coefficient of the massless tables along the
    lattice axes and along the diagonals (stencil rotated by 45 degrees): at
    N = 2 they are 0.980 and 0.520, whose mean is the UR 3/4 of Eq.
    ce-ur-limit (a degree-4 average over the two directions); at N = 3 both
    are within 0.3 % of 3/4.  The Taylor-Green vortex, whose wavevectors lie
    along the diagonals, therefore decays at 0.52 (tau - 1/2) P at N = 2."""
    from oracle import transport as TR

    def eta(order, ang):
        q = L.massless_quadrature(order)
        c, s_ = math.cos(ang), math.sin(ang)
        p = q.p.copy()
        p[:, 1], p[:, 2] = c * q.p[:, 1] - s_ * q.p[:, 2], s_ * q.p[:, 1] + c * q.p[:, 2]
        qr = L.Quadrature(q.n, p, q.w, q.m, q.order, q.v0)
        return TR.first_order(qr.p, TR.lattice_feq(L.Expansion(qr)), 0.0)["eta"]

    a2, d2 = eta(2, 0.0), eta(2, math.pi / 4)
    assert abs(a2 - 0.9802) < 1e-4 and abs(d2 - 0.5198) < 1e-4
    assert abs(0.5 * (a2 + d2) - 0.75) < 1e-10          # the derivatives are 4th-order differences
    a3, d3_ = eta(3, 0.0), eta(3, math.pi / 4)
    assert abs(a3 / 0.75 - 1) < 3e-3 and abs(d3_ / 0.75 - 1) < 3e-3


def _shear_wave_eta(order, Lx, tau, amp=0.01):
    q = L.massless_quadrature(order)
    e = L.Expansion(q)
    sim = S.Simulation(q, e, Lx, 1, tau=tau)
    x = np.arange(Lx)[None, :]
    k = 2 * np.pi / Lx
    sim.init(np.ones((1, Lx)), 0.0 * x, amp * np.sin(k * x), np.ones((1, Lx)))
    kphys = 10 * np.pi / Lx                  # delta x = 1/5: ||n_i|| = 5 cells per unit time
    rate_guess = 0.75 * (tau - 0.5) / 3 * kphys ** 2
    nsteps = int(1.5 / rate_guess)
    ts, amps = [], []
    for t in range(nsteps):
        sim.step(1)
        if t > 0.15 * nsteps and t % 5 == 0:
            ts.append(sim.t)
            amps.append(2 / Lx * np.sum(sim.fields.uy * np.sin(k * x)))
    rate = -np.polyfit(ts, np.log(amps), 1)[0]
    return 3.0 * rate / kphys ** 2             # eta / P, from rate = eta k^2 / (eps + P), eps + P = 3 P


@pytest.mark.slow
@pytest.mark.parametrize("tau", [0.8, 1.4])
def test_order3_shear_wave_viscosity_matches_chapman_enskog(tau):
    """Whole-scheme pin (Sec. 7.1 procedure with a single shear wave): the
    order-3 massless scheme decays at eta = (3/4) P (tau - dt/2): the CE
    value of App. C with the second-order lattice shift of tau by half a step."""
    eta = _shear_wave_eta(3, 200, tau)
    assert abs(eta / (0.75 * (tau - 0.5)) - 1.0) < 0.01


# ------------------------------------------------------- App. D Riemann problem


def _ur_conserved(n, P, beta, d=2):
    """(N^0, T^00, T^0x) and their x-fluxes (N^x, T^0x, T^xx) of an ideal
    ultra-relativistic fluid, eps = d P (definitions of Sec. 3)."""
    g2 = 1.0 / (1.0 - beta ** 2)
    h = (d + 1) * P                      # eps + P
    N0, Nx = n * np.sqrt(g2), n * np.sqrt(g2) * beta
    T00, T0x, Txx = h * g2 - P, h * g2 * beta, h * g2 * beta ** 2 + P
    return np.array([N0, T00, T0x]), np.array([Nx, T0x, Txx])


@pytest.mark.parametrize("d", [2, 3])
def test_riemann_ur_satisfies_jump_conditions_from_the_definitions(d):
    """Across the shock (speed beta_s) the lab-frame fluxes of N and T jump as
    beta_s times the jump of the densities; across the contact P and beta are
    continuous; the fan ends on the plateau."""
    s = P.riemann_ur(1.0, 1.0, 0.5, 0.4, d=d)
    q2, f2 = _ur_conserved(s["n_II"], s["P_C"], s["beta_C"], d)
    qR, fR = _ur_conserved(s["nR"], s["PR"], 0.0, d)
    assert np.abs(s["beta_s"] * (q2 - qR) - (f2 - fR)).max() < 1e-14
    # tail of the fan: the profile just inside reaches (P_C, beta_C, n_I)
    w = np.array([s["w_T"] - 1e-12])
    n, Pw, b = P.riemann_ur_profile(s, w)
    assert abs(Pw[0] - s["P_C"]) < 1e-10 and abs(b[0] - s["beta_C"]) < 1e-10
    assert abs(n[0] - s["n_I"]) < 1e-10
    # head of the fan: the left state
    n, Pw, b = P.riemann_ur_profile(s, np.array([s["w_H"] + 1e-12]))
    assert abs(Pw[0] - 1.0) < 1e-10 and abs(b[0]) < 1e-10 and abs(n[0] - 1.0) < 1e-10


def test_riemann_ur_fan_is_a_self_similar_solution_of_the_conservation_laws():
    """On the fan, d/dt Q + d/dx F = 0 with Q(w), F(w), w = x/t, reads
    -w Q'(w) + F'(w) = 0 for N^0, T^00 and T^0x (central differences)."""
    s = P.riemann_ur(1.0, 1.0, 0.5, 0.4)
    h = 1e-5
    for w in np.linspace(s["w_H"] + 0.01, s["w_T"] - 0.01, 7):
        qa, fa = _ur_conserved(*P.riemann_ur_profile(s, np.array([w - h])))
        qb, fb = _ur_conserved(*P.riemann_ur_profile(s, np.array([w + h])))
        dq, df = (qb - qa) / (2 * h), (fb - fa) / (2 * h)
        assert np.abs(-w * dq + df).max() < 1e-8 * np.abs(df).max()


def test_riemann_ur_weak_shock_limit():
    """P_R -> P_L: no flow, and the shock and the rarefaction head move at
    the sound speed c/sqrt(d)."""
    s = P.riemann_ur(1.0, 1.0, 1.0 - 1e-9, 1.0 - 1e-9)
    assert abs(s["beta_C"]) < 1e-8
    assert abs(s["beta_s"] - 1 / np.sqrt(2)) < 1e-8
    assert abs(s["w_T"] - s["w_H"]) < 1e-8


def test_oracle_sod_matches_app_d_solution():
    """Config-1 shock tube (1024 x 1, eta/s = 0.1, free-flow ends) after 100
    steps, before any wave reaches an end, against the inviscid App. D
    solution: plateau pressure and velocity within 0.5 %, the densities on
    either side of the contact within 1 % / 2.5 % (the contact is diffused by
    the viscosity), the shock and the middle of the fan within 2 % in w."""
    q = L.massless_quadrature(2)
    nx, t = 1024, 100
    sim = S.Simulation(q, L.Expansion(q), nx, 1, tau=(0.1, 15.79), boundary="freeflow_x")
    left = np.arange(nx) < nx // 2
    n0 = np.where(left, 1.0, 0.5)[None, :]
    T0 = np.where(left, 1.0, 0.8)[None, :]
    z = np.zeros((1, nx))
    sim.init(n0, z, z.copy(), T0)
    sim.step(t)
    fl = sim.fields
    Pn, b, n = (fl.n * fl.T)[0], fl.ux[0], fl.n[0]
    s = P.riemann_ur(1.0, 1.0, 0.5, 0.4)
    w = (np.arange(nx) - (nx // 2 - 0.5)) / (5.0 * t)       # c = 5 cells per step
    plateau = (w > -0.1) & (w < 0.5)
    assert abs(Pn[plateau].mean() / s["P_C"] - 1) < 5e-3
    assert abs(b[plateau].mean() / s["beta_C"] - 1) < 5e-3
    assert abs(n[np.argmin(abs(w + 0.25))] / s["n_I"] - 1) < 1e-2
    assert abs(n[np.argmin(abs(w - 0.45))] / s["n_II"] - 1) < 2.5e-2

    def crossing(level, lo, hi):
        i = np.where((w > lo) & (w < hi) & (Pn < level))[0][0]
        return w[i - 1] + (w[i] - w[i - 1]) * (Pn[i - 1] - level) / (Pn[i - 1] - Pn[i])

    ws = crossing(0.5 * (s["P_C"] + 0.4), 0.5, 1.0)
    assert abs(ws - s["w_S"]) < 0.02
    Pmid = 0.5 * (1.0 + s["P_C"])
    _, Pa, _ = P.riemann_ur_profile(s, w)
    i = np.where((w > s["w_H"]) & (Pa < Pmid))[0][0]
    assert abs(crossing(Pmid, -1.0, 0.0) - w[i]) < 0.02


# ------------------------------------------------------------ forcing, walls


@pytest.mark.parametrize("m", [1.0, 5.0])
def test_forcing_term_moments_follow_from_the_equilibrium_stress(m):
    """Scheme B with a gravity-like force (Sec. 4.4).  Its moments follow from
    T_E^ab = (eps + P) U^a U^b - P eta^ab (exact for the quadrature at order
    2): no particle source, momentum source n m U^0 g (along g), energy
    source n m g.U, for any (n, U, T)."""
    import paper_1909_04502_gb300.inputs as inputs
    q = _massive_q(m)
    e = L.Expansion(q)
    n, ux, uy, T = inputs.random_smooth(8, 4, seed=3, umax=0.4, dn=0.3, dT=0.3)
    U = P.four_velocity(ux, uy)
    feq = e.feq(n, U, T)
    fl = S.macroscopic(feq, q)
    g = (3e-3, -2e-3)
    F = S.forcing_term(feq, fl, q, g)
    p0, px, py = (q.p[:, k, None, None] for k in range(3))
    assert np.abs(np.sum(p0 * F, axis=0)).max() < 1e-13
    assert np.allclose(np.sum(p0 * px * F, axis=0), n * m * U[0] * g[0], rtol=1e-10, atol=0)
    assert np.allclose(np.sum(p0 * py * F, axis=0), n * m * U[0] * g[1], rtol=1e-10, atol=0)
    assert np.allclose(np.sum(p0 * p0 * F, axis=0), n * m * (g[0] * U[1] + g[1] * U[2]), rtol=1e-9,
                       atol=1e-15)


def _massive_q(m):
    """Order-2 quadrature at the middle of the v0 window where the oracle's
    own solve gives non-negative weights: the Sec. 5.3 worked-example stencil
    (m~ = 5) or App. H column C (m~ = 1)."""
    groups = ([(0, 0), (1, 0), (1, 1), (2, 1), (2, 2), (3, 1)] if m >= 5 else
              [(0, 0), (3, 3), (4, 2), (4, 3), (5, 0), (5, 1)])
    ok = L.search_v0(groups, m, order=2, npts=400)
    assert ok
    q, res = L.massive_quadrature(groups, m, 0.5 * (ok[0] + ok[-1]), 2)
    assert res < 1e-9
    return q


def test_equilibrium_walls_leave_the_wall_columns_at_rest():
    """After a collision with equilibrium walls the first and last columns
    carry no flow (N^x = N^y = 0, T^0x = T^0y = 0) and keep the n and T of
    the streamed populations; interior columns are untouched."""
    import paper_1909_04502_gb300.inputs as inputs
    q = _massive_q(5.0)
    e = L.Expansion(q)
    n, ux, uy, T = inputs.random_smooth(8, 4, seed=9, umax=0.3)
    f = e.feq(n, P.four_velocity(ux, uy), T)
    fs0, _ = S.collide(f, q, e, 0.9)
    fs, fl = S.collide(f, q, e, 0.9, eqwall=True)
    for col in (0, 7):
        after = S.macroscopic(fs[:, :, col:col + 1], q)
        assert np.abs(after.N[1:]).max() < 1e-13 and np.abs(after.Tab[0, 1:]).max() < 1e-13
        assert np.allclose(after.n[:, 0], fl.n[:, col], rtol=1e-12)
        assert np.allclose(after.T[:, 0], fl.T[:, col], rtol=1e-12)
    assert np.array_equal(fs[:, :, 1:7], fs0[:, :, 1:7])


@pytest.mark.parametrize("m,groups", [(15.0, [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2), (3, 0), (3, 2),
                                              (3, 3), (4, 0)]),
                                      (20.0, [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (3, 1), (3, 2), (3, 3),
                                              (4, 0), (4, 2)])])
def test_order3_massive_equilibrium_matches_arbitrary_precision_evaluation(m, groups):
    """The order-3 massive equilibrium (Sec. 5.2, Gram-Schmidt basis, App. B
    moments) against the same definition evaluated with mpmath at 40 digits
    (Bessel functions K_{n+1/2} from mpmath, not the closed form the oracle
    uses): the extended-precision evaluation keeps 1e-15 of max |f| where
    plain double loses up to 1e-12 at these masses.  Stencils: the paper's
    45-vector performance stencil (Sec. 6.3) at m~ = 15, App. H column D
    at m~ = 20; v0 from the oracle's own Sec. 5.3 search."""
    mp = pytest.importorskip("mpmath")
    from decimal import localcontext
    mp.mp.dps = 40
    win = L.search_v0(groups, m, order=3, npts=800)
    assert win, "no non-negative v0"
    v0 = 0.5 * (min(win) + max(win))
    q, res = L.massive_quadrature(groups, m, v0, 3)
    e = L.Expansion(q)
    n, T, ux, uy = 1.07, 0.93, 0.21, -0.13
    g = 1 / math.sqrt(1 - ux * ux - uy * uy)
    U = np.array([g, g * ux, g * uy])
    f = e.feq(np.array([n]), U.reshape(3, 1), np.array([T]))[:, 0]

    def mj(alphas):
        zeta = mp.mpf(m) / mp.mpf(T)
        tot = mp.mpf(0)
        for pairs, singles in L._pairings(range(len(alphas))):
            r = len(alphas) - len(pairs)
            term = (-1) ** len(pairs) * zeta ** (r - 1) * mp.besselk(r + 0.5, zeta) / mp.besselk(1.5, zeta)
            for (i, j) in pairs:
                term *= L.ETA[alphas[i], alphas[j]]
            for s in singles:
                term *= mp.mpf(float(U[alphas[s]]))
            tot += term
        return mp.mpf(n) * mp.mpf(T) ** (len(alphas) - 1) * tot

    with localcontext() as ctx:
        ctx.prec = 50
        rows, mons = L._gram_schmidt_decimal(3, m)
    M = [mj((0,) * c + (1,) * a + (2,) * b) for (c, a, b) in mons]
    a = [sum(mp.mpf(str(r[k])) * M[k] for k in range(len(mons))) for r in rows]
    want = np.array([float(mp.mpf(float(q.w[i])) * sum(a[k] * mp.mpf(str(e.J_ld[k, i])) for k in range(len(a))))
                     for i in range(q.Q)])
    assert np.abs(f - want).max() <= 1e-15 * np.abs(want).max()


def test_non_physical_cells_are_left_unrelaxed():
    """A cell without a physical Landau frame (here its populations negated:
    no positive density) keeps its populations through the collision, and
    every other cell is relaxed as usual (reading of states the paper does
    not discuss)."""
    q = L.massless_quadrature(2)
    e = L.Expansion(q)
    n, ux, uy, T = _random_state((6, 7), umax=0.2)
    f = e.feq(n, P.four_velocity(ux, uy), T)
    f = f * (1 + 0.05 * RNG.standard_normal(f.shape))
    f[:, 2, 3] = -f[:, 2, 3]
    with np.errstate(invalid="ignore", divide="ignore"):
        fs, fl = S.collide(f, q, e, 0.9)
    assert not S.physical(fl)[2, 3] and S.physical(fl).sum() == 41
    assert np.array_equal(fs[:, 2, 3], f[:, 2, 3])
    assert np.all(np.isfinite(fs))
    good = S.physical(fl)
    assert np.abs(fs - f)[:, good].max() > 1e-6                 # the others do relax
