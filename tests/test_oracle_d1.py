"""Pins of the (1+1)-d massless oracle (oracle/d1.py) against what the paper
and the mathematics fix: the App. H table digits as Gauss-Laguerre rules,
the printed first-order equilibrium, Maxwell-Juttner moments by numerical
integration, the Landau frame of boosted ideal fluids, conservation."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import d1

RNG = np.random.default_rng(11)


@pytest.mark.parametrize("order", [2, 3, 4, 5])
def test_tables_are_gauss_laguerre_rules_divided_by_the_node(order):
    """App. H (1+1)-d: shells = roots of the Laguerre polynomial L_N and
    weights = Gauss-Laguerre weight / node (the measure dp/p0), with the
    order-4 columns read exchanged (as printed, they are not)."""
    x, wgl = np.polynomial.laguerre.laggauss(order)
    shells, w = d1.massless_table_1d(order)
    idx = np.argsort(shells)
    assert np.abs(np.array(shells)[idx] - x).max() < 1e-14 * x.max()
    assert np.abs(np.array(w)[idx] - wgl / x).max() < 1e-13 * (wgl / x).max()
    if order == 4:
        p0_printed, _ = d1.MASSLESS_D1_PRINTED[4]
        assert np.abs(np.sort(p0_printed) - x).max() > 0.1       # the printed column is not the nodes


@pytest.mark.parametrize("order", [2, 3, 4, 5])
def test_quadrature_integrates_omega_moments_up_to_degree_2N(order):
    """sum_i w_i (p0)^a sign^s = int exp(-p0)/2 (p0)^a sign^s dp/p0 =
    Gamma(a) (s even), 0 (s odd), for 1 <= a <= 2N."""
    q = d1.massless_quadrature_1d(order)
    sg = np.sign(q.p[:, 1])
    for a in range(1, 2 * order + 1):
        for s in (0, 1):
            got = np.sum(q.w * q.p[:, 0] ** a * sg ** s)
            want = math.gamma(a) if s == 0 else 0.0
            assert abs(got - want) <= 1e-12 * math.gamma(a)


@pytest.mark.parametrize("a,s", [(1, 0), (1, 1), (2, 0), (2, 1), (3, 0), (3, 1), (4, 1)])
def test_mj_moments_match_numerical_integration(a, s):
    """int f_MJ (p0)^a sign^s dp/p0 with f_MJ = n/(2T) exp(-p.U/T),
    integrated numerically on both half-lines."""
    for (n, T, u) in [(1.0, 1.0, 0.0), (0.7, 1.3, 0.4), (1.4, 0.8, -0.6)]:
        g = 1 / math.sqrt(1 - u * u)
        U0, Ux = g, g * u
        tot = 0.0
        for sg in (1, -1):
            f = lambda x: n / (2 * T) * math.exp(-x * (U0 - sg * Ux) / T) * x ** (a - 1) * sg ** s
            tot += integrate.quad(f, 0, np.inf, epsabs=0, epsrel=1e-13)[0]
        assert abs(d1.mj_moment_1d(a, s, n, U0, Ux, T) - tot) <= 1e-11 * max(1.0, abs(tot))


def test_first_order_expansion_is_the_printed_formula():
    """The massless limit at N = 1 (basis p0, p^x plus the constant limit)
    is Eq. after mj-expanded-1D-massless: F = n ((1 - p0)/T + p0 U^0 + p^x U^x),
    for any momentum, not only at quadrature nodes."""
    q1 = d1.Quadrature1(np.array([1, -1]), np.array([[1.0, 1.0], [1.0, -1.0]]), np.array([0.5, 0.5]), 1)
    e = d1.Expansion1(q1)
    for (n, T, u) in [(1.0, 1.0, 0.2), (0.6, 1.7, -0.5), (2.0, 0.5, 0.7)]:
        U = d1.four_velocity1(np.array([u]))
        for p0 in (0.1, 0.7, 2.5, 9.0):
            for sg in (1, -1):
                F = e.F(np.array([n]), U, np.array([T]), np.array([[p0, sg * p0]]))[0, 0]
                printed = n * ((1 - p0) / T + p0 * U[0, 0] + sg * p0 * U[1, 0])
                assert abs(F - printed) <= 1e-13 * max(1.0, abs(printed))


@pytest.mark.parametrize("order", [2, 3, 4])
def test_equilibrium_recovers_the_maxwell_juttner_moments(order):
    """sum_i f^eq_i (p0)^a sign^s = M_{a,s}(n, U, T) for every member of the
    basis (a <= N): in particular N^a = n U^a and T^{ab} of the ideal fluid."""
    q = d1.massless_quadrature_1d(order)
    e = d1.Expansion1(q)
    n = RNG.uniform(0.5, 1.5, 6)
    T = RNG.uniform(0.6, 1.6, 6)
    u = RNG.uniform(-0.6, 0.6, 6)
    U = d1.four_velocity1(u)
    f = e.feq(n, U, T)
    sg = np.sign(q.p[:, 1])
    for a in range(1, order + 1):
        for s in (0, 1):
            got = np.sum(f * (q.p[:, 0] ** a * sg ** s)[:, None], axis=0)
            want = d1.mj_moment_1d(a, s, n, U[0], U[1], T)
            assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max() + 1e-14


def test_rest_frame_at_reference_temperature_is_n_times_weight():
    """At rest and T = T0 = 1, f_MJ / omega = n exactly, so f^eq_i = n w_i."""
    for order in (2, 3, 5):
        q = d1.massless_quadrature_1d(order)
        e = d1.Expansion1(q)
        f = e.feq(np.array([1.3]), np.array([[1.0], [0.0]]), np.array([1.0]))[:, 0]
        assert np.abs(f - 1.3 * q.w).max() <= 1e-13 * f.max()


@pytest.mark.parametrize("beta", [0.0, 0.3, -0.7, 0.95])
def test_landau_frame_of_boosted_ideal_fluid(beta):
    """T^{ab} = (eps + P) U^a U^b - P eta^{ab}, N = n U with eps = P = n T:
    the 2 x 2 solve returns eps, U and n of the boost."""
    n, T = 0.8, 1.3
    eps = P = n * T
    g = 1 / math.sqrt(1 - beta * beta)
    U = np.array([g, g * beta])
    Tab = (eps + P) * np.outer(U, U) - P * d1.ETA2
    e_, U_, n_, ok = d1.landau2((n * U).reshape(2, 1), Tab.reshape(2, 2, 1))
    assert ok[0]
    assert abs(e_[0] - eps) < 1e-13 and abs(n_[0] - n) < 1e-13
    assert np.abs(U_[:, 0] - U).max() < 1e-12 * g


def test_collision_conserves_N0_and_T0a_per_cell():
    q = d1.massless_quadrature_1d(3)
    e = d1.Expansion1(q)
    nx = 16
    f = e.feq(RNG.uniform(0.7, 1.3, nx), d1.four_velocity1(RNG.uniform(-0.4, 0.4, nx)), RNG.uniform(0.8, 1.2, nx))
    f = f * (1 + 0.05 * RNG.standard_normal(f.shape))          # off equilibrium
    fs, _ = d1.collide1(f, q, e, 0.8)
    # N^0, T^00, T^0x are collision invariants (Landau matching); N^x is not
    for moment in (q.p[:, 0], q.p[:, 0] ** 2, q.p[:, 0] * q.p[:, 1]):
        d = np.sum(moment[:, None] * (fs - f), axis=0)
        assert np.abs(d).max() <= 1e-13 * np.sum(np.abs(moment)[:, None] * f, axis=0).max()


def test_periodic_run_conserves_global_moments_and_streams_exactly():
    q = d1.massless_quadrature_1d(2)
    nx = 40
    sim = d1.Simulation1(q, nx, tau=0.9)
    x = np.arange(nx)
    sim.init(1 + 0.1 * np.sin(2 * np.pi * x / nx), 0.2 * np.cos(2 * np.pi * x / nx),
             1 + 0.05 * np.cos(4 * np.pi * x / nx))
    N0 = np.sum(q.p[:, 0][:, None] * sim.fs)
    T00 = np.sum((q.p[:, 0] ** 2)[:, None] * sim.fs)
    T0x = np.sum((q.p[:, 0] * q.p[:, 1])[:, None] * sim.fs)
    sim.step(50)
    assert abs(np.sum(q.p[:, 0][:, None] * sim.fs) / N0 - 1) < 1e-13
    assert abs(np.sum((q.p[:, 0] ** 2)[:, None] * sim.fs) / T00 - 1) < 1e-13
    assert abs(np.sum((q.p[:, 0] * q.p[:, 1])[:, None] * sim.fs) - T0x) < 1e-13 * T00
    # a single population moves by exactly its direction each step
    f = np.zeros((q.Q, nx))
    f[1, 7] = 1.0
    out = d1.stream1(f, q.n)
    assert out[1, 7 + q.n[1]] == 1.0 and out.sum() == 1.0
