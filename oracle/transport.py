"""First-order Chapman-Enskog transport coefficients of a discrete velocity
set, FP64 (oracle; test infrastructure only).

App. C obtains eta, lambda and mu from the Anderson-Witting correction
f^(1) = -(tau / (p.U)) p^mu d_mu f_eq, with the gradients' time parts taken
from the Euler equations, integrated over momentum space.  A lattice replaces
the integrals by sums over its quadrature and f_eq by the polynomial
equilibrium of Eq. mj-discrete-feq; the same first-order correction summed
that way is what the scheme's pre-collision populations carry.  It differs
from App. C where the quadrature does not integrate the correction exactly:
the factor 1/p0 makes the integrands non-polynomial.  ``first_order``
takes the velocity set and the equilibrium as inputs, so a fine quadrature of
the exact Maxwell-Juttner distribution reproduces App. C (the pin of this
module) and a lattice quadrature gives the lattice's own coefficients.

Lattice units c = k_B = 1, d = 2; everything is evaluated at rest with
n = T = 1 (so P = n T = 1).
"""
from __future__ import annotations

import numpy as np

from oracle import physics as P


def _ddx(f, h=1e-3):
    """Derivative at 0 by the fourth-order central difference
    (8 (f(h) - f(-h)) - (f(2h) - f(-2h))) / (12 h)."""
    return (8.0 * (f(h) - f(-h)) - (f(2 * h) - f(-2 * h))) / (12.0 * h)


def first_order(p, feq, m, d=2):
    """eta / (P tau), lambda / (n tau), mu / (P tau) of the velocity set.

    p:   (Q, 3) momenta p^mu of the populations.
    feq: callable (n, ux, uy, T) -> (Q,) equilibrium populations (weights
         included, so that N^mu = sum_i f_i p_i^mu).
    m:   particle mass (m~ with T = 1).

    Flows, each with unit gradient at a point of a fluid at rest, n = T = 1,
    the time derivatives from the Euler equations:
      shear  d_y U^x = 1:                      d_t = 0
      heat   d_x T = 1, d_x n = -1 (d_x P = 0): d_t = 0
      bulk   theta = d_x U^x = 1:              d_t n = -n theta,
             d_t T = -(T / c_v) theta, c_v = d(eps/n)/dT (Eq. eos-ddim).
    f^(1) = -tau p^mu d_mu f_eq / p0 (p.U = p0 at rest), tau = 1, and
      eta    = -pi^xy          = -sum_i p^x p^y f^(1)_i,
      lambda = -q^x / d_x T    = h_e sum_i p^x f^(1)_i   (q = h_e (N_E - N),
                                 N_E^x = 0; h_e = (eps + P) / n),
      mu     = -varpi / theta  = (1/d) sum_i (p.p) f^(1)_i  (Eq. varpi-from-
                                 tensor with T^mu_mu = m^2 sum_i f_i).
    """
    p = np.asarray(p, dtype=np.float64)
    p0, px, py = p[:, 0], p[:, 1], p[:, 2]
    e = lambda T: float(P.energy_per_particle(np.array(T), m, d))
    cv = _ddx(lambda h: e(1.0 + h))
    he = e(1.0) + 1.0
    f_n = _ddx(lambda h: feq(1.0 + h, 0.0, 0.0, 1.0))
    f_T = _ddx(lambda h: feq(1.0, 0.0, 0.0, 1.0 + h))
    f_ux = _ddx(lambda h: feq(1.0, h, 0.0, 1.0))
    shear = -(py / p0) * f_ux
    heat = -(px / p0) * (-f_n + f_T)
    bulk = -(1.0 / p0) * (p0 * (-f_n - f_T / cv) + px * f_ux)
    msq = p0 * p0 - px * px - py * py
    return dict(eta=-float(np.sum(px * py * shear)),
                lam=he * float(np.sum(px * heat)),
                mu=float(np.sum(msq * bulk)) / d)


def lattice_feq(expansion):
    """The polynomial equilibrium of an oracle ``Expansion`` as the callable
    ``first_order`` takes."""
    def feq(n, ux, uy, T):
        g = 1.0 / np.sqrt(1.0 - ux * ux - uy * uy)
        U = np.array([g, g * ux, g * uy])
        return expansion.feq(np.array(float(n)), U, np.array(float(T)))
    return feq


def first_order_3d(p, feq):
    """``first_order`` for massless particles in d = 3: eta / (P tau) and
    mu / (P tau) (the latter zero: T^mu_mu = 0 on the light cone).

    p:   (Q, 4) momenta (p0, px, py, pz);
    feq: callable (n, ux, uy, uz, T) -> (Q,) equilibrium populations.
    Shear flow d_y U^x = 1 at rest, n = T = 1 (d_t = 0):
    f^(1) = -tau (p^y / p0) d f_eq / d U^x, eta = -sum_i p^x p^y f^(1)_i;
    uniform expansion theta = d_x U^x = 1: d_t n = -n, d_t T = -T / c_v with
    c_v = 3 (eps = 3 n T), mu = (1/3) sum_i (p.p) f^(1)_i."""
    p = np.asarray(p, dtype=np.float64)
    p0, px, py, pz = p[:, 0], p[:, 1], p[:, 2], p[:, 3]
    f_n = _ddx(lambda h: feq(1.0 + h, 0.0, 0.0, 0.0, 1.0))
    f_T = _ddx(lambda h: feq(1.0, 0.0, 0.0, 0.0, 1.0 + h))
    f_ux = _ddx(lambda h: feq(1.0, h, 0.0, 0.0, 1.0))
    shear = -(py / p0) * f_ux
    bulk = -(1.0 / p0) * (p0 * (-f_n - f_T / 3.0) + px * f_ux)
    msq = p0 * p0 - px * px - py * py - pz * pz
    return dict(eta=-float(np.sum(px * py * shear)), mu=float(np.sum(msq * bulk)) / 3.0)


def lattice_feq_3d(expansion):
    """The equilibrium of an oracle ``d3.Expansion3`` as ``first_order_3d`` takes it."""
    def feq(n, ux, uy, uz, T):
        g = 1.0 / np.sqrt(1.0 - ux * ux - uy * uy - uz * uz)
        U = np.array([g, g * ux, g * uy, g * uz])
        return expansion.feq(np.array(float(n)), U, np.array(float(T)))
    return feq
