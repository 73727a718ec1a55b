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


def oracle_sim(quad, nx, ny, tau=1.0, boundary="periodic", stream="onlattice", lam=None):
    return OS.Simulation(quad, OL.Expansion(quad), nx, ny, tau=tau, boundary=boundary,
                         stream=stream, lam=lam)


def rel_linf(a, b):
    """max |a - b| / max |b| (relative L-infinity, normalised by the reference)."""
    return float(np.abs(a - b).max() / np.abs(b).max())
