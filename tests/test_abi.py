"""CPU-side checks of the C-ABI library: it loads, exports every symbol that
include/rlbm.h declares, and its host-side setup (quadratures, equilibrium
matrix: Sec. 5.2-5.3, App. F-H) agrees with the oracle.  No compute call here
needs a GPU."""
import json
import os
import re

import numpy as np
import pytest

from oracle import lattice as OL
from oracle import physics as OP
from tests.cases import oracle_quadrature

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def rl():
    from paper_1909_04502_gb300 import build, rlbm
    build.build()
    return rlbm


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "rlbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rlbm_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(rl):
    L = rl.lib()
    syms = declared_symbols()
    assert len(syms) >= 15
    for s in syms:
        assert hasattr(L, s), s
    # and the Python binding knows every one of them
    assert set(syms) <= set(rl.SIGNATURES)


def test_strerror_and_invalid_create(rl):
    L = rl.lib()
    assert L.rlbm_strerror(-4).decode() == "non-physical cell state"
    p, keep = rl.make_params(0, 8)                       # nx = 0
    import ctypes
    h = ctypes.c_void_p()
    assert L.rlbm_create(ctypes.byref(p), ctypes.byref(h)) == -1
    assert "grid" in L.rlbm_last_error(None).decode()
    p, keep = rl.make_params(8, 8, tau=0.4)
    assert L.rlbm_create(ctypes.byref(p), ctypes.byref(h)) == -1
    p, keep = rl.make_params(8, 8)
    p.d = 3
    assert L.rlbm_create(ctypes.byref(p), ctypes.byref(h)) == -2
    # d = 1 is a one-dimensional problem on an nx x 1 grid
    p, keep = rl.make_params(8, 2, d=1)
    assert L.rlbm_create(ctypes.byref(p), ctypes.byref(h)) == -1
    assert "ny = 1" in L.rlbm_last_error(None).decode()
    p, keep = rl.make_params(8, 1, d=4)
    assert L.rlbm_create(ctypes.byref(p), ctypes.byref(h)) == -1


def test_one_dimensional_plan_uses_the_two_dimensional_stencil(rl):
    a = rl.plan(nx=64, ny=1, d=1)
    b = rl.plan(nx=64, ny=1, d=2)
    assert a["Q"] == b["Q"] == 28
    assert np.array_equal(a["p"], b["p"]) and np.array_equal(a["H"], b["H"])


def _key(n, p0):
    return (int(n[0]), int(n[1]), round(float(p0), 10))


def _match(plan, quad):
    """Permutation idx with plan row idx[j] == oracle row j."""
    pos = {_key(plan["n"][i], plan["p"][i, 0]): i for i in range(plan["Q"])}
    return np.array([pos[_key(quad.n[j], quad.p[j, 0])] for j in range(quad.Q)])


@pytest.mark.parametrize("order", [2, 3])
def test_massless_tables_agree_with_oracle(rl, order):
    d = rl.plan(nx=16, ny=16, order=order)
    q = OL.massless_quadrature(order)
    assert d["Q"] == q.Q
    idx = _match(d, q)
    assert np.abs(d["p"][idx] - q.p).max() < 1e-15
    assert np.abs(d["w"][idx] - q.w).max() == 0.0


def test_mass5_example_weights_from_product_solver(rl):
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "mass5_worked_example.json")))
    d = rl.plan(nx=8, ny=8, m=5.0, groups=g["groups"], v0=g["v0"])
    q, _ = OL.massive_quadrature([tuple(x) for x in g["groups"]], 5.0, g["v0"])
    idx = _match(d, q)
    # the 45 x 6 system has condition number ~2.9e3 at v0 = 0.2726 (w2 sits
    # next to its pruning value): independent double-precision solutions
    # agree to ~1e-13 absolute, and the printed digits carry the same error
    assert np.abs(d["w"][idx] - q.w).max() < 1e-13
    assert np.allclose(sorted(set(np.round(d["w"], 15))), sorted(g["weights"]), rtol=0, atol=5e-14)


def _mj_vector(order, m, n, U, T):
    """MJ moments of the product basis p0^e px^a py^b via the oracle's App. B;
    at order 3 the members with p0 are shifted, <(p0 - m) X> = <p0 X> - m <X>."""
    mons = []
    for deg in range(order + 1):
        if deg >= 1:
            mons += [(1, a, deg - 1 - a) for a in range(deg - 1, -1, -1)]
        mons += [(0, a, deg - a) for a in range(deg, -1, -1)]
    M = {mo: OL.mj_monomial_moment(mo, n, U, T, m) for mo in mons}
    if order == 3:
        return np.array([M[mo] - m * M[(0, mo[1], mo[2])] if mo[0] == 1 else M[mo] for mo in mons])
    return np.array([M[mo] for mo in mons])


@pytest.mark.parametrize("case", [("massless", 2, 0.0), ("massless", 3, 0.0), ("massive", 2, 1.0),
                                  ("massive", 2, 5.0), ("massive", 2, 10.0), ("massive", 3, 2.0),
                                  ("massive", 3, 5.0)])
def test_equilibrium_matrix_reproduces_oracle_feq(rl, case):
    kind, order, m = case
    d = rl.plan(nx=8, ny=8, m=m, order=order)
    if kind == "massless":
        q = OL.massless_quadrature(order)
    else:
        # the product's weights satisfy the orthonormality conditions (oracle basis)
        C, mons = OL.gram_schmidt_basis(order, m)
        J = C @ OL.eval_monomials(mons, d["p"])
        assert np.abs((J * d["w"]) @ J.T - np.eye(J.shape[0])).max() < 1e-11
        assert np.all(d["w"] > 0)
        # the oracle's own weights on the same stencil and v0
        q = oracle_quadrature(m, order, d["n"], d["v0"])
    idx = _match(d, q)
    e = OL.Expansion(q)
    rng = np.random.default_rng(7)
    for _ in range(5):
        n, T = rng.uniform(0.5, 2), rng.uniform(0.7, 1.5)
        u = rng.uniform(-0.5, 0.5, 2)
        U = OP.four_velocity(np.array(u[0]), np.array(u[1]))
        feq_o = e.feq(np.array(n), U, np.array(T))
        feq_p = d["H"] @ _mj_vector(order, m, n, U, T)
        # both sides round the same exact weights; the rest is the rounding of
        # the two equilibrium evaluations (raw monomials on the oracle side)
        tol = 1e-13 if kind == "massless" else 5e-13
        assert np.abs(feq_p[idx] - feq_o).max() < tol * np.abs(feq_o).max()


def test_builtin_massive_quadratures_exist_for_sweep_masses(rl):
    for m in (1.0, 10.0):
        d = rl.plan(nx=8, ny=8, m=m)
        assert d["Q"] <= 40 and np.all(d["w"] > 0) and abs(d["w"].sum() - 1) < 1e-12


@pytest.mark.parametrize("order", [2, 3])
def test_massless_tables_are_in_orbit_order_with_exactly_symmetric_H(rl, order):
    """The built-in massless stencil comes in orbit order: per (3, 4) shell the
    sign quartets of (a, b) and of (b, a), per (5, 0) shell (p, 0), (-p, 0),
    (0, p), (0, -p); every H row equals its orbit's first row with the column
    signs of the flips and, for the swapped members, px <-> py exchanged
    columns -- exactly (the kernels evaluate moments and equilibrium from the
    first rows only)."""
    d = rl.plan(nx=16, ny=16, order=order)
    Q, K, p, H = d["Q"], d["K"], d["p"], d["H"]
    basis = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1), (0, 0, 2),
             (1, 2, 0), (1, 1, 1), (1, 0, 2), (0, 3, 0), (0, 2, 1), (0, 1, 2), (0, 0, 3)][:K]
    swap = [basis.index((e, b, a)) for (e, a, b) in basis]
    n8, n4 = (3, 1) if order == 2 else (4, 3)
    assert Q == 8 * n8 + 4 * n4

    def image(i0, sx, sy, sw):
        bx, by = (p[i0, 2], p[i0, 1]) if sw else (p[i0, 1], p[i0, 2])
        sgn = np.array([sx ** a * sy ** b for (_, a, b) in basis], dtype=float)
        row = H[i0][swap] if sw else H[i0]
        return np.array([p[i0, 0], sx * bx, sy * by]), sgn * row

    members8 = [(1, 1, 0), (-1, 1, 0), (1, -1, 0), (-1, -1, 0), (1, 1, 1), (-1, 1, 1), (1, -1, 1), (-1, -1, 1)]
    members4 = [(1, 1, 0), (-1, 1, 0), (1, 1, 1), (1, -1, 1)]
    for o in range(n8 + n4):
        i0 = 8 * o if o < n8 else 8 * n8 + 4 * (o - n8)
        for m, (sx, sy, sw) in enumerate(members8 if o < n8 else members4):
            pm, row = image(i0, sx, sy, sw)
            assert np.array_equal(p[i0 + m], pm), (o, m)
            assert np.array_equal(H[i0 + m], row), (o, m)
        if o >= n8:
            assert p[i0, 2] == 0.0 and all(H[i0][k] == 0.0 for k, (_, a, b) in enumerate(basis) if b % 2)


@pytest.mark.parametrize("m,order,Q,comp", [
    (1.0, 2, 33, (3, 1, 1, 1)), (5.0, 2, 29, (2, 1, 2, 1)), (10.0, 2, 25, (1, 2, 2, 1)),
    (2.0, 3, 65, (7, 0, 2, 1)), (3.0, 3, 57, (5, 1, 3, 1)), (5.0, 3, 49, (3, 4, 2, 1)),
    (10.0, 3, 53, (4, 3, 2, 1))])
def test_builtin_massive_tables_are_in_orbit_order_with_exactly_symmetric_H(rl, m, order, Q, comp):
    """The built-in massive stencils come in orbit order too: eight-member
    orbits (sign quartets of (a, b) and (b, a)), axis quartets (p, 0), (-p, 0),
    (0, p), (0, -p), diagonal quartets (a, a), (-a, a), (a, -a), (-a, -a), the
    rest population; weights and H rows are exact images of each orbit's first
    member (what the kernels' symmetric evaluation uses)."""
    d = rl.plan(nx=16, ny=16, m=m, order=order)
    assert d["Q"] == Q
    p, H, w = d["p"], d["H"], d["w"]
    # exponents (e, a, b) of p0^e px^a py^b in the library's moment order
    basis = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1), (0, 0, 2)]
    if order == 3:
        basis += [(1, 2, 0), (1, 1, 1), (1, 0, 2), (0, 3, 0), (0, 2, 1), (0, 1, 2), (0, 0, 3)]
    swap = [basis.index((e, b, a)) for (e, a, b) in basis]

    def member(i0, sx, sy, sw):
        bx, by = (p[i0, 2], p[i0, 1]) if sw else (p[i0, 1], p[i0, 2])
        sgn = np.array([sx ** a * sy ** b for (_, a, b) in basis], dtype=float)
        return np.array([p[i0, 0], sx * bx, sy * by]), sgn * (H[i0][swap] if sw else H[i0])

    quart = [(1, 1, 0), (-1, 1, 0), (1, -1, 0), (-1, -1, 0)]
    layouts = ([quart + [(sx, sy, 1) for sx, sy, _ in quart]] * comp[0]
               + [[(1, 1, 0), (-1, 1, 0), (1, 1, 1), (1, -1, 1)]] * comp[1] + [quart] * comp[2])
    i0 = 0
    for lay in layouts:
        for k, (sx, sy, sw) in enumerate(lay):
            pm, row = member(i0, sx, sy, sw)
            assert np.array_equal(p[i0 + k], pm) and w[i0 + k] == w[i0]
            assert np.array_equal(H[i0 + k], row)
        i0 += len(lay)
    for _ in range(comp[3]):
        assert p[i0, 1] == 0.0 and p[i0, 2] == 0.0
        assert all(H[i0][k] == 0.0 for k, (_, a, b) in enumerate(basis) if a % 2 or b % 2)
        i0 += 1
    assert i0 == Q


# the library's moment order: 1 | p0 px py pz | p0px p0py p0pz pxpx pxpy pxpz
# pypy pypz pzpz, then (order 3) p0 (xx xy xz yy yz zz) | xxx ... zzz
_D3_BASIS = [(0, 0, 0, 0), (1, 0, 0, 0), (0, 1, 0, 0), (0, 0, 1, 0), (0, 0, 0, 1),
             (1, 1, 0, 0), (1, 0, 1, 0), (1, 0, 0, 1), (0, 2, 0, 0), (0, 1, 1, 0),
             (0, 1, 0, 1), (0, 0, 2, 0), (0, 0, 1, 1), (0, 0, 0, 2),
             (1, 2, 0, 0), (1, 1, 1, 0), (1, 1, 0, 1), (1, 0, 2, 0), (1, 0, 1, 1), (1, 0, 0, 2),
             (0, 3, 0, 0), (0, 2, 1, 0), (0, 2, 0, 1), (0, 1, 2, 0), (0, 1, 1, 1), (0, 1, 0, 2),
             (0, 0, 3, 0), (0, 0, 2, 1), (0, 0, 1, 2), (0, 0, 0, 3)]


@pytest.mark.parametrize("order,Q,K", [(2, 78, 14), (3, 288, 30)])
def test_d3_tables_agree_with_oracle(rl, order, Q, K):
    """The (3+1)-d massless tables: the same stencil, momenta and weights as
    the oracle's reading of App. H, and an equilibrium matrix that reproduces
    the oracle's f^eq at random states (moments from the oracle's App. B
    closed forms, in the library's order)."""
    from oracle import d3
    d = rl.plan3(order)
    q = d3.massless_quadrature_3d(order)
    assert d["Q"] == q.Q == Q and d["K"] == K
    key = lambda n, p0: (tuple(int(v) for v in n), round(float(p0), 12))
    ko = {key(n, p[0]): i for i, (n, p) in enumerate(zip(q.n, q.p))}
    idx = np.array([ko[key(n, p[0])] for n, p in zip(d["n"], d["p"])])
    assert sorted(idx.tolist()) == list(range(Q))
    assert np.abs(d["p"] - q.p[idx]).max() < 1e-14 * q.p[:, 0].max() and np.array_equal(d["w"], q.w[idx])
    E = d3.Expansion3(q, order=order)
    rng = np.random.default_rng(2)
    for _ in range(5):
        n, T = rng.uniform(0.5, 1.5), rng.uniform(0.7, 1.4)
        u = rng.uniform(-0.3, 0.3, 3)
        g = 1 / np.sqrt(1 - u @ u)
        U = np.concatenate([[g], g * u])
        M = np.array([d3.mj_moment_3d(mon, n, U, T) for mon in _D3_BASIS[:K]])
        fo = E.feq(np.array(n), U, np.array(T))
        assert np.abs(d["H"] @ M - fo[idx]).max() < 1e-13 * np.abs(fo).max()


@pytest.mark.parametrize("order", [2, 3])
def test_d3_tables_come_in_sign_orbits(rl, order):
    """The (3+1)-d tables in sign-orbit order: each run shares p0, the weight
    and |n| componentwise, its member s negates the components whose bit is
    set in s (over the non-zero components), and its equilibrium rows are the
    first row times the sign each basis member takes, exactly; at order 2 the
    runs are nine of eight, then the axis pairs along x, y and z (the layout
    the sign-orbit kernels take)."""
    d = rl.plan3(order)
    n, p, w, H = d["n"], d["p"], d["w"], d["H"]
    basis = np.array(_D3_BASIS[:d["K"]])
    i, masks = 0, []
    while i < d["Q"]:
        a = n[i]
        assert np.all(a >= 0)
        mask = sum(1 << k for k in range(3) if a[k])
        members = [sg for sg in range(8) if not (sg & ~mask)]
        for j, sg in enumerate(members):
            sign = np.array([-1 if (sg >> k) & 1 else 1 for k in range(3)])
            assert np.array_equal(n[i + j], sign * a)
            assert p[i + j, 0] == p[i, 0] and np.array_equal(p[i + j, 1:], sign * p[i, 1:])
            assert w[i + j] == w[i]
            chi = np.prod(sign[None, :] ** basis[:, 1:], axis=1)
            assert np.array_equal(H[i + j], chi * H[i])
        masks.append(mask)
        i += len(members)
    assert i == d["Q"]
    if order == 2:
        assert masks == [7] * 9 + [1, 2, 4]


def _cuda_int_table(path, name):
    """The integers of a brace-initialised constant table in a CUDA source."""
    import re as _re
    src = open(path).read()
    m = _re.search(name + r"\[[^=]*=\s*\{(.*?)\};", src, _re.S)
    body = _re.sub(r"//[^\n]*", "", m.group(1))
    return [int(t) for t in _re.findall(r"-?\d+", body)]


def test_sign_orbit_tables_of_the_kernels_match_the_basis():
    """The parity tables compiled into the (3+1)-d sign-orbit kernels are the
    parities of the basis members' x, y, z exponents."""
    csrc = os.path.join(os.path.dirname(__file__), "..", "paper_1909_04502_gb300", "csrc")
    par = _cuda_int_table(os.path.join(csrc, "step3q.cu"), "kBasis3o3Par")
    want = [(b[1] & 1) | ((b[2] & 1) << 1) | ((b[3] & 1) << 2) for b in _D3_BASIS]
    assert par == want
    exp2 = _cuda_int_table(os.path.join(csrc, "step3.cu"), "kBasis3Exp")
    assert exp2 == [e for b in _D3_BASIS[:14] for e in b[1:]]


@pytest.mark.parametrize("order", [2, 3])
def test_sign_orbit_evaluation_equals_row_by_row(rl, order):
    """The sign-orbit kernels' algebra on the library's tables: per run, the
    Walsh-Hadamard transform of the populations times the first member's
    monomials gives the moments N^a, T^ab, and the transformed parity-class
    sums of the first H row give every member's f^eq; both agree with the
    row-by-row sums to rounding."""
    d = rl.plan3(order)
    n, p, H, K = d["n"], d["p"], d["H"], d["K"]
    basis = np.array(_D3_BASIS[:K])
    cls = (basis[:, 1] & 1) | ((basis[:, 2] & 1) << 1) | ((basis[:, 3] & 1) << 2)
    rng = np.random.default_rng(order)
    f = rng.uniform(0.1, 1.0, d["Q"])
    M = rng.normal(size=K)
    N_row = p.T @ f
    T_row = np.einsum("qa,qb,q->ab", p, p, f)
    feq_row = H @ M
    N_orb, T_orb, feq_orb = np.zeros(4), np.zeros((4, 4)), np.zeros(d["Q"])
    i = 0
    while i < d["Q"]:
        mask = sum(1 << k for k in range(3) if n[i][k])
        members = [sg for sg in range(8) if not (sg & ~mask)]
        L = len(members)
        # characters chi_c(s) = (-1)^popcount(c & s) over the run's members
        chi = np.array([[(-1) ** bin(c & sg).count("1") for sg in members] for c in members], dtype=float)
        F = chi @ f[i:i + L]
        Fc = dict(zip(members, F))
        p0 = p[i]
        for a in range(4):
            ca = 0 if a == 0 else 1 << (a - 1)
            N_orb[a] += p0[a] * Fc.get(ca, 0.0)
            for b in range(4):
                cb = 0 if b == 0 else 1 << (b - 1)
                T_orb[a, b] += p0[a] * p0[b] * Fc.get(ca ^ cb, 0.0)
        C = {c: 0.0 for c in members}
        for k in range(K):
            c = cls[k] & mask
            C[c] += H[i, k] * M[k]
        for j, sg in enumerate(members):
            feq_orb[i + j] = sum((-1) ** bin(c & sg).count("1") * C[c] for c in members)
        i += L
    assert np.allclose(N_orb, N_row, rtol=1e-13, atol=1e-13 * np.abs(N_row).max())
    assert np.allclose(T_orb, T_row, rtol=1e-13, atol=1e-13 * np.abs(T_row).max())
    assert np.allclose(feq_orb, feq_row, rtol=1e-12, atol=1e-13 * np.abs(feq_row).max())


def test_d3_plan_rejects_other_orders(rl):
    with pytest.raises(rl.RLBMError):
        rl.plan3(4)
