"""The (3+1)-d massless step (rlbm3_*) against the (3+1)-d oracle: element by
element on small ragged grids, the fields it reports, and conservation of
N^0 and T^{0a} over a longer periodic run."""
import numpy as np
import pytest

from oracle import d3
from paper_1909_04502_gb300 import inputs
from tests.cases import rel_linf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rl():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_04502_gb300 import build, rlbm
    build.build()
    return rlbm


def _pair(rl, nx, ny, nz, tau, fields, precision="fp64", order=2):
    lat = rl.Lattice3(nx, ny, nz, tau=tau, precision=precision, order=order)
    q = d3.massless_quadrature_3d(order)
    key = lambda n, p0: (tuple(int(v) for v in n), round(float(p0), 12))
    ko = {key(n, p[0]): i for i, (n, p) in enumerate(zip(q.n, q.p))}
    idx = np.array([ko[key(n, p[0])] for n, p in zip(lat.n, lat.p)])
    sim = d3.Simulation3(q, d3.Expansion3(q, order=order), nx, ny, nz, tau=tau)
    fields = [np.ascontiguousarray(a) for a in fields]
    lat.init(*fields)
    sim.init(*fields)
    return lat, sim, idx


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
@pytest.mark.parametrize("order,nx,ny,nz,tau", [(2, 13, 11, 9, 0.9), (2, 37, 5, 3, 1.3), (2, 3, 4, 33, 0.7),
                                                (3, 13, 7, 6, 0.9), (3, 35, 6, 9, 1.3), (3, 6, 8, 7, 0.7)])
def test_step_matches_oracle(rl, order, nx, ny, nz, tau, precision, tol):
    """Ragged grids, 8 steps, both expansion orders: sides of one row segment
    (32 cells) and a tail, others down to the halo width (3 at order 2, 6 at
    order 3: every halo cell an image); the FP64 bar for FP64 storage, 1e-5
    for FP32 storage (populations and fields)."""
    lat, sim, idx = _pair(rl, nx, ny, nz, tau, inputs.random_smooth3(nx, ny, nz, seed=nx, umax=0.2), precision,
                          order)
    for _ in range(2):
        lat.step(4)
        sim.step(4)
        f = lat.populations()
        assert rel_linf(f, sim.fs[idx]) <= tol
    mo = lat.moments()
    fl = sim.fields
    assert rel_linf(mo["n"], fl.n) <= tol and rel_linf(mo["T"], fl.T) <= tol
    umax = max(np.abs(fl.u(k)).max() for k in (1, 2, 3))
    for k, name in ((1, "ux"), (2, "uy"), (3, "uz")):
        assert np.abs(mo[name] - fl.u(k)).max() <= tol * umax
    assert lat.sync_status()[0] == 0
    lat.close()


@pytest.mark.parametrize("order", [2, 3])
def test_init_reports_the_input_fields(rl, order):
    nx, ny, nz = 16, 8, 6
    n, ux, uy, uz, T = inputs.random_smooth3(nx, ny, nz, seed=4, umax=0.3)
    lat = rl.Lattice3(nx, ny, nz, order=order)
    lat.init(*[np.ascontiguousarray(a) for a in (n, ux, uy, uz, T)])
    mo = lat.moments()
    for k, a in (("n", n), ("ux", ux), ("uy", uy), ("uz", uz), ("T", T)):
        assert np.abs(mo[k] - a).max() < 1e-12
    lat.close()


def test_taylor_green_run_conserves_N0_and_T0a(rl):
    """The paper's Taylor-Green flow in the (3+1)-d solver (64^2 x 4, u0 =
    0.2, n = T = 1), 500 steps: the totals of N^0 and T^{0a} move only by
    rounding (a quasi-steady flow rounds the same way every step, so the
    bar is 100 units in the last place per step; measured 39 for T^00), and
    the flow decays."""
    L, nz = 64, 4
    lat = rl.Lattice3(L, L, nz, tau=0.8)
    lat.init(*[np.ascontiguousarray(a) for a in inputs.taylor_green3(L, nz, u0=0.2)])
    p = lat.p

    def totals():
        f = lat.populations().reshape(lat.Q, -1)
        # N^0, then T^{0a} for a = 0..3
        return [float(np.sum(p[:, 0] @ f))] + [float(np.sum((p[:, 0] * p[:, a]) @ f)) for a in range(4)]

    t0 = totals()
    u0 = np.abs(lat.moments()["ux"]).max()
    lat.step(500)
    t1 = totals()
    assert lat.sync_status()[0] == 0
    tol = 100 * 500 * np.finfo(np.float64).eps
    assert abs(t1[0] - t0[0]) <= tol * t0[0]
    for a in range(1, 5):
        assert abs(t1[a] - t0[a]) <= tol * t0[1]
    assert np.abs(lat.moments()["ux"]).max() < 0.9 * u0
    lat.close()


@pytest.mark.parametrize("tau", [0.8, 1.2])
def test_shear_wave_decays_at_the_lattice_viscosity(rl, tau):
    """u_y = A sin(2 pi x / L) on 192 x 3 x 3 cells (dx = 1/3: a population
    moves 3 cells per step at c) decays at eta k^2 / (eps + P), eps + P = 4 n T,
    with eta = (the order-2 table's first-order coefficient, 0.937, against
    the UR 4/5 of Eq. ce-ur-limit) P (tau - 1/2)."""
    from oracle import transport as TR
    q = d3.massless_quadrature_3d(2)
    coef = TR.first_order_3d(q.p, TR.lattice_feq_3d(d3.Expansion3(q)))["eta"]
    L = 192
    x = np.arange(L)
    s = np.sin(2 * np.pi * x / L)
    one = np.ones((3, 3, L))
    z = np.zeros((3, 3, L))
    lat = rl.Lattice3(L, 3, 3, tau=tau)
    lat.init(one, z, np.ascontiguousarray(1e-4 * s * one), z.copy(), one.copy())
    k = 2 * np.pi / (L / 3.0)
    pred = coef * (tau - 0.5) * k * k / 4.0
    ts, a = [], []
    every = max(1, int(0.02 / pred))
    for t in range(every, int(1.0 / pred), every):
        lat.step(every)
        uy = lat.moments()["uy"].mean(axis=(0, 1))
        ts.append(t)
        a.append(np.sum(uy * s) / np.sum(s * s))
    assert lat.sync_status()[0] == 0
    lat.close()
    sl = slice(len(ts) // 5, None)
    rate = -np.polyfit(np.array(ts)[sl], np.log(np.array(a)[sl]), 1)[0]
    assert abs(rate / pred - 1) < 0.02, (rate, pred)


def test_fp32_taylor_green_run_conserves_within_the_rounding_bound(rl):
    """FP32 storage (g = f - f_ref, f_ref = w_i / 2 at n = T = 1 at rest), the
    Taylor-Green flow of the FP64 test for 500 steps: each step rounds the
    stored g to FP32 and forms f^eq from FP32 tables, so a sum of c_i g_i
    moves by at most about 2 * 2^-24 * sum |c_i g_i| per step (the flow only
    decays, so the start bounds every step)."""
    L, nz, steps = 64, 4, 500
    lat = rl.Lattice3(L, L, nz, tau=0.8, precision="fp32")
    lat.init(*[np.ascontiguousarray(a) for a in inputs.taylor_green3(L, nz, u0=0.2)])
    p, w = lat.p, lat.w

    def sums():
        f = lat.populations().reshape(lat.Q, -1)
        g = f - 0.5 * w[:, None]
        c = [p[:, 0]] + [p[:, 0] * p[:, a] for a in range(4)]
        return [float(np.sum(ci @ f)) for ci in c], [float(np.sum(np.abs(ci) @ np.abs(g))) for ci in c]

    t0, g0 = sums()
    lat.step(steps)
    t1, _ = sums()
    assert lat.sync_status()[0] == 0
    for a in range(5):
        assert abs(t1[a] - t0[a]) <= 2 * steps * 2.0 ** -24 * g0[a], (a, t1[a] - t0[a], g0[a])
    lat.close()


def test_order3_rejects_sides_below_the_halo(rl):
    with pytest.raises(rl.RLBMError):
        rl.Lattice3(8, 8, 5, order=3)


@pytest.mark.parametrize("tau", [0.6, 0.8, 1.0])
def test_order3_taylor_green_decay_gives_the_printed_viscosity(rl, tau):
    """Sec. 7.1, Table 2, zeta = 0: the Taylor-Green vortex in the (3+1)-d
    solver with the order-3 table (L^2 x 6 cells, u0 = 0.01; a population
    moves sqrt(41) cells per step at c, so dx = 1/sqrt(41) and k =
    2 pi sqrt(41) / L per axis).  The vortex decays at 2 eta k^2 / (eps + P),
    eps + P = 4 P; f = eta / (P (tau - 1/2)) measured from the decay rate
    agrees with the printed 0.8002 within 1 % and with the table's own
    first-order coefficient along the xy diagonals (0.8024) within 1 %."""
    import json
    import os
    from oracle import transport as TR
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "tg3d_f_zeta0.json")))
    printed = g["f"][g["tau"].index(tau)]
    q = d3.massless_quadrature_3d(3)
    c, s_ = np.cos(np.pi / 4), np.sin(np.pi / 4)
    pr = q.p.copy()
    pr[:, 1], pr[:, 2] = c * q.p[:, 1] - s_ * q.p[:, 2], s_ * q.p[:, 1] + c * q.p[:, 2]
    qr = d3.Quadrature3(q.n, pr, q.w)
    diag = TR.first_order_3d(qr.p, TR.lattice_feq_3d(d3.Expansion3(qr, order=3)))["eta"]
    L, nz, u0 = 192, 6, 0.01
    n, ux, uy, uz, T = inputs.taylor_green3(L, nz, u0=u0)
    px, py = ux / u0, uy / u0
    lat = rl.Lattice3(L, L, nz, tau=tau, order=3)
    lat.init(n, ux, uy, uz, T)
    k = 2 * np.pi * np.sqrt(41.0) / L
    guess = 2 * diag * (tau - 0.5) * k * k / 4.0
    every = max(1, int(0.05 / guess))
    ts, amps = [], []
    for t in range(every, int(1.5 / guess), every):
        lat.step(every)
        m = lat.moments()
        ts.append(t)
        amps.append(float(np.sum(m["ux"] * px + m["uy"] * py) / np.sum(px * px + py * py)))
    assert lat.sync_status()[0] == 0
    lat.close()
    sl = slice(len(ts) // 5, None)
    rate = -np.polyfit(np.array(ts)[sl], np.log(np.array(amps)[sl]), 1)[0]
    f = rate * 4.0 / (2 * k * k * (tau - 0.5))
    assert abs(f / printed - 1) < 0.01, (f, printed)
    assert abs(f / diag - 1) < 0.01, (f, diag)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_order3_full_size_equals_the_tiled_small_run(rl, precision):
    """192^3 cells with the order-3 table (288 planes of 8.7 M elements, more
    than 2^31 elements in all: the 64-bit plane offsets), a flow periodic in
    z with period 6 (a random 192 x 192 x 6 field tiled 32 times): each
    cell's update depends only on the populations it pulls, so after three
    steps every field equals, bit for bit, the 192 x 192 x 6 run tiled."""
    L, p, steps = 192, 6, 3
    small = inputs.random_smooth3(L, L, p, seed=11, umax=0.2)
    a = rl.Lattice3(L, L, p, tau=0.9, precision=precision, order=3)
    a.init(*[np.ascontiguousarray(f) for f in small])
    a.step(steps)
    ms = a.moments()
    a.close()
    b = rl.Lattice3(L, L, L, tau=0.9, precision=precision, order=3)
    b.init(*[np.ascontiguousarray(np.tile(f, (L // p, 1, 1))) for f in small])
    b.step(steps)
    mb = b.moments()
    assert b.sync_status()[0] == 0
    b.close()
    for k in ("n", "ux", "uy", "uz", "T"):
        assert np.array_equal(mb[k], np.tile(ms[k], (L // p, 1, 1))), k
