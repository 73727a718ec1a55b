"""Hand-written adjoint of the RLBM step against central finite differences
of the FP64 oracle, against itself across checkpoint intervals, FP32 against
FP64, and through torch.autograd."""
import numpy as np
import pytest

from paper_1909_04502_gb300 import inputs
from oracle import lattice as OL
from oracle import scheme as OS
from oracle import physics as OP

pytestmark = pytest.mark.gpu

NX, NY, T = 16, 12, 6


@pytest.fixture(scope="module")
def rl():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_04502_gb300 import build, rlbm
    build.build()
    return rlbm


def _setup(seed=31, nx=NX, ny=NY):
    rng = np.random.default_rng(seed)
    n, ux, uy, Tf = [np.ascontiguousarray(a) for a in inputs.random_smooth(nx, ny, seed=seed, umax=0.2)]
    tau = np.ascontiguousarray(rng.uniform(0.7, 1.3, (ny, nx)))
    uxt = np.ascontiguousarray(0.05 * rng.standard_normal((ny, nx)))
    uyt = np.ascontiguousarray(0.05 * rng.standard_normal((ny, nx)))
    return n, ux, uy, Tf, tau, uxt, uyt


def _oracle_loss(n, ux, uy, Tf, tau, uxt, uyt, steps=T, stream="onlattice", lam=None):
    q = OL.massless_quadrature(2)
    sim = OS.Simulation(q, OL.Expansion(q), n.shape[1], n.shape[0], tau=tau, stream=stream, lam=lam)
    sim.init(n, ux, uy, Tf)
    sim.step(steps)
    return 0.5 * np.sum((sim.fields.ux - uxt) ** 2 + (sim.fields.uy - uyt) ** 2)


def _adjoint(rl, precision, K, data, stream="onlattice", lam=0.0, steps=T):
    n, ux, uy, Tf, tau, uxt, uyt = data
    lat = rl.Lattice(n.shape[1], n.shape[0], tau_mode="field", precision=precision, stream=stream, lam=lam)
    lat.set_tau_field(tau)
    adj = rl.Adjoint(lat, steps, K)
    adj.forward(n, ux, uy, Tf)
    res = adj.backward(uxt, uyt)
    assert lat.sync_status()[0] == 0
    adj.close()
    lat.close()
    return res


@pytest.mark.parametrize("stream,lam", [("onlattice", 0.0), ("bilinear", 1.0)])
def test_fp64_adjoint_matches_oracle_central_differences(rl, stream, lam):
    data = _setup()
    n, ux, uy, Tf, tau, uxt, uyt = data
    loss, gtau, gux, guy = _adjoint(rl, "fp64", 4, data, stream, lam)
    olam = lam if stream == "bilinear" else None
    L0 = _oracle_loss(n, ux, uy, Tf, tau, uxt, uyt, stream=stream, lam=olam)
    assert abs(loss - L0) < 1e-12 * abs(L0)
    rng = np.random.default_rng(5)
    h = 1e-4
    # directional derivative along a random tau perturbation
    d = rng.standard_normal(tau.shape)
    fd = (_oracle_loss(n, ux, uy, Tf, tau + h * d, uxt, uyt, stream=stream, lam=olam)
          - _oracle_loss(n, ux, uy, Tf, tau - h * d, uxt, uyt, stream=stream, lam=olam)) / (2 * h)
    ad = float(np.sum(gtau * d))
    assert abs(ad - fd) < 1e-6 * abs(fd), (ad, fd)
    # and along a random initial-velocity perturbation
    dx, dy = 0.1 * rng.standard_normal(ux.shape), 0.1 * rng.standard_normal(uy.shape)
    fd = (_oracle_loss(n, ux + h * dx, uy + h * dy, Tf, tau, uxt, uyt, stream=stream, lam=olam)
          - _oracle_loss(n, ux - h * dx, uy - h * dy, Tf, tau, uxt, uyt, stream=stream, lam=olam)) / (2 * h)
    ad = float(np.sum(gux * dx + guy * dy))
    assert abs(ad - fd) < 1e-6 * abs(fd), (ad, fd)


def test_fp64_adjoint_single_cell_sensitivities(rl):
    data = _setup(seed=44)
    n, ux, uy, Tf, tau, uxt, uyt = data
    _, gtau, gux, _ = _adjoint(rl, "fp64", 2, data)
    h = 1e-4
    for (j, i) in [(0, 0), (5, 9), (11, 15)]:
        tp, tm = tau.copy(), tau.copy()
        tp[j, i] += h
        tm[j, i] -= h
        fd = (_oracle_loss(n, ux, uy, Tf, tp, uxt, uyt) - _oracle_loss(n, ux, uy, Tf, tm, uxt, uyt)) / (2 * h)
        assert abs(gtau[j, i] - fd) < 1e-6 * np.abs(gtau).max(), (j, i, gtau[j, i], fd)
        up, um = ux.copy(), ux.copy()
        up[j, i] += h
        um[j, i] -= h
        fd = (_oracle_loss(n, up, uy, Tf, tau, uxt, uyt) - _oracle_loss(n, um, uy, Tf, tau, uxt, uyt)) / (2 * h)
        assert abs(gux[j, i] - fd) < 1e-6 * np.abs(gux).max(), (j, i, gux[j, i], fd)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_checkpoint_interval_does_not_change_the_gradient(rl, precision):
    """Recomputation is deterministic, so the gradient is bitwise the same for
    any checkpoint interval (FP32: the recompute also stores the cells'
    macroscopic states, which the adjoint steps read)."""
    data = _setup(seed=8)
    a = _adjoint(rl, precision, 1, data, steps=9)
    b = _adjoint(rl, precision, 4, data, steps=9)
    c = _adjoint(rl, precision, 9, data, steps=9)
    for x, y in ((a, b), (a, c)):
        assert x[0] == y[0]
        for k in (1, 2, 3):
            assert np.array_equal(x[k], y[k])


def test_fp32_adjoint_against_fp64_and_differences(rl):
    data = _setup(seed=12, nx=40, ny=32)
    n, ux, uy, Tf, tau, uxt, uyt = data
    l32, g32, gx32, gy32 = _adjoint(rl, "fp32", 3, data, steps=20)
    l64, g64, gx64, gy64 = _adjoint(rl, "fp64", 3, data, steps=20)
    assert abs(l32 - l64) < 1e-5 * l64
    assert np.abs(g32 - g64).max() < 1e-4 * np.abs(g64).max()
    assert np.abs(gx32 - gx64).max() < 1e-4 * np.abs(gx64).max()
    rng = np.random.default_rng(2)
    d = rng.standard_normal(tau.shape)
    h = 1e-4
    fd = (_oracle_loss(n, ux, uy, Tf, tau + h * d, uxt, uyt, steps=20)
          - _oracle_loss(n, ux, uy, Tf, tau - h * d, uxt, uyt, steps=20)) / (2 * h)
    assert abs(float(np.sum(g32 * d)) - fd) < 1e-4 * abs(fd)


def test_torch_autograd_function(rl):
    import torch
    from paper_1909_04502_gb300.autograd import CalibrationRun, shear_loss
    data = _setup(seed=3)
    n, ux, uy, Tf, tau, uxt, uyt = [torch.tensor(a, dtype=torch.float64, device="cuda") for a in data]
    run = CalibrationRun(NX, NY, T, checkpoint_every=3, precision="fp64")
    tau_p = tau.clone().requires_grad_(True)
    ux_p = ux.clone().requires_grad_(True)
    uy_p = uy.clone().requires_grad_(True)
    loss = shear_loss(run, tau_p, ux_p, uy_p, n, Tf, uxt, uyt)
    loss.backward()
    L_ref, g_ref, gx_ref, gy_ref = _adjoint(rl, "fp64", 3, data)
    assert abs(loss.item() - L_ref) < 1e-12 * L_ref
    assert np.array_equal(tau_p.grad.cpu().numpy(), g_ref)
    assert np.array_equal(ux_p.grad.cpu().numpy(), gx_ref)
    run.close()


def test_calibration_full_size_gradient(rl):
    """The 512^2 calibration run (massless shear flow u_y = 0.05 sin(2 pi x/L),
    2000 steps, checkpoints every 100, hidden smooth tau): the FP32 adjoint's
    tau gradient within 1e-4 of the FP64 adjoint's, and the FP64 directional
    derivative within 1e-4 of central differences (h = 1e-4, relative on
    tau) of the FP64 forward run (the forward and adjoint kernels share no
    derivative code; the oracle is too slow for 5e8 cell updates)."""
    L, nsteps, K = 512, 2000, 100
    n, ux, uy, Tf = [np.ascontiguousarray(a) for a in inputs.shear_wave(L, L, amp=0.05)]
    hidden = np.ascontiguousarray(inputs.smooth_tau(L, L))
    tau = np.ones((L, L))

    def run(precision, tau_field, target=None):
        lat = rl.Lattice(L, L, tau_mode="field", precision=precision)
        lat.set_tau_field(np.ascontiguousarray(tau_field))
        if target is None:
            lat.init(n, ux, uy, Tf)
            lat.step(nsteps)
            m = lat.moments()
            assert lat.sync_status()[0] == 0
            lat.close()
            return m
        adj = rl.Adjoint(lat, nsteps, K)
        adj.forward(n, ux, uy, Tf)
        res = adj.backward(*target)
        assert lat.sync_status()[0] == 0
        adj.close()
        lat.close()
        return res

    mt = run("fp64", hidden)
    target = (np.ascontiguousarray(mt["ux"]), np.ascontiguousarray(mt["uy"]))
    l64, g64, _, _ = run("fp64", tau, target)
    l32, g32, _, _ = run("fp32", tau, target)
    # the loss is a residual: with |du| <= 1e-5 * 0.05 per cell (the FP32
    # forward's parity bar on velocities), |l32 - l64| <= 2 sqrt(2 l64 N) |du|
    bound = 2 * np.sqrt(2 * l64 * L * L) * 1e-5 * 0.05
    assert abs(l32 - l64) < bound, (l32, l64, bound)
    g_err = float(np.abs(g32 - g64).max() / np.abs(g64).max())
    rng = np.random.default_rng(7)
    d = np.ascontiguousarray(np.cos(2 * np.pi * rng.integers(1, 4) * np.arange(L) / L)[None, :]
                             * np.ones((L, 1)) * tau)
    h = 1e-4

    def loss(tf):
        m = run("fp64", tf)
        return 0.5 * np.sum((m["ux"] - target[0]) ** 2 + (m["uy"] - target[1]) ** 2)

    fd = (loss(tau + h * d) - loss(tau - h * d)) / (2 * h)
    ad = float(np.sum(g64 * d))
    ad32 = float(np.sum(g32 * d))
    info = dict(fd=fd, ad64=ad, ad32=ad32, g32_vs_g64=g_err, l32=l32, l64=l64)
    assert abs(ad - fd) < 1e-4 * abs(fd), info
    assert abs(ad32 - fd) < 1e-4 * abs(fd), info
    assert g_err < 1e-3, info


def test_single_adjoint_step_entry_point(rl):
    """rlbm_adjoint_step against central differences of one forward step
    (FP64, on-lattice, periodic).  With f(t) = S x and x(t) = C(f(t)), and
    L(x) = <a_next, S C(S x)>, the step returns a = C'^T S^T a_next, so
    dL/dx . dx = <S^T a, dx> = <a, S dx>.  S is the periodic pull, applied on
    the host with the oracle's streaming."""
    import ctypes
    import torch
    nx, ny, tau = 24, 16, 0.9
    fields = [np.ascontiguousarray(a) for a in inputs.random_smooth(nx, ny, seed=17, umax=0.2)]
    mk = lambda: rl.Lattice(nx, ny, precision="fp64", tau=tau)
    base = mk()
    base.init(*fields)
    base.step(2)
    x = base.populations()
    shifts = base.n
    rng = np.random.default_rng(3)
    a_next = rng.standard_normal(x.shape) * 1e-2
    dx = rng.standard_normal(x.shape) * np.abs(x).max() * 1e-2
    hx, ha, ho = mk(), mk(), mk()
    hx.set_populations(x)
    ha.set_populations(a_next)
    ho.set_populations(np.zeros_like(x))
    gt = torch.zeros((ny, nx), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    rc = rl.lib().rlbm_adjoint_step(hx.h, hx.buffers()[0], ha.buffers()[0], ho.buffers()[0], gt.data_ptr())
    assert rc == 0
    torch.cuda.synchronize()
    a = ho.populations()

    def L(xs):
        hf = mk()
        hf.set_populations(xs)
        hf.step(1)
        y = hf.populations()
        hf.close()
        return float(np.sum(a_next * OS.stream_onlattice(y, shifts, "periodic")))

    h = 1e-4
    fd = (L(x + h * dx) - L(x - h * dx)) / (2 * h)
    ad = float(np.sum(a * OS.stream_onlattice(dx, shifts, "periodic")))
    assert abs(ad - fd) < 1e-6 * abs(fd), (ad, fd)
    for lat in (base, hx, ha, ho):
        lat.close()
