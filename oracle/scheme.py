"""The RLBM time step, FP64 CPU (oracle; test infrastructure only).

State convention.  The oracle holds the post-collision populations f*(t)
(shape (Q, ny, nx), population order of the quadrature).  One step is
    f(t+1)  = S f*(t)              streaming, Eq. discrete-rbe (left side)
    f*(t+1) = C(f(t+1))            steps 1-8 of Sec. 6.2 (right side)
Initialisation (Sec. 6.2, first paragraph): f(0) = f^eq(n0, U0, T0) and
f*(0) = f(0), since the collision of an exact equilibrium is the identity
(moments up to order N are recovered exactly by the quadrature).
``fields`` of time t are the Landau-frame quantities of the streamed f(t),
i.e. the ones the algorithm computes in steps 1-4 at time t.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import physics
from .lattice import Expansion, Quadrature

ETA = physics.ETA


# --------------------------------------------------------------------------
# Streaming
# --------------------------------------------------------------------------


def stream_onlattice(fs, shifts, boundary="periodic"):
    """f_i(x) = f*_i(x - n_i) (Eq. discrete-rbe: population i moves by
    v_i dt = n_i lattice sites per step, Sec. 6.1).

    boundary ``periodic``: wrap in x and y.  ``freeflow_x``: zero-gradient
    ends in x -- the source index x - n_ix is clamped into [0, nx-1]; y stays
    periodic.  (Reading: the paper's Sod runs use a mirror-periodic domain;
    clamping is this library's free-flow end.)"""
    Q, ny, nx = fs.shape
    out = np.empty_like(fs)
    ys = np.arange(ny)
    xs = np.arange(nx)
    for i in range(Q):
        sx, sy = int(shifts[i, 0]), int(shifts[i, 1])
        yy = (ys - sy) % ny
        if boundary == "periodic":
            xx = (xs - sx) % nx
        elif boundary in ("freeflow_x", "eqwall_x"):
            xx = np.clip(xs - sx, 0, nx - 1)
        else:
            raise ValueError(boundary)
        out[i] = fs[i][np.ix_(yy, xx)]
    return out


def bilinear_taps(disp):
    """Pull taps of the off-lattice scheme for displacement ``disp`` (2,) in
    cells: source point x - disp, o = floor(-disp), phi = -disp - o; taps at
    x + o + (a, b), a, b in {0, 1}, weights (1-|a-phi_x|)(1-|b-phi_y|).
    Reading (not in the paper, whose streaming is on-lattice only): bilinear
    interpolation of the post-collision field at the departure point."""
    src = -np.asarray(disp, dtype=np.float64)
    # a displacement within 1e-12 of a whole number of cells is that number
    # (lambda v_i is computed in floating point; lambda = ||n_i|| must give
    # exactly the on-lattice shift)
    src = np.where(np.abs(src - np.round(src)) < 1e-12, np.round(src), src)
    o = np.floor(src)
    phi = src - o
    taps = []
    for a in (0, 1):
        for b in (0, 1):
            wgt = (1.0 - abs(a - phi[0])) * (1.0 - abs(b - phi[1]))
            taps.append((int(o[0]) + a, int(o[1]) + b, wgt))
    return taps


def stream_bilinear(fs, disp, boundary="periodic"):
    """f_i(x) = sum_ab W_ab f*_i(x + o_i + (a, b)), disp_i = lambda v_i."""
    Q, ny, nx = fs.shape
    out = np.zeros_like(fs)
    ys = np.arange(ny)
    xs = np.arange(nx)
    for i in range(Q):
        for (ox, oy, wgt) in bilinear_taps(disp[i]):
            if wgt == 0.0:
                continue
            yy = (ys + oy) % ny
            if boundary == "periodic":
                xx = (xs + ox) % nx
            else:
                xx = np.clip(xs + ox, 0, nx - 1)
            out[i] += wgt * fs[i][np.ix_(yy, xx)]
    return out


# --------------------------------------------------------------------------
# Steps 1-8 of Sec. 6.2
# --------------------------------------------------------------------------


def moments(f, p):
    """Step 1: N^a = sum_i f_i p_i^a, T^{ab} = sum_i f_i p_i^a p_i^b."""
    N = np.tensordot(p.T, f, axes=1)                                  # (3, ny, nx)
    T = np.einsum("ia,ib,i...->ab...", p, p, f)                       # (3, 3, ny, nx)
    return N, T


@dataclass
class Fields:
    n: np.ndarray
    U: np.ndarray      # (3, ...) contravariant four-velocity
    T: np.ndarray
    eps: np.ndarray
    N: np.ndarray      # (3, ...)
    Tab: np.ndarray    # (3, 3, ...)
    ok: np.ndarray

    @property
    def ux(self):
        return self.U[1] / self.U[0]

    @property
    def uy(self):
        return self.U[2] / self.U[0]


def macroscopic(f, quad: Quadrature, d_eos=2):
    """Steps 1-4: moments, Landau eigen-solve, n = U_a N^a, T from the EOS."""
    N, Tab = moments(f, quad.p)
    eps, U, n, ok = physics.landau(N, Tab)
    T = physics.temperature_from_energy(eps / n, quad.m, d_eos)
    return Fields(n, U, T, eps, N, Tab, ok)


def relaxation_factor(U, tau, p):
    """Step 8: Omega_i = p_i^mu U_mu / (p_i^0 tau) (Delta t = 1)."""
    pU = p[:, 0, None, None] * U[0] - p[:, 1, None, None] * U[1] - p[:, 2, None, None] * U[2]
    return pU / (p[:, 0, None, None] * tau)


def tau_from_eta_over_s(T, eta_over_s, kappa, d=2):
    """Step 7 with eta/s fixed.  Reading: massless d = 2, eta = (3/4) P tau
    (App. C), s = (d + 1) n (the BAMPS entropy form without its 3-d log
    term), so tau = (eta/s)(d + 2) kappa / T with kappa = hbar/(k_B T0 dt)."""
    return eta_over_s * (d + 2) * kappa / T


def forcing_term(feq, fl, quad: Quadrature, g):
    """Step 6, scheme B of Sec. 4.4 (Delta t = 1): the external-force term of
    Eq. rbe-rta-lattice-friendly, -(m K^a / p^0) df/dp^a, with df/dp^a taken
    from the Maxwell-Juttner derivative -(U_a / T) f^eq, for a gravity-like
    Minkowski force K = (g.p, p^0 g) (K^a p_a = 0):
        F_i = (m / T) f^eq_i (K^a U_a) / p^0_i = (m / T) f^eq_i (U^0 g.v_i - g.U).
    Reading: the sign follows the continuous equation, so that the fluid is
    pushed along g (the printed discrete equation adds F^ext with the
    opposite sign convention).  Massless particles (m = 0) feel no force."""
    gx, gy = g
    v = quad.velocity()
    gv = gx * v[:, 0, None, None] + gy * v[:, 1, None, None]
    gU = gx * fl.U[1] + gy * fl.U[2]
    return (quad.m / fl.T) * feq * (fl.U[0] * gv - gU)


def collide(f, quad: Quadrature, exp: Expansion, tau, g=None, eqwall=False, wall_T=(0.0, 0.0)):
    """Steps 1-8: returns f*(x) and the fields of f.  g: optional gravity-like
    force (gx, gy), added as forcing_term.  eqwall: equilibrium walls at the
    first and last column (reading of the no-slip walls of Sec. 8.1: the
    post-collision populations there are the equilibrium at zero flow speed,
    f^eq(n, U = (1, 0, 0), T), with the cell's own n and T, or with the
    prescribed wall temperature wall_T[side] > 0 -- the heated plates of the
    thermal-conductivity runs of Sec. 7.2, whose density the paper takes from
    the neighbouring points; reading: the cell's own n)."""
    fl = macroscopic(f, quad)
    feq = exp.feq(fl.n, fl.U, fl.T)                                    # step 5
    if isinstance(tau, tuple):                                          # step 7
        tau = tau_from_eta_over_s(fl.T, *tau)
    omega = relaxation_factor(fl.U, tau, quad.p)                        # step 8
    fs = (1.0 - omega) * f + omega * feq
    if g is not None:
        fs = fs + forcing_term(feq, fl, quad, g)
    if eqwall:
        for side, col in enumerate((0, f.shape[2] - 1)):
            n, T = fl.n[:, col], fl.T[:, col]
            if wall_T[side] > 0:
                T = np.full_like(T, wall_T[side])
            rest = np.zeros((3,) + n.shape)
            rest[0] = 1.0
            fs[:, :, col] = exp.feq(n, rest, T)
    # a cell without a physical Landau frame (no timelike eigenvector, n or T
    # not positive, non-finite moments) is left unrelaxed (reading of the
    # states the paper does not discuss)
    bad = ~physical(fl)
    if np.any(bad):
        fs = np.where(bad[None], f, fs)
    return fs, fl


def physical(fl):
    """Cells whose Landau frame exists: a timelike eigenvector with a real
    positive eigenvalue, n > 0, T > 0, all finite."""
    with np.errstate(invalid="ignore"):
        return fl.ok & (fl.n > 0) & (fl.T > 0) & np.isfinite(fl.n) & np.isfinite(fl.T)


class Simulation:
    """Time integration with the state convention of the module docstring."""

    def __init__(self, quad: Quadrature, exp: Expansion, nx, ny, tau=1.0,
                 boundary="periodic", stream="onlattice", lam=None, g=None, wall_T=(0.0, 0.0)):
        self.quad, self.exp = quad, exp
        self.g = g                           # optional gravity-like force (gx, gy)
        self.wall_T = wall_T                 # equilibrium-wall temperatures (0: own T)
        self.nx, self.ny = nx, ny
        self.tau = tau                       # scalar, (ny, nx) array or (eta/s, kappa)
        self.boundary = boundary
        self.stream_mode = stream
        if stream == "onlattice":
            self.shifts = quad.n
        else:
            if lam is None:
                raise ValueError("bilinear streaming needs lambda")
            self.disp = lam * quad.velocity()
        self.fs = None
        self.fields = None
        self.t = 0

    def init(self, n, ux, uy, T):
        U = physics.four_velocity(ux, uy)
        f0 = self.exp.feq(n, U, T)
        self.fs = f0
        self.fields = macroscopic(f0, self.quad)
        self.t = 0

    def stream(self, fs):
        if self.stream_mode == "onlattice":
            return stream_onlattice(fs, self.shifts, self.boundary)
        return stream_bilinear(fs, self.disp, self.boundary)

    def step(self, nsteps=1):
        for _ in range(nsteps):
            f = self.stream(self.fs)
            self.fs, self.fields = collide(f, self.quad, self.exp, self.tau, self.g,
                                           self.boundary == "eqwall_x", self.wall_T)
            self.t += 1
        return self.fs
