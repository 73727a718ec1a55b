// Hand-written adjoint (vector-Jacobian product) of the fused RLBM step.
//
// Forward: x(t+1) = C(S x(t); tau) with S the streaming (linear) and C the
// per-cell collision of Sec. 6.2 (steps 1-8; Eq. discrete-rbe).  For a loss
// L on the fields of f(T) = S x(T-1), the adjoint populations
//   a(t) = dL/df(t),  lambda(t) = dL/dx(t) = S^T a(t+1),
// obey a(t) = C'(f(t))^T lambda(t); the tau gradient accumulates
// dC/dtau^T lambda(t) and the initial state x(0) = f^eq(n0, U(u0), T0) gives
// dL/du0.  S^T of the pull is a pull with reversed offsets (Tables.roff), so
// every adjoint kernel is again a fused gather-compute-store over cells.
//
// The per-cell VJP follows the forward algorithm backwards: relaxation
// (Omega_i), equilibrium f^eq = H dM(n, U, T), the EOS (T of eps/n), n = U.N,
// the normalisation U = v/|v|, the eigenvector v(eps, T^ab), and the
// eigenvalue through the implicit function p(eps; T^ab) = det(A - eps I) = 0.
// Periodic boundaries, order 2, constant or per-cell tau.
#include <cuda_runtime.h>

#include "../../include/rlbm.h"
#include "dispatch.h"
#include "handle.h"
#include "step_impl.cuh"

namespace rlbm {

// Reference scalars and tau in the working precision: the FP32 path reads
// the FP32 copies, since a conversion from double runs on the FP64 pipe.
template <typename S>
__device__ __forceinline__ void ref_scalars(const Scalars& sc, S& T00, S& Tii, S& N0, S& m) {
  if constexpr (sizeof(S) == 4) { T00 = sc.f_T00_ref; Tii = sc.f_Tii_ref; N0 = sc.f_n_ref; m = sc.f_m; }
  else { T00 = (S)sc.T00_ref; Tii = (S)sc.Tii_ref; N0 = (S)sc.N0_ref; m = (S)sc.m; }
}
template <typename S>
__device__ __forceinline__ S const_tau(const Scalars& sc) {
  if constexpr (sizeof(S) == 4) return sc.f_tau;
  else return sc.tau;
}
template <typename S>
__device__ __forceinline__ S inv_sqrt(S x) {
  if constexpr (sizeof(S) == 4) return rsqrtf(x);
  else return S(1) / sqrt(x);
}

// Transposed streaming: lambda_i(x) = (S^T a)_i(x).
template <typename S, int QT, bool EX, int MODE>
__device__ __forceinline__ void gather_rev(const Tables<S>& tb, const Scalars& s, const S* __restrict__ a,
                                           long long si, S (&lam)[QT]) {
  const S* __restrict__ base = a + si;
  const int Qn = EX ? QT : s.Q;
#pragma unroll
  for (int i = 0; i < QT; ++i) {
    lam[i] = S(0);
    if (i < Qn) {
      const int o = tb.roff[i];
      if constexpr (MODE == kOnLattice) {
        lam[i] = __ldg(base + o);
      } else {
        S v = tb.bw[i][3] * __ldg(base + o);
        v = fma(tb.bw[i][2], __ldg(base + o + 1), v);
        v = fma(tb.bw[i][1], __ldg(base + o + s.pitch), v);
        v = fma(tb.bw[i][0], __ldg(base + o + s.pitch + 1), v);
        lam[i] = v;
      }
    }
  }
}

// Moment-vector derivatives for order 2 (basis of setup.h, K = 9):
// dM0 = n/(m+T) - ref, dM1 = n U0 - ref, dM2 = n Ux, dM3 = n Uy,
// dM4 = n r2 U0 Ux, dM5 = n r2 U0 Uy, dM6 = n r2 Ux^2 + n T - ref,
// dM7 = n r2 Ux Uy, dM8 = n r2 Uy^2 + n T - ref, r2 = (m^2 + 3mT + 3T^2)/(m+T).
// Given h_k = ds/d(dM_k), accumulate ds/dn, ds/dT, ds/dU.
template <typename S>
__device__ __forceinline__ void dM_vjp(const S (&h)[9], S n, S T, S U0, S Ux, S Uy, S m, S& gn, S& gT,
                                       S& gU0, S& gUx, S& gUy) {
  const S mT = m + T;
  const S imT = qdiv(S(1), mT);
  const S r2 = (m * m + S(3) * m * T + S(3) * T * T) * imT;
  const S dr2 = (S(3) * m + S(6) * T) * imT - r2 * imT;
  const S A = h[4] * U0 * Ux + h[5] * U0 * Uy + h[6] * Ux * Ux + h[7] * Ux * Uy + h[8] * Uy * Uy;
  gn += h[0] * imT + h[1] * U0 + h[2] * Ux + h[3] * Uy + r2 * A + (h[6] + h[8]) * T;
  gT += -h[0] * n * imT * imT + n * dr2 * A + (h[6] + h[8]) * n;
  const S nr2 = n * r2;
  gU0 += h[1] * n + nr2 * (h[4] * Ux + h[5] * Uy);
  gUx += h[2] * n + nr2 * (h[4] * U0 + S(2) * h[6] * Ux + h[7] * Uy);
  gUy += h[3] * n + nr2 * (h[5] * U0 + h[7] * Ux + S(2) * h[8] * Uy);
}

// ds/dmoments from ds/d(eps, U) through the Landau eigen-solve (Sec. 4).
// mm: the 9 stored-population moment sums; the totals add the reference.
template <typename S>
__device__ __forceinline__ void landau_vjp(const Scalars& sc, const S (&mm)[9], S eps, S gE, S gU0, S gUx,
                                           S gUy, S (&gm)[9]) {
  S T00r, Tiir, N0r, mr;
  ref_scalars<S>(sc, T00r, Tiir, N0r, mr);
  const S T00 = T00r + mm[3], s = mm[4], t = mm[5];
  const S Txx = Tiir + mm[6], r = mm[7], Tyy = Tiir + mm[8];
  // the reference parts must be added in the working precision
  const S a = T00 - eps, b = Txx + eps, c = Tyy + eps;
  const S D = b * c - r * r;
  const S vx = s * c - r * t, vy = t * b - r * s;
  const S nu2 = D * D - vx * vx - vy * vy;
  const S inu = inv_sqrt(nu2);
  // U = v / nu, nu^2 = v0^2 - vx^2 - vy^2
  const S gdot = (gU0 * D + gUx * vx + gUy * vy) * inu * inu * inu;
  const S gv0 = gU0 * inu - gdot * D;
  const S gvx = gUx * inu + gdot * vx;
  const S gvy = gUy * inu + gdot * vy;
  // eigenvalue: p(eps) = a D - s vx - t vy = 0
  const S dp = -D + a * (b + c) - s * s - t * t;
  const S gEt = gE + gv0 * (b + c) + gvx * s + gvy * t;
  const S k = qdiv(gEt, dp);
  gm[3] = -k * D;                                                              // T00
  gm[6] = gv0 * c + gvy * t - k * (a * c - t * t);                             // Txx
  gm[8] = gv0 * b + gvx * s - k * (a * b - s * s);                             // Tyy
  gm[7] = -S(2) * r * gv0 - t * gvx - s * gvy - k * (S(2) * (s * t - a * r));  // Txy
  gm[4] = c * gvx - r * gvy - k * (S(2) * (r * t - s * c));                    // T0x
  gm[5] = -r * gvx + b * gvy - k * (S(2) * (r * s - t * b));                   // T0y
}

// Orbit-symmetric transposes for the built-in massless stencils (member
// order of moments_sym / feq_orbit8 in step_impl.cuh).
// h += sum over the eight members m of r_m * (row of member m), the rows being
// the first row h0 with the members' column signs and swaps.
template <typename S>
__device__ __forceinline__ void hrow_accum8(const S (&h0)[kMaxK], const S (&r)[8], S (&h)[9]) {
  const S u0 = r[0] + r[1], u1 = r[0] - r[1], u2 = r[2] + r[3], u3 = r[2] - r[3];
  const S v0 = r[4] + r[5], v1 = r[4] - r[5], v2 = r[6] + r[7], v3 = r[6] - r[7];
  // sums weighted by 1, sx, sy, sx sy over each sign quartet
  const S A[4] = {u0 + u2, u1 + u3, u0 - u2, u1 - u3};
  const S B[4] = {v0 + v2, v1 + v3, v0 - v2, v1 - v3};
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int cls = mono_ax(k) + 2 * mono_ay(k);
    h[k] = fma(h0[k], A[cls], h[k]);
    h[k] = fma(h0[mono_swap(k)], B[cls], h[k]);
  }
}

template <typename S>
__device__ __forceinline__ void hrow_accum4(const S (&h0)[kMaxK], const S (&r)[4], S (&h)[9]) {
  // members (p,0), (-p,0), (0,p), (0,-p); the row of (p,0) has no py-odd entries
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    if (!mono_ay(k)) h[k] = fma(h0[k], mono_ax(k) ? r[0] - r[1] : r[0] + r[1], h[k]);
    if (!mono_ax(k)) h[k] = fma(h0[mono_swap(k)], mono_ay(k) ? r[2] - r[3] : r[2] + r[3], h[k]);
  }
}

// a_i += sum_k gm_k c_ik for the members of the orbits (transposed moments).
template <typename S, int QT>
__device__ __forceinline__ void moments_sym_transpose(const Tables<S>& tb, const S (&gm)[9], S (&a)[QT]) {
  using O = Orbits<QT>;
  static_assert(O::nd == 0 && O::n1 == 0, "adjoint symmetric path: massless stencils only");
#pragma unroll
  for (int o = 0; o < O::n8; ++o) {
    const int i = 8 * o;
    const S (&c)[9] = tb.c[i];   // p0, a, b, p0^2, p0 a, p0 b, a^2, a b, b^2 of the base (a, b)
    const S E = fma(gm[0], c[0], fma(gm[3], c[3], fma(gm[6], c[6], gm[8] * c[8])));
    const S X = fma(gm[1], c[1], gm[4] * c[4]), Y = fma(gm[2], c[2], gm[5] * c[5]), XY = gm[7] * c[7];
    const S Eb = fma(gm[0], c[0], fma(gm[3], c[3], fma(gm[6], c[8], gm[8] * c[6])));
    const S Xb = fma(gm[1], c[2], gm[4] * c[5]), Yb = fma(gm[2], c[1], gm[5] * c[4]);
    const S A = E + XY, B = E - XY, C = X + Y, D = X - Y;
    a[i] += A + C; a[i + 1] += B - D; a[i + 2] += B + D; a[i + 3] += A - C;
    const S Ab = Eb + XY, Bb = Eb - XY, Cb = Xb + Yb, Db = Xb - Yb;
    a[i + 4] += Ab + Cb; a[i + 5] += Bb - Db; a[i + 6] += Bb + Db; a[i + 7] += Ab - Cb;
  }
#pragma unroll
  for (int o = 0; o < O::n4; ++o) {
    const int i = 8 * O::n8 + 4 * o;
    const S (&c)[9] = tb.c[i];   // p0, p, 0, p0^2, p0 p, 0, p^2, 0, 0
    const S E = fma(gm[0], c[0], fma(gm[3], c[3], gm[6] * c[6]));
    const S Eb = fma(gm[0], c[0], fma(gm[3], c[3], gm[8] * c[6]));
    const S X = fma(gm[1], c[1], gm[4] * c[4]), Y = fma(gm[2], c[1], gm[5] * c[4]);
    a[i] += E + X; a[i + 1] += E - X; a[i + 2] += Eb + Y; a[i + 3] += Eb - Y;
  }
}

// Per-cell VJP of one collision.  g: f(t) (stored precision, shifted),
// lam: dL/dx(t).  Outputs a = dL/df(t) and the tau sensitivity.
// SYM: orbit-symmetric moments, equilibrium and their transposes.
// MIN (FP32 storage): the macroscopic state of the cell is read from mac
// (planes written by the recomputing forward step) instead of re-solving the
// Landau problem; a cell the forward step left unrelaxed (non-physical,
// n stored as NaN) has the identity as its collision, so a = lam there.
template <typename S, int QT, bool EX, bool SYM = false, bool MIN = false>
__device__ __forceinline__ void collide_vjp(const Tables<S>& tb, const Scalars& sc, const S (&g)[QT],
                                            const S (&lam)[QT], S tau, S (&a)[QT], S& gtau,
                                            unsigned long long* status, const float* __restrict__ mac = nullptr,
                                            int cell = 0) {
  const int Qn = EX ? QT : sc.Q;
  S mm[9];
  if constexpr (SYM) moments_sym<S, QT>(tb, g, mm);
  else moments9<S, QT, EX>(tb, sc.Q, g, mm);
  Macro M;
  S eps;
  if constexpr (MIN && sizeof(S) == 4) {
    const int nc = sc.ncell;
    M.fn = __ldg(mac + cell);
    M.fT = __ldg(mac + nc + cell);
    M.fU0 = __ldg(mac + 2 * nc + cell);
    M.fUx = __ldg(mac + 3 * nc + cell);
    M.fUy = __ldg(mac + 4 * nc + cell);
    M.fdn = __ldg(mac + 5 * nc + cell);
    M.fdT = __ldg(mac + 6 * nc + cell);
    eps = __ldg(mac + 7 * nc + cell);
    M.ok = !isnan(M.fn);
    if (!M.ok) {
#pragma unroll
      for (int i = 0; i < QT; ++i) a[i] = lam[i];
      gtau = S(0);
      return;
    }
  } else {
    M = landau<S, SYM ? (Orbits<QT>::massless ? 1 : 0) : -1>(sc, mm);
    if (!M.ok) {
      // the forward step left this cell unrelaxed: its collision is the identity
      atomicAdd(status, 1ULL);
#pragma unroll
      for (int i = 0; i < QT; ++i) a[i] = lam[i];
      gtau = S(0);
      return;
    }
    eps = (S)M.eps;
  }
  S T00r, Tiir, N0r, mr;
  ref_scalars<S>(sc, T00r, Tiir, N0r, mr);
  S dM[9];
  eq_moments_of<S, 9>(sc, M, dM);
  S n, T, U0, Ux, Uy;
  if constexpr (sizeof(S) == 4) { n = M.fn; T = M.fT; U0 = M.fU0; Ux = M.fUx; Uy = M.fUy; }
  else { n = M.n; T = M.T; U0 = M.U0; Ux = M.Ux; Uy = M.Uy; }
  const S inv_tau = qdiv(S(1), tau);
  S h[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) h[k] = S(0);
  S q0 = 0, qx = 0, qy = 0, sr = 0;
  // one population: returns ds/dfeq_i, accumulates the Omega and tau parts
  auto pop = [&](int i, S feq) {
    const S om = (U0 - Ux * tb.vx[i] - Uy * tb.vy[i]) * inv_tau;
    const S diff = feq - g[i];
    const S r = lam[i] * om;                 // ds/dfeq_i
    const S q = lam[i] * diff * inv_tau;     // ds/d(tau Omega_i)
    q0 += q;
    qx = fma(-q, tb.vx[i], qx);
    qy = fma(-q, tb.vy[i], qy);
    sr = fma(r, diff, sr);
    a[i] = lam[i] * (S(1) - om);
    return r;
  };
  if constexpr (SYM) {
    using O = Orbits<QT>;
#pragma unroll
    for (int o = 0; o < O::n8; ++o) {
      const int i0 = 8 * o;
      S f[8], r[8];
      feq_orbit8<S, 9>(tb.H[i0], dM, f);
#pragma unroll
      for (int m = 0; m < 8; ++m) r[m] = pop(i0 + m, f[m]);
      hrow_accum8<S>(tb.H[i0], r, h);
    }
#pragma unroll
    for (int o = 0; o < O::n4; ++o) {
      const int i0 = 8 * O::n8 + 4 * o;
      S f[4], r[4];
      feq_orbit4<S, 9>(tb.H[i0], dM, f);
#pragma unroll
      for (int m = 0; m < 4; ++m) r[m] = pop(i0 + m, f[m]);
      hrow_accum4<S>(tb.H[i0], r, h);
    }
  } else {
#pragma unroll
    for (int i = 0; i < QT; ++i) {
      if (i < Qn) {
        S feq = S(0);
#pragma unroll
        for (int k = 0; k < 9; ++k) feq = fma(tb.H[i][k], dM[k], feq);
        const S r = pop(i, feq);
#pragma unroll
        for (int k = 0; k < 9; ++k) h[k] = fma(r, tb.H[i][k], h[k]);
      }
    }
  }
  gtau = -sr * inv_tau;
  S gn = 0, gT = 0, gU0 = q0, gUx = qx, gUy = qy;
  dM_vjp<S>(h, n, T, U0, Ux, Uy, mr, gn, gT, gU0, gUx, gUy);
  // temperature from eps/n (d = 2 closed form)
  S gE;
  const S in_ = qdiv(S(1), n);
  if (sc.massless) {
    gE = S(0.5) * gT * in_;
    gn += -gT * T * in_;
  } else {
    const S m = mr, e = eps * in_;
    const S dTde = qdiv(T + m, S(4) * T + S(2) * m - e);
    gE = gT * dTde * in_;
    gn += -gT * dTde * e * in_;
  }
  // n = U0 N0 - Ux Nx - Uy Ny
  const S N0 = N0r + mm[0], Nx = mm[1], Ny = mm[2];
  gU0 += gn * N0;
  gUx -= gn * Nx;
  gUy -= gn * Ny;
  S gm[9];
  gm[0] = gn * U0;
  gm[1] = -gn * Ux;
  gm[2] = -gn * Uy;
  landau_vjp<S>(sc, mm, eps, gE, gU0, gUx, gUy, gm);
  if constexpr (SYM) {
    moments_sym_transpose<S, QT>(tb, gm, a);
  } else {
#pragma unroll
    for (int i = 0; i < QT; ++i) {
      if (i < Qn) {
        S acc = a[i];
#pragma unroll
        for (int k = 0; k < 9; ++k) acc = fma(gm[k], tb.c[i][k], acc);
        a[i] = acc;
      }
    }
  }
}

template <typename S>
struct AdjArgs {
  Scalars s;
  const S* xprev;        // x(t-1): f(t) = S x(t-1)
  const S* anext;        // a(t+1)
  S* aout;               // a(t)
  const S* tau_field;    // per-cell tau (tau_mode 1) or null
  double* gtau;          // accumulated dL/dtau per cell [ny][nx]
  unsigned long long* status;
  const float* macro = nullptr;   // macroscopic state of f(t) (FP32 storage), or null: recompute
};

template <typename S, int QT, bool EX, int MODE, bool SYM, bool MIN>
__global__ void __launch_bounds__(kThreads, (sizeof(S) == 4 ? 640 : 256) / kThreads) k_adj_step(const __grid_constant__ Tables<S> tb,
                                                       const __grid_constant__ AdjArgs<S> a) {
  const int x = blockIdx.x * kBX + threadIdx.x;
  const int y = blockIdx.y * kBY + threadIdx.y;
  if (x >= a.s.nx || y >= a.s.ny) return;
  const long long si = sidx(a.s, x, y);
  const int cell = y * a.s.nx + x;
  const int Qn = EX ? QT : a.s.Q;
  S g[QT], lam[QT], out[QT];
  gather<S, QT, EX, MODE>(tb, a.s, a.xprev, si, g);
  gather_rev<S, QT, EX, MODE>(tb, a.s, a.anext, si, lam);
  const S tau = (a.s.tau_mode == 1) ? a.tau_field[cell] : const_tau<S>(a.s);
  S gt;
  collide_vjp<S, QT, EX, SYM, MIN>(tb, a.s, g, lam, tau, out, gt, a.status, a.macro, cell);
  if constexpr (sizeof(S) == 4) a.gtau[cell] += f2d(gt);   // exact conversion on the integer pipe
  else a.gtau[cell] += gt;
  S* __restrict__ ob = a.aout + si;
#pragma unroll
  for (int i = 0; i < QT; ++i)
    if (i < Qn) ob[tb.pl[i]] = out[i];
  for_each_halo_image(a.s, x, y, [&](long long hi) {
    S* __restrict__ hb = a.aout + hi;
#pragma unroll
    for (int i = 0; i < QT; ++i)
      if (i < Qn) hb[tb.pl[i]] = out[i];
  });
}

// Loss L = 1/2 sum_x |u(x) - u_target(x)|^2 on the fields of f(T) = S x(T-1):
// writes a(T) = dL/df(T) and adds L to *loss.
template <typename S>
struct AdjLossArgs {
  Scalars s;
  const S* xlast;        // x(T-1)
  const double* ux_t;
  const double* uy_t;
  S* aout;
  double* loss;
  unsigned long long* status;
};

template <typename S, int QT, bool EX, int MODE>
__global__ void __launch_bounds__(kThreads) k_adj_loss(const __grid_constant__ Tables<S> tb,
                                                       const __grid_constant__ AdjLossArgs<S> a) {
  __shared__ double s_red[kThreads];
  const int tid = threadIdx.y * kBX + threadIdx.x;
  const int x = blockIdx.x * kBX + threadIdx.x;
  const int y = blockIdx.y * kBY + threadIdx.y;
  double part = 0.0;
  if (x < a.s.nx && y < a.s.ny) {
    const long long si = sidx(a.s, x, y);
    const int cell = y * a.s.nx + x;
    const int Qn = EX ? QT : a.s.Q;
    S g[QT];
    gather<S, QT, EX, MODE>(tb, a.s, a.xlast, si, g);
    S mm[9];
    moments9<S, QT, EX>(tb, a.s.Q, g, mm);
    const Macro M = landau<S>(a.s, mm);
    if (!M.ok) atomicAdd(a.status, 1ULL);
    S U0, Ux, Uy;
    if constexpr (sizeof(S) == 4) { U0 = M.fU0; Ux = M.fUx; Uy = M.fUy; }
    else { U0 = M.U0; Ux = M.Ux; Uy = M.Uy; }
    const S ux = Ux / U0, uy = Uy / U0;
    const S ex = ux - (S)a.ux_t[cell], ey = uy - (S)a.uy_t[cell];
    part = 0.5 * ((double)ex * (double)ex + (double)ey * (double)ey);
    const S gUx = ex / U0, gUy = ey / U0, gU0 = -(ex * ux + ey * uy) / U0;
    S gm[9];
    gm[0] = gm[1] = gm[2] = S(0);
    landau_vjp<S>(a.s, mm, (S)M.eps, S(0), gU0, gUx, gUy, gm);
    S out[QT];
#pragma unroll
    for (int i = 0; i < QT; ++i) {
      S acc = S(0);
      if (i < Qn) {
#pragma unroll
        for (int k = 0; k < 9; ++k) acc = fma(gm[k], tb.c[i][k], acc);
      }
      out[i] = acc;
    }
    S* __restrict__ ob = a.aout + si;
#pragma unroll
    for (int i = 0; i < QT; ++i)
      if (i < Qn) ob[i * a.s.iplane] = out[i];
    for_each_halo_image(a.s, x, y, [&](long long hi) {
      S* __restrict__ hb = a.aout + hi;
#pragma unroll
      for (int i = 0; i < QT; ++i)
        if (i < Qn) hb[i * a.s.iplane] = out[i];
    });
  }
  s_red[tid] = part;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (tid < w) s_red[tid] += s_red[tid + w];
    __syncthreads();
  }
  if (tid == 0) atomicAdd(a.loss, s_red[0]);
}

// Initial state x(0) = f_ref + H dM(n0, U(u0), T0): dL/du0 from lambda(0) = S^T a(1).
template <typename S>
struct AdjInitArgs {
  Scalars s;
  const S* a1;
  const double* n0;
  const double* ux0;
  const double* uy0;
  const double* T0;
  double* gux;
  double* guy;
};

template <typename S, int QT, bool EX, int MODE>
__global__ void __launch_bounds__(kThreads) k_adj_init(const __grid_constant__ Tables<S> tb,
                                                       const __grid_constant__ AdjInitArgs<S> a) {
  const int x = blockIdx.x * kBX + threadIdx.x;
  const int y = blockIdx.y * kBY + threadIdx.y;
  if (x >= a.s.nx || y >= a.s.ny) return;
  const long long si = sidx(a.s, x, y);
  const int cell = y * a.s.nx + x;
  const int Qn = EX ? QT : a.s.Q;
  S lam[QT];
  gather_rev<S, QT, EX, MODE>(tb, a.s, a.a1, si, lam);
  S h[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) h[k] = S(0);
#pragma unroll
  for (int i = 0; i < QT; ++i)
    if (i < Qn)
#pragma unroll
      for (int k = 0; k < 9; ++k) h[k] = fma(lam[i], tb.H[i][k], h[k]);
  const double ux = a.ux0[cell], uy = a.uy0[cell];
  const double gam = 1.0 / sqrt(1.0 - ux * ux - uy * uy);
  const S n = (S)a.n0[cell], T = (S)a.T0[cell];
  S gn = 0, gT = 0, gU0 = 0, gUx = 0, gUy = 0;
  dM_vjp<S>(h, n, T, (S)gam, (S)(gam * ux), (S)(gam * uy), (S)a.s.m, gn, gT, gU0, gUx, gUy);
  const double g3 = gam * gam * gam;
  // U0 = gam, Ux = gam ux, Uy = gam uy
  a.gux[cell] = (double)gU0 * g3 * ux + (double)gUx * (gam + g3 * ux * ux) + (double)gUy * g3 * ux * uy;
  a.guy[cell] = (double)gU0 * g3 * uy + (double)gUx * g3 * ux * uy + (double)gUy * (gam + g3 * uy * uy);
}

// ---------------------------------------------------------------------------

template <typename S, int QT, bool EX, bool SYM>
cudaError_t adj_step_q(const Tables<S>& tb, const AdjArgs<S>& a, int mode, cudaStream_t st) {
  if constexpr (SYM && sizeof(S) == 4) {
    if (a.macro) {
      if (mode == kOnLattice) k_adj_step<S, QT, EX, kOnLattice, SYM, true><<<grid_for(a.s), block_dim(), 0, st>>>(tb, a);
      else k_adj_step<S, QT, EX, kBilinear, SYM, true><<<grid_for(a.s), block_dim(), 0, st>>>(tb, a);
      return cudaGetLastError();
    }
  }
  if (a.macro) return cudaErrorInvalidValue;
  if (mode == kOnLattice) k_adj_step<S, QT, EX, kOnLattice, SYM, false><<<grid_for(a.s), block_dim(), 0, st>>>(tb, a);
  else k_adj_step<S, QT, EX, kBilinear, SYM, false><<<grid_for(a.s), block_dim(), 0, st>>>(tb, a);
  return cudaGetLastError();
}

// the built-in massless stencil (orbit order, exactly symmetric H) takes the
// orbit-symmetric VJP; any other order-2 stencil the bounded generic one
template <typename S>
cudaError_t adj_step(const Tables<S>& tb, const AdjArgs<S>& a, int mode, cudaStream_t st) {
  if (a.s.Q == 28 && a.s.sym) return adj_step_q<S, 28, true, true>(tb, a, mode, st);
  if (a.s.Q <= 40) return adj_step_q<S, 40, false, false>(tb, a, mode, st);
  return cudaErrorInvalidValue;
}

template <typename S>
cudaError_t adj_loss(const Tables<S>& tb, const AdjLossArgs<S>& a, int mode, cudaStream_t st) {
  if (a.s.Q == 28) {
    if (mode == kOnLattice) k_adj_loss<S, 28, true, kOnLattice><<<grid_for(a.s), block_dim(), 0, st>>>(tb, a);
    else k_adj_loss<S, 28, true, kBilinear><<<grid_for(a.s), block_dim(), 0, st>>>(tb, a);
  } else if (a.s.Q <= 40) {
    if (mode == kOnLattice) k_adj_loss<S, 40, false, kOnLattice><<<grid_for(a.s), block_dim(), 0, st>>>(tb, a);
    else k_adj_loss<S, 40, false, kBilinear><<<grid_for(a.s), block_dim(), 0, st>>>(tb, a);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename S>
cudaError_t adj_init(const Tables<S>& tb, const AdjInitArgs<S>& a, int mode, cudaStream_t st) {
  if (a.s.Q == 28) {
    if (mode == kOnLattice) k_adj_init<S, 28, true, kOnLattice><<<grid_for(a.s), block_dim(), 0, st>>>(tb, a);
    else k_adj_init<S, 28, true, kBilinear><<<grid_for(a.s), block_dim(), 0, st>>>(tb, a);
  } else if (a.s.Q <= 40) {
    if (mode == kOnLattice) k_adj_init<S, 40, false, kOnLattice><<<grid_for(a.s), block_dim(), 0, st>>>(tb, a);
    else k_adj_init<S, 40, false, kBilinear><<<grid_for(a.s), block_dim(), 0, st>>>(tb, a);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace rlbm

using namespace rlbm;

// ---------------------------------------------------------------------------
// Driver: forward with checkpoints, backward with recomputation.
// ---------------------------------------------------------------------------

struct rlbm_adjoint {
  rlbm_handle* h = nullptr;               // borrowed
  int T = 0;                              // forward steps of the run
  int K = 0;                              // checkpoint interval
  void* ckpt = nullptr;                   // checkpoints x(0), x(K), x(2K), ...
  // recomputed states of a segment (K + 1 buffers) and, FP32 storage, their
  // macroscopic states [K + 1][planes][ncell]: two sets, so that the
  // recomputation of segment s - 1 (on stream st2) overlaps the adjoint
  // steps of segment s (on the handle's stream)
  void* seg[2] = {nullptr, nullptr};
  float* macro[2] = {nullptr, nullptr};
  cudaStream_t st2 = nullptr;             // recomputation stream (lowest priority)
  cudaEvent_t ev_start = nullptr;         // work before the backward pass (handle's stream)
  cudaEvent_t ev_rec[2] = {nullptr, nullptr};   // segment set b recomputed
  cudaEvent_t ev_adj[2] = {nullptr, nullptr};   // adjoint steps on segment set b done
  void* adj[2] = {nullptr, nullptr};      // adjoint populations (ping-pong)
  double* gtau = nullptr;                 // dL/dtau per cell
  double* init_fields = nullptr;          // n0, ux0, uy0, T0 of the run [4][ncell]
  double* loss = nullptr;
  size_t buf_bytes = 0;
  int nckpt = 0;
  bool forward_done = false;
  std::string err = "no error";
};

namespace {

int adj_fail(rlbm_adjoint* A, int code, const std::string& msg) {
  if (A) A->err = msg;
  return code;
}

void* state_ptr(void* base, size_t bytes, int k) { return (char*)base + bytes * (size_t)k; }

float* macro_ptr(rlbm_adjoint* A, int b, int j) {
  return A->macro[b] + (size_t)j * kMacroPlanes * (size_t)A->h->sc.ncell;
}

// One forward step from src into dst using the handle's tables; with macro
// (FP32 storage) the step also writes the macroscopic state of its cells.
cudaError_t fwd_step(rlbm_handle* h, const void* src, void* dst, float* macro, cudaStream_t st) {
  const int mode = h->p.stream_mode == RLBM_BILINEAR ? kBilinear : kOnLattice;
  if (h->elem == 4) {
    StepArgs<float> a{h->sc, (const float*)src, (float*)dst, (const float*)h->tau_field, h->status, macro};
    return launch_step<float>(*h->tf, a, mode, st);
  }
  StepArgs<double> a{h->sc, (const double*)src, (double*)dst, (const double*)h->tau_field, h->status};
  return launch_step<double>(*h->td, a, mode, st);
}

void free_adjoint(rlbm_adjoint* A) {
  cudaFree(A->ckpt);
  for (int b = 0; b < 2; ++b) {
    cudaFree(A->seg[b]);
    cudaFree(A->macro[b]);
    if (A->ev_rec[b]) cudaEventDestroy(A->ev_rec[b]);
    if (A->ev_adj[b]) cudaEventDestroy(A->ev_adj[b]);
  }
  if (A->ev_start) cudaEventDestroy(A->ev_start);
  if (A->st2) cudaStreamDestroy(A->st2);
  cudaFree(A->adj[0]);
  cudaFree(A->adj[1]);
  cudaFree(A->gtau);
  cudaFree(A->init_fields);
  cudaFree(A->loss);
}

}  // namespace

extern "C" {

int rlbm_adjoint_create(rlbm_handle* h, int nsteps, int checkpoint_every, rlbm_adjoint** out) {
  if (!h || !out || nsteps < 1 || checkpoint_every < 1) return RLBM_ERR_INVALID_ARG;
  *out = nullptr;
  if (h->p.boundary != RLBM_BC_PERIODIC || h->p.order != 2 || h->p.tau_mode == RLBM_TAU_ETA_OVER_S ||
      h->q.Q > 40 || h->sc.force)
    return RLBM_ERR_UNSUPPORTED;   // adjoint: periodic, order 2, constant or per-cell tau
  std::unique_ptr<rlbm_adjoint> A(new rlbm_adjoint());
  A->h = h;
  A->T = nsteps;
  A->K = std::min(checkpoint_every, nsteps);
  A->buf_bytes = (size_t)h->q.Q * h->sc.plane * h->elem;
  A->nckpt = (nsteps + A->K - 1) / A->K;
  const size_t nc = (size_t)h->sc.ncell;
  cudaError_t e = cudaMalloc(&A->ckpt, A->buf_bytes * A->nckpt);
  const bool with_macro = h->elem == 4 && h->sc.sym && h->q.Q == 28;
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
    e = cudaMalloc(&A->seg[b], A->buf_bytes * (A->K + 1));
    if (e == cudaSuccess && with_macro) e = cudaMalloc(&A->macro[b], sizeof(float) * kMacroPlanes * nc * (A->K + 1));
  }
  if (e == cudaSuccess) e = cudaMalloc(&A->adj[0], A->buf_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&A->adj[1], A->buf_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&A->gtau, nc * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&A->init_fields, 4 * nc * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&A->loss, sizeof(double));
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_adjoint(A.get());
    return RLBM_ERR_OOM;
  }
  int prio_lo = 0, prio_hi = 0;
  e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&A->st2, cudaStreamNonBlocking, prio_lo);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&A->ev_start, cudaEventDisableTiming);
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
    e = cudaEventCreateWithFlags(&A->ev_rec[b], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&A->ev_adj[b], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_adjoint(A.get());
    return RLBM_ERR_CUDA;
  }
  cudaMemset(A->adj[0], 0, A->buf_bytes);
  cudaMemset(A->adj[1], 0, A->buf_bytes);
  *out = A.release();
  return RLBM_OK;
}

void rlbm_adjoint_destroy(rlbm_adjoint* A) {
  if (!A) return;
  cudaStreamSynchronize(A->h->stream);
  if (A->st2) cudaStreamSynchronize(A->st2);
  free_adjoint(A);
  delete A;
}

int rlbm_adjoint_forward(rlbm_adjoint* A, const double* n, const double* ux, const double* uy, const double* T,
                         int on_device) {
  if (!A || !n || !ux || !uy || !T) return RLBM_ERR_INVALID_ARG;
  rlbm_handle* h = A->h;
  const size_t nc = (size_t)h->sc.ncell;
  const double* src[4] = {n, ux, uy, T};
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  for (int k = 0; k < 4; ++k) {
    cudaError_t e = cudaMemcpyAsync(A->init_fields + k * nc, src[k], nc * sizeof(double), kind, h->stream);
    if (e != cudaSuccess) return adj_fail(A, RLBM_ERR_CUDA, cudaGetErrorString(e));
  }
  int rc = rlbm_init(h, A->init_fields, A->init_fields + nc, A->init_fields + 2 * nc, A->init_fields + 3 * nc, 1);
  if (rc != RLBM_OK) return adj_fail(A, rc, h->err);
  // x(0) in the handle's current buffer; run T steps, saving x(cK)
  for (int t = 0; t < A->T; ++t) {
    if (t % A->K == 0) {
      cudaError_t e = cudaMemcpyAsync(state_ptr(A->ckpt, A->buf_bytes, t / A->K), h->buf[h->cur], A->buf_bytes,
                                      cudaMemcpyDeviceToDevice, h->stream);
      if (e != cudaSuccess) return adj_fail(A, RLBM_ERR_CUDA, cudaGetErrorString(e));
    }
    rc = rlbm_step(h, 1);
    if (rc != RLBM_OK) return adj_fail(A, rc, h->err);
  }
  A->forward_done = true;
  return RLBM_OK;
}

int rlbm_adjoint_backward(rlbm_adjoint* A, const double* ux_target, const double* uy_target, int on_device,
                          double* loss, double* grad_tau, double* grad_ux0, double* grad_uy0, int out_on_device) {
  if (!A || !ux_target || !uy_target) return RLBM_ERR_INVALID_ARG;
  if (!A->forward_done) return adj_fail(A, RLBM_ERR_INVALID_ARG, "rlbm_adjoint_forward must run first");
  rlbm_handle* h = A->h;
  const Scalars& s = h->sc;
  const size_t nc = (size_t)s.ncell;
  const int mode = h->p.stream_mode == RLBM_BILINEAR ? kBilinear : kOnLattice;
  cudaStream_t st = h->stream;
  cudaError_t e;
  // targets: stage on the device (the handle's field planes 0, 1)
  const double* uxt = ux_target;
  const double* uyt = uy_target;
  if (!on_device) {
    e = cudaMemcpyAsync(h->fields, ux_target, nc * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->fields + nc, uy_target, nc * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return adj_fail(A, RLBM_ERR_CUDA, cudaGetErrorString(e));
    uxt = h->fields;
    uyt = h->fields + nc;
  }
  cudaMemsetAsync(A->gtau, 0, nc * sizeof(double), st);
  cudaMemsetAsync(A->loss, 0, sizeof(double), st);
  int an = 0;                  // adj[an] holds a(t+1)
  bool have_a = false;
  // Segment sgi covers the states x(c) .. x(last), c = sgi K.  Its adjoint
  // steps t (x(t-1) in the segment: t = t_hi .. c+1, t_hi = min(last+1, T-1);
  // t = T is the loss) read segment set sgi & 1.  The recomputation of
  // segment sgi - 1 runs on st2 while they execute; it waits for the
  // adjoint steps of segment sgi + 1, the last readers of its set.
  auto seg_bounds = [&](int sgi, int& c, int& last, int& t_hi) {
    c = sgi * A->K;
    last = std::min(c + A->K, A->T) - 1;
    t_hi = std::min(last + 1, A->T - 1);
  };
  // recompute the segment: seg[j] = x(c + j).  With stored macroscopic
  // states, macro[j] is that of f(c + j), which adjoint step t = c + j needs,
  // so the recompute runs up to j = t_hi - c (<= K)
  auto recompute = [&](int sgi) -> cudaError_t {
    const int b = sgi & 1;
    int c, last, t_hi;
    seg_bounds(sgi, c, last, t_hi);
    cudaError_t r = cudaMemcpyAsync(state_ptr(A->seg[b], A->buf_bytes, 0), state_ptr(A->ckpt, A->buf_bytes, sgi),
                                    A->buf_bytes, cudaMemcpyDeviceToDevice, A->st2);
    const int jmax = A->macro[b] ? std::max(t_hi - c, last - c) : last - c;
    for (int j = 1; j <= jmax && r == cudaSuccess; ++j)
      r = fwd_step(h, state_ptr(A->seg[b], A->buf_bytes, j - 1), state_ptr(A->seg[b], A->buf_bytes, j),
                   A->macro[b] ? macro_ptr(A, b, j) : nullptr, A->st2);
    if (r == cudaSuccess) r = cudaEventRecord(A->ev_rec[b], A->st2);
    return r;
  };
  e = cudaEventRecord(A->ev_start, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(A->st2, A->ev_start, 0);
  if (e == cudaSuccess) e = recompute(A->nckpt - 1);
  if (e != cudaSuccess) return adj_fail(A, RLBM_ERR_CUDA, cudaGetErrorString(e));
  for (int sgi = A->nckpt - 1; sgi >= 0; --sgi) {
    const int b = sgi & 1;
    int c, last, t_hi;
    seg_bounds(sgi, c, last, t_hi);
    if (sgi >= 1) {
      if (sgi + 1 <= A->nckpt - 1) e = cudaStreamWaitEvent(A->st2, A->ev_adj[b ^ 1], 0);
      if (e == cudaSuccess) e = recompute(sgi - 1);
    }
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, A->ev_rec[b], 0);
    if (e != cudaSuccess) return adj_fail(A, RLBM_ERR_CUDA, cudaGetErrorString(e));
    if (!have_a) {
      // a(T) from the loss on f(T) = S x(T-1), x(T-1) = seg[last - c]
      if (h->elem == 4) {
        AdjLossArgs<float> la{s, (const float*)state_ptr(A->seg[b], A->buf_bytes, last - c), uxt, uyt,
                              (float*)A->adj[an], A->loss, h->status};
        e = adj_loss<float>(*h->tf, la, mode, st);
      } else {
        AdjLossArgs<double> la{s, (const double*)state_ptr(A->seg[b], A->buf_bytes, last - c), uxt, uyt,
                               (double*)A->adj[an], A->loss, h->status};
        e = adj_loss<double>(*h->td, la, mode, st);
      }
      if (e != cudaSuccess) return adj_fail(A, RLBM_ERR_CUDA, cudaGetErrorString(e));
      have_a = true;
    }
    for (int t = t_hi; t >= c + 1; --t) {
      const void* xprev = state_ptr(A->seg[b], A->buf_bytes, t - 1 - c);
      if (h->elem == 4) {
        AdjArgs<float> aa{s, (const float*)xprev, (const float*)A->adj[an], (float*)A->adj[an ^ 1],
                          (const float*)h->tau_field, A->gtau, h->status,
                          A->macro[b] ? macro_ptr(A, b, t - c) : nullptr};
        e = adj_step<float>(*h->tf, aa, mode, st);
      } else {
        AdjArgs<double> aa{s, (const double*)xprev, (const double*)A->adj[an], (double*)A->adj[an ^ 1],
                           (const double*)h->tau_field, A->gtau, h->status};
        e = adj_step<double>(*h->td, aa, mode, st);
      }
      if (e != cudaSuccess) return adj_fail(A, RLBM_ERR_CUDA, cudaGetErrorString(e));
      an ^= 1;
    }
    e = cudaEventRecord(A->ev_adj[b], st);
    if (e != cudaSuccess) return adj_fail(A, RLBM_ERR_CUDA, cudaGetErrorString(e));
  }
  // dL/du0 from lambda(0) = S^T a(1)
  double* gux = h->fields + 2 * nc;
  double* guy = h->fields + 3 * nc;
  if (h->elem == 4) {
    AdjInitArgs<float> ia{s, (const float*)A->adj[an], A->init_fields, A->init_fields + nc, A->init_fields + 2 * nc,
                          A->init_fields + 3 * nc, gux, guy};
    e = adj_init<float>(*h->tf, ia, mode, st);
  } else {
    AdjInitArgs<double> ia{s, (const double*)A->adj[an], A->init_fields, A->init_fields + nc, A->init_fields + 2 * nc,
                           A->init_fields + 3 * nc, gux, guy};
    e = adj_init<double>(*h->td, ia, mode, st);
  }
  if (e != cudaSuccess) return adj_fail(A, RLBM_ERR_CUDA, cudaGetErrorString(e));
  const cudaMemcpyKind kind = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (grad_tau) e = cudaMemcpyAsync(grad_tau, A->gtau, nc * sizeof(double), kind, st);
  if (e == cudaSuccess && grad_ux0) e = cudaMemcpyAsync(grad_ux0, gux, nc * sizeof(double), kind, st);
  if (e == cudaSuccess && grad_uy0) e = cudaMemcpyAsync(grad_uy0, guy, nc * sizeof(double), kind, st);
  if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, A->loss, sizeof(double), kind, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return adj_fail(A, RLBM_ERR_CUDA, cudaGetErrorString(e));
  return RLBM_OK;
}

int rlbm_adjoint_step(rlbm_handle* h, const void* x_prev, const void* a_next, void* a_out, double* grad_tau) {
  if (!h || !x_prev || !a_next || !a_out || !grad_tau) return RLBM_ERR_INVALID_ARG;
  if (h->p.boundary != RLBM_BC_PERIODIC || h->p.order != 2 || h->p.tau_mode == RLBM_TAU_ETA_OVER_S ||
      h->q.Q > 40 || h->sc.force)
    return RLBM_ERR_UNSUPPORTED;
  const int mode = h->p.stream_mode == RLBM_BILINEAR ? kBilinear : kOnLattice;
  const void* tf = h->p.tau_mode == RLBM_TAU_FIELD ? h->tau_field : nullptr;
  cudaError_t e;
  if (h->elem == 4) {
    AdjArgs<float> aa{h->sc, (const float*)x_prev, (const float*)a_next, (float*)a_out, (const float*)tf, grad_tau,
                      h->status};
    e = adj_step<float>(*h->tf, aa, mode, h->stream);
  } else {
    AdjArgs<double> aa{h->sc, (const double*)x_prev, (const double*)a_next, (double*)a_out, (const double*)tf,
                       grad_tau, h->status};
    e = adj_step<double>(*h->td, aa, mode, h->stream);
  }
  if (e != cudaSuccess) {
    h->err = std::string("adjoint step kernel: ") + cudaGetErrorString(e);
    return RLBM_ERR_CUDA;
  }
  return RLBM_OK;
}

const char* rlbm_adjoint_last_error(const rlbm_adjoint* A) { return A ? A->err.c_str() : "null adjoint"; }

}  // extern "C"
