// Templates of the fused RLBM kernels: pull-stream + collide (Sec. 6.2 of
// arXiv:1909.04502), initialisation to equilibrium, and the macroscopic
// field extraction.  Instantiated per precision / order in step_o2.cu and
// step_o3.cu.
#pragma once
#include "fpconv.cuh"
#include "kernels.cuh"

namespace rlbm {

// 2-d thread blocks: a warp covers 32 consecutive cells of one row.
constexpr int kBX = 32;
constexpr int kBY = 4;
constexpr int kThreads = kBX * kBY;

// kernel parameters are limited to 32764 bytes
static_assert(sizeof(Tables<double>) + sizeof(MomentArgs<double>) <= 32764, "kernel parameter space");

// ---------------------------------------------------------------------------
// Step 1 of the update: streaming by pull (Eq. discrete-rbe, left side) from
// the padded layout: the halo already holds the periodic images / free-flow
// copies, so every tap is base + constant offset.
// On-lattice: f_i(x) = f*_i(x - n_i).  Bilinear: f_i(x) = sum_ab W_ab
// f*_i(x + o_i + (a, b)).
// ---------------------------------------------------------------------------
// DYN: offsets computed from (dx, dy) and the run-time pitch (tables shared
// by grids of different sizes), otherwise taken precomputed from tb.off.
// NC: read through the non-coherent read-only path; only valid when the
// source buffer is not written while the kernel runs (not in the persistent
// batched kernel, which writes the buffer its next step reads).
template <typename T, bool NC>
__device__ __forceinline__ T ld(const T* p) {
  if constexpr (NC) return __ldg(p);
  else return *p;
}

template <typename S, int QT, bool EX, int MODE, bool DYN = false, bool NC = true>
__device__ __forceinline__ void gather(const Tables<S>& tb, const Scalars& s,
                                       const S* __restrict__ fin, long long si, S (&g)[QT]) {
  const S* __restrict__ base = fin + si;
  const int Qn = EX ? QT : s.Q;
#pragma unroll
  for (int i = 0; i < QT; ++i) {
    g[i] = S(0);
    if (i < Qn) {
      const int o = DYN ? i * s.iplane + (int)tb.dy[i] * s.pitch + (int)tb.dx[i] : tb.offp[i];
      if constexpr (MODE == kOnLattice) {
        g[i] = ld<S, NC>(base + o);
      } else {
        const int o2 = DYN ? o + s.pitch : tb.offr[i];
        S v = tb.bw[i][0] * ld<S, NC>(base + o);
        v = fma(tb.bw[i][1], ld<S, NC>(base + o + 1), v);
        v = fma(tb.bw[i][2], ld<S, NC>(base + o2), v);
        v = fma(tb.bw[i][3], ld<S, NC>(base + o2 + 1), v);
        g[i] = v;
      }
    }
  }
}

// Step 1: N^a = sum_i f_i p_i^a, T^ab = sum_i f_i p_i^a p_i^b (of the
// stored, possibly shifted, populations).
template <typename S, int QT, bool EX>
__device__ __forceinline__ void moments9(const Tables<S>& tb, int Q, const S (&g)[QT], S (&mm)[9]) {
  const int Qn = EX ? QT : Q;
#pragma unroll
  for (int j = 0; j < 9; ++j) mm[j] = S(0);
#pragma unroll
  for (int i = 0; i < QT; ++i) {
    if (i < Qn) {
#pragma unroll
      for (int j = 0; j < 9; ++j) mm[j] = fma(g[i], tb.c[i][j], mm[j]);
    }
  }
}

// ---------------------------------------------------------------------------
// Steps 2-4: Landau frame eps U^a = T^ab U_b (largest eigenvalue of the mixed
// tensor T^a_b with a timelike eigenvector, Sec. 4), n = U_a N^a, T from
// eps/n = T (G_2(m/T) - 1) (Eq. eos-ddim), inverted in closed form for d = 2.
//
// The eigenvalue is the largest root of p(l) = det(A - l I),
//   p(l) = a D - s vx - t vy,  a = T00 - l, b = Txx + l, c = Tyy + l,
//   D = b c - r^2, vx = s c - r t, vy = t b - r s  (s = T0x, t = T0y, r = Txy),
// and v = (D, vx, vy) is its eigenvector.  The first guess is the exact root
// for an ideal fluid with P = kappa eps (kappa of the reference state),
// refined by FP32 Newton steps.
// ---------------------------------------------------------------------------

// FP64 mode: the whole solve in FP64 (two Newton steps from the FP32 root).
__device__ __forceinline__ Macro landau_fp64(const Scalars& sc, const double (&mm)[9]) {
  const double N0 = sc.N0_ref + mm[0], Nx = mm[1], Ny = mm[2];
  const double T00 = sc.T00_ref + mm[3], T0x = mm[4], T0y = mm[5];
  const double Txx = sc.Tii_ref + mm[6], Txy = mm[7], Tyy = sc.Tii_ref + mm[8];
  const float fE = (float)T00, fxx = (float)Txx, fyy = (float)Tyy;
  const float fs = (float)T0x, ft = (float)T0y, fr = (float)Txy;
  const float k = sc.kappa_guess;
  const float M2 = fs * fs + ft * ft;
  const float disc = (1.f - k) * (1.f - k) * fE * fE + 4.f * k * (fE * fE - M2);
  float lam = (-(1.f - k) * fE + sqrtf(fmaxf(disc, 0.f))) / (2.f * k);
#pragma unroll
  for (int it = 0; it < 3; ++it) {
    float a = fE - lam, b = fxx + lam, c = fyy + lam;
    float D = b * c - fr * fr;
    float p = a * D - fs * (fs * c - fr * ft) - ft * (ft * b - fr * fs);
    float dp = -D + a * (b + c) - M2;
    lam -= p / dp;
  }
  double L = (double)lam;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    double a = T00 - L, b = Txx + L, c = Tyy + L;
    double D = fma(b, c, -Txy * Txy);
    double vx = fma(T0x, c, -Txy * T0y), vy = fma(T0y, b, -Txy * T0x);
    double p = fma(a, D, -fma(T0x, vx, T0y * vy));
    double dp = -D + a * (b + c) - T0x * T0x - T0y * T0y;
    L -= p / dp;
  }
  const double b = Txx + L, c = Tyy + L;
  const double D = fma(b, c, -Txy * Txy);
  const double vx = fma(T0x, c, -Txy * T0y);
  const double vy = fma(T0y, b, -Txy * T0x);
  const double nrm2 = fma(D, D, -fma(vx, vx, vy * vy));
  const double inv = rsqrt(nrm2);
  Macro M;
  M.eps = L;
  M.U0 = D * inv;
  M.Ux = vx * inv;
  M.Uy = vy * inv;
  M.n = fma(M.U0, N0, -fma(M.Ux, Nx, M.Uy * Ny));
  const double m = sc.m;
  if (m == 0.0) {
    M.T = 0.5 * L / M.n;   // eps = 2 P = 2 n T
  } else {
    const double e = L / M.n;
    M.T = 0.25 * ((e - 2.0 * m) + sqrt(fma(e, e, 4.0 * m * (e - m))));
  }
  M.ok = (D > 0.0) && (nrm2 > 0.0) && (M.n > 0.0) && (M.T > 0.0) && (L > 0.0) && isfinite(M.T) &&
         isfinite(M.U0);
  return M;
}

// Approximate FP32 square root (PTX sqrt.approx.f32, a few ulp): used only
// for the first guess, which the Newton steps refine.
__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// FP32 storage: the solve runs in FP32, then one Newton correction whose
// residual p(l) is evaluated in float-float arithmetic (about 48 bits) at
// the FP32 root (the eigenvalue, and with it eps, carries that accuracy: it
// decides energy conservation).  The
// rest is formed in FP32 from quantities accurate relative to the deviation
// from the reference state, so that every FP32 rounding is proportional to
// that deviation, like the storage of g = f - f_ref itself:
//   v = (D, vx, vy), the eigenvector, shifted to the corrected root to first
//     order (v is quadratic in l: the remainder is O(dl^2));
//   U = v / nu, nu^2 = v.v;
//   dn = n - n_ref = (w - n_ref nu) / nu with w = v.N (n = U.N, step 3), in
//     the difference form
//       w - n_ref nu = D dN0 - vx Nx - vy Ny + n_ref (vx^2 + vy^2) / (D + nu),
//     dN0 = N0 - n_ref (the FP32 moment of g), whose terms are all of the
//     size of the deviation (D - nu = (vx^2 + vy^2)/(D + nu) without
//     cancellation);
//   d_eps = eps - eps_ref (the FP32 Newton unknown plus its correction);
//   dT = T - T_ref from the EOS written for differences.
// No FP64 operation.  The moments are reference + FP32 sums of g,
// and the eigenvalue is written l = eps_ref + delta.
// ML: 1 massless, 0 massive (known at compile time), -1 decided by sc.massless.
template <int ML = -1>
__device__ __forceinline__ Macro landau_fp32(const Scalars& sc, const float (&mm)[9]) {
  const float epsr = sc.f_T00_ref;
  const float Pr = sc.f_Tii_ref;
  const float fs = mm[4], ft = mm[5], fr = mm[7];
  const float M2 = fs * fs + ft * ft;
  // FP32 guess for delta = l - eps_ref
  const float fE = epsr + mm[3];
  const float k = sc.kappa_guess;
  const float disc = (1.f - k) * (1.f - k) * fE * fE + 4.f * k * (fE * fE - M2);
  const float lam0 = __fdividef(-(1.f - k) * fE + sqrt_approx(fmaxf(disc, 0.f)), 2.f * k);
  float del = lam0 - epsr;
  const float PE = Pr + epsr;
  float b = 0.f, c = 0.f, dp = 1.f;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const float a = mm[3] - del;
    b = PE + mm[6] + del;
    c = PE + mm[8] + del;
    const float D = b * c - fr * fr;
    const float p = a * D - fs * (fs * c - fr * ft) - ft * (ft * b - fr * fs);
    dp = -D + a * (b + c) - M2;
    del -= __fdividef(p, dp);
  }
  // residual p(l) at l = eps_ref + del in float-float arithmetic; every
  // input but P_ref + eps_ref is an FP32 number
  {
    const ff PE = {sc.f_PE_hi, sc.f_PE_lo};
    const ff cd = ff_add(PE, ff_sum(mm[8], del));             // Tyy + l
    ff acc = ff_mulf(fs, ff_sub(ff_mulf(fs, cd), ff_prod(fr, ft)));       // s vx
    const ff bd = ff_add(PE, ff_sum(mm[6], del));             // Txx + l
    acc = ff_add(acc, ff_mulf(ft, ff_sub(ff_mulf(ft, bd), ff_prod(fr, fs))));   // + t vy
    const ff D = ff_sub(ff_mul(bd, cd), ff_prod(fr, fr));
    const ff p = ff_sub(ff_mul(ff_sum(mm[3], -del), D), acc);   // (T00 - l) D - s vx - t vy
    dp = -__fdividef(p.hi + p.lo, dp);     // Newton correction dl (FP32 is enough)
  }
  const float dl = dp;
  const float fNx = mm[1], fNy = mm[2];
  // the eigenvector at the corrected root, in FP32 (D ~ (P + eps)^2 and the
  // leading terms of vx, vy do not cancel)
  const float fb = PE + mm[6] + del, fc = PE + mm[8] + del;
  const float bc = fb + fc;
  const float fD = fmaf(dl, bc, fb * fc - fr * fr);
  const float fvx = fmaf(dl, fs, fs * fc - fr * ft);
  const float fvy = fmaf(dl, ft, ft * fb - fr * fs);
  const float vv = fvx * fvx + fvy * fvy;
  const float fnu2 = fD * fD - vv;
  const float inu = rsqrtf(fnu2);
  const float fnu = fnu2 * inu;
  const float nr = sc.f_n_ref;
  const float X = fD * mm[0] - fvx * fNx - fvy * fNy + __fdividef(nr * vv, fD + fnu);
  Macro M;
  M.fU0 = fD * inu;
  M.fUx = fvx * inu;
  M.fUy = fvy * inu;
  M.fdn = X * inu;
  M.fn = nr + M.fdn;
  const float deps = del + dl;                          // eps - eps_ref
  const float fn = M.fn, fm = sc.f_m, fTr = sc.f_T_ref;
  if (ML == 1 || (ML == -1 && sc.massless)) {
    // eps = 2 n T with eps_ref = 2 n_ref T_ref:  dT = (d_eps - 2 T_ref dn) / (2 n)
    M.fdT = __fdividef(deps - 2.f * fTr * M.fdn, 2.f * fn);
  } else if (sc.f_n_ref > 0.f) {
    // 2T^2 + (2m - e) T + m (m - e) = 0 for (T, e) and (T_ref, e_ref):
    // dT (2 (T + T_ref + m) - e) = de (T_ref + m),  e = eps/n
    // with T = T_ref + dT:  2 dT^2 + B dT - de (T_ref + m) = 0,  B = 4 T_ref + 2m - e
    const float feps = epsr + deps;
    const float de = __fdividef(deps * nr - epsr * M.fdn, fn * nr);
    const float e = __fdividef(feps, fn);
    const float Bq = 4.f * fTr + 2.f * fm - e, Cq = de * (fTr + fm);
    M.fdT = __fdividef(2.f * Cq, Bq + sqrtf(fmaxf(Bq * Bq + 8.f * Cq, 0.f)));
  } else {
    const float e = __fdividef(epsr + deps, fn);
    const float T0 = 0.25f * ((e - 2.f * fm) + sqrtf(fmaxf(e * e + 4.f * e * fm - 4.f * fm * fm, 0.f)));
    M.fdT = T0 - fTr;
  }
  M.fT = fTr + M.fdT;
  M.feps = epsr + deps;
  M.eps = sc.T00_ref + f2d(deps);
  M.n = f2d(fn);
  M.T = f2d(M.fT);
  M.U0 = f2d(M.fU0);
  M.Ux = f2d(M.fUx);
  M.Uy = f2d(M.fUy);
  // a timelike eigenvector with v^0 > 0, n > 0, T > 0; the FP32 tests also
  // catch non-finite values
  M.ok = (fD > 0.f) && (fnu2 > 0.f) && (fn > 0.f) && (M.fT > 0.f) && isfinite(M.fT) && isfinite(M.fU0) &&
         isfinite(M.fn) && isfinite(M.fdn);
  return M;
}

// Step 5, moment side: dM = M(n, U, T) - M(n_ref, e0, T_ref) for the basis of
// setup.h (p0^e px^a py^b, e + a + b <= N), using the App. B moments
//   <1> = n/(m+T), <p^a> = n U^a, <p^a p^b> = n (r2 U^a U^b - T eta^ab),
//   <p^a p^b p^c> = n (r3 U^a U^b U^c - T r2 (eta^ab U^c + eta^ac U^b + eta^bc U^a)),
//   r2 = (m^2 + 3mT + 3T^2)/(m+T), r3 = (m^3 + 6m^2 T + 15 m T^2 + 15 T^3)/(m+T).
// The differences from the reference are rearranged so that the result is
// accurate relative to dM itself given accurate dn = n - n_ref and dT = T - T_ref.
// Quotient: the FP32 path uses the fast reciprocal-based division (2 ulp,
// no special-case branches), the FP64 path the IEEE one.
template <typename S>
__device__ __forceinline__ S qdiv(S a, S b) {
  if constexpr (sizeof(S) == 4) return __fdividef(a, b);
  else return a / b;
}

template <typename S, int KT>
__device__ __forceinline__ void eq_moments(S dn, S dT, S n, S T, S U0, S Ux, S Uy, S m, S nr, S Tr,
                                           S (&dM)[KT]) {
  const S U0m1 = qdiv(Ux * Ux + Uy * Uy, U0 + S(1));
  const S mT = m + T, mTr = m + Tr;
  const S r2 = qdiv(m * m + S(3) * m * T + S(3) * T * T, mT);
  const S D1 = qdiv(dn * mTr - nr * dT, mT * mTr);
  const S D2 = dn * U0 + nr * U0m1;
  const S D3 = dn * T + nr * dT;
  const S nr2 = n * r2;
  dM[0] = D1;
  dM[1] = D2;
  dM[2] = n * Ux;
  dM[3] = n * Uy;
  dM[4] = nr2 * U0 * Ux;
  dM[5] = nr2 * U0 * Uy;
  dM[6] = nr2 * Ux * Ux + D3;
  dM[7] = nr2 * Ux * Uy;
  dM[8] = nr2 * Uy * Uy + D3;
  if constexpr (KT == 16) {
    // Order 3: the members with p0 are the shifted (p0 - m) X, X = 1, px, py,
    // pxpx, pxpy, pypy (the basis the host builds H for), with
    //   <(p0 - m) X> = <p0 X> - m <X>,  r2 U0 - m = r2 (U0 - 1) + T c2,
    //   r3 U0 - m r2 = r3 (U0 - 1) + T c3,
    //   c2 = (2m + 3T)/(m + T),  c3 = 3 (m^2 + 4mT + 5T^2)/(m + T):
    // positive terms only, where <p0 X> and m <X> cancel to 1e-3 at m~ = 20.
    // Differences from the reference (n_ref, rest, T_ref):
    //   <p0 - m>:  n (U0 - 1) + (dn T (m + T_ref) + n_ref m dT) / ((m + T)(m + T_ref)),
    //   T (r2 U0 - m) part of <(p0 - m) pxpx>:  n T r2 (U0 - 1) + dn T^2 c2
    //     + n_ref (h(T) - h(T_ref)),  h(T) = T^2 (2m + 3T)/(m + T),
    //   h(T) - h(T_ref) = dT (2m^2 (T + T_ref) + 2m T T_ref
    //     + 3m (T^2 + T T_ref + T_ref^2) + 3 T T_ref (T + T_ref)) / ((m + T)(m + T_ref)).
    // one quotient for the five divisions by (m + T) and (m + T)(m + T_ref)
    const S iden = qdiv(S(1), mT * mTr), imT = iden * mTr;
    const S q2 = T * r2;
    const S r3 = (m * m * m + S(6) * m * m * T + S(15) * m * T * T + S(15) * T * T * T) * imT;
    const S c2 = (S(2) * m + S(3) * T) * imT;
    const S c3 = S(3) * (m * m + S(4) * m * T + S(5) * T * T) * imT;
    const S A2 = r2 * U0m1 + T * c2;
    const S A3 = r3 * U0m1 + T * c3;
    dM[1] = n * U0m1 + (dn * T * mTr + nr * m * dT) * iden;
    dM[4] = n * Ux * A2;
    dM[5] = n * Uy * A2;
    const S Nh = dT * (S(2) * m * m * (T + Tr) + S(2) * m * T * Tr + S(3) * m * (T * T + T * Tr + Tr * Tr) +
                       S(3) * T * Tr * (T + Tr));
    const S D5 = n * T * r2 * U0m1 + dn * T * T * c2 + nr * Nh * iden;
    const S nA3 = n * A3;
    const S nr3 = n * r3, nq2 = n * q2;
    dM[9] = nA3 * Ux * Ux + D5;
    dM[10] = nA3 * Ux * Uy;
    dM[11] = nA3 * Uy * Uy + D5;
    dM[12] = nr3 * Ux * Ux * Ux + S(3) * nq2 * Ux;
    dM[13] = nr3 * Ux * Ux * Uy + nq2 * Uy;
    dM[14] = nr3 * Ux * Uy * Uy + nq2 * Ux;
    dM[15] = nr3 * Uy * Uy * Uy + S(3) * nq2 * Uy;
  }
}

template <typename S, int KT>
__device__ __forceinline__ void eq_moments_of(const Scalars& sc, const Macro& M, S (&dM)[KT]) {
  if constexpr (sizeof(S) == 4) {
    eq_moments<S, KT>(M.fdn, M.fdT, M.fn, M.fT, M.fU0, M.fUx, M.fUy, sc.f_m, sc.f_n_ref, sc.f_T_ref, dM);
  } else {
    eq_moments<S, KT>(M.n - sc.n_ref, M.T - sc.T_ref, M.n, M.T, M.U0, M.Ux, M.Uy, sc.m, sc.n_ref,
                      sc.T_ref, dM);
  }
}

// The reference state (rest, n_ref, T_ref; n = 1 without the storage
// shift) in place of a cell's non-physical frame, as selects on the members
// the step of storage type S reads; ok stays false.
template <typename S>
__device__ __forceinline__ void unphysical_to_reference(const Scalars& sc, Macro& M) {
  const bool bad = !M.ok;
  if constexpr (sizeof(S) == 4) {
    const float n = sc.f_n_ref > 0.f ? sc.f_n_ref : 1.f;
    M.fU0 = bad ? 1.f : M.fU0;
    M.fUx = bad ? 0.f : M.fUx;
    M.fUy = bad ? 0.f : M.fUy;
    M.fn = bad ? n : M.fn;
    M.fT = bad ? sc.f_T_ref : M.fT;
    M.fdn = bad ? 0.f : M.fdn;
    M.fdT = bad ? 0.f : M.fdT;
  } else {
    const double n = sc.n_ref > 0.0 ? sc.n_ref : 1.0;
    M.U0 = bad ? 1.0 : M.U0;
    M.Ux = bad ? 0.0 : M.Ux;
    M.Uy = bad ? 0.0 : M.Uy;
    M.n = bad ? n : M.n;
    M.T = bad ? sc.T_ref : M.T;
  }
}

template <typename S, int ML = -1>
__device__ __forceinline__ Macro landau(const Scalars& sc, const S (&mm)[9]) {
  if constexpr (sizeof(S) == 4) return landau_fp32<ML>(sc, mm);
  else return landau_fp64(sc, mm);
}

template <typename S>
__device__ __forceinline__ S local_tau(const Scalars& sc, const S* __restrict__ tau_field, int cell,
                                       const Macro& M) {
  if (sc.tau_mode == 1) return tau_field[cell];
  if constexpr (sizeof(S) == 4) {
    if (sc.tau_mode == 2) return __fdividef(sc.f_tau_coef, M.fT);   // step 7, eta/s fixed
    return sc.f_tau;
  } else {
    if (sc.tau_mode == 2) return sc.tau_coef / M.T;   // step 7, eta/s fixed: tau = (eta/s)(d+2) kappa / T
    return sc.tau;
  }
}

// Halo images of interior cell (x, y): every padded position outside the
// interior that shows this cell -- periodic images in y, and in x either
// periodic images or, for free-flow ends, the halo columns beside the first
// and last column.  Calls st(storage index) for each image.
template <typename F>
__device__ __forceinline__ void for_each_halo_image(const Scalars& s, int x, int y, F&& st) {
  const bool xband = (s.boundary == 0) ? (x < s.hx || x >= s.nx - s.hx) : (x == 0 || x == s.nx - 1);
  const bool yband = (y < s.hy || y >= s.ny - s.hy);
  if (!xband && !yband) return;
  int xlo, xhi, xstep;
  if (s.boundary == 0) {
    xlo = x - ((x + s.hx) / s.nx) * s.nx;       // smallest image >= -hx
    xhi = s.nx + s.hx - 1;
    xstep = s.nx;
  } else {
    xlo = (x == 0) ? -s.hx : x;
    xhi = (x == s.nx - 1) ? s.nx - 1 + s.hx : x;
    xstep = 1;
  }
  for (int yp = y - ((y + s.hy) / s.ny) * s.ny; yp < s.ny + s.hy; yp += s.ny) {
    for (int xp = xlo; xp <= xhi; xp += xstep) {
      if (xp == x && yp == y) continue;
      st((long long)(yp + s.hy) * s.pitch + (xp + s.px));
    }
  }
}

// ---------------------------------------------------------------------------
// Fused step kernel: one thread per cell, 32 x 4 cells per block.
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Orbit-symmetric evaluation for the built-in massless stencils.  Their
// populations come in orbit order (setup.cpp): per shell of the (3, 4) family
// two sign quartets, (a, b), (-a, b), (a, -b), (-a, -b) and the same for the
// swap (b, a); per shell of the (5, 0) family (p, 0), (-p, 0), (0, p), (0, -p).
// Under a sign flip of px (py) the monomials of odd px (py) degree change sign,
// and the swap px <-> py permutes them, so
//   * the moments need per quartet only its sum and its x-, y- and
//     xy-antisymmetric combinations (butterflies), and
//   * the equilibrium row of every member is its orbit's first row with
//     signs and (for the swapped quartet) permuted columns: per quartet the
//     four parity classes of H_k dM_k are summed once and combined.
// The host enables this only after checking these identities on H exactly.
// ---------------------------------------------------------------------------
// Orbit composition of the stencils with a symmetric evaluation, in the
// population order of setup.cpp: n8 eight-member orbits, then n4 axis
// quartets, nd diagonal quartets and n1 rest populations.
// (massless: the stencil belongs to m~ = 0, which fixes the EOS branch at
// compile time)
template <int QT>
struct Orbits {
  static constexpr int n8 = 0, n4 = 0, nd = 0, n1 = 0;
  static constexpr bool massless = false;
};
template <>
struct Orbits<28> {   // massless order 2: 3 shells x 8 + 1 shell x 4
  static constexpr int n8 = 3, n4 = 1, nd = 0, n1 = 0;
  static constexpr bool massless = true;
};
template <>
struct Orbits<44> {   // massless order 3: 4 shells x 8 + 3 shells x 4
  static constexpr int n8 = 4, n4 = 3, nd = 0, n1 = 0;
  static constexpr bool massless = true;
};
template <>
struct Orbits<33> {   // built-in m~ = 1, order 2
  static constexpr int n8 = 3, n4 = 1, nd = 1, n1 = 1;
  static constexpr bool massless = false;
};
template <>
struct Orbits<29> {   // built-in m~ = 5, order 2
  static constexpr int n8 = 2, n4 = 1, nd = 2, n1 = 1;
  static constexpr bool massless = false;
};
template <>
struct Orbits<25> {   // built-in m~ = 10, order 2
  static constexpr int n8 = 1, n4 = 2, nd = 2, n1 = 1;
  static constexpr bool massless = false;
};
template <>
struct Orbits<65> {   // built-in order 3, App. H column A (m~ = 1.5 ... 4)
  static constexpr int n8 = 7, n4 = 0, nd = 2, n1 = 1;
  static constexpr bool massless = false;
};
template <>
struct Orbits<57> {   // built-in order 3, App. H column B (m~ = 3)
  static constexpr int n8 = 5, n4 = 1, nd = 3, n1 = 1;
  static constexpr bool massless = false;
};
template <>
struct Orbits<49> {   // built-in order 3, App. H column C (m~ = 5)
  static constexpr int n8 = 3, n4 = 4, nd = 2, n1 = 1;
  static constexpr bool massless = false;
};
template <>
struct Orbits<53> {   // built-in order 3, App. H column D (m~ = 7 ... 20)
  static constexpr int n8 = 4, n4 = 3, nd = 2, n1 = 1;
  static constexpr bool massless = false;
};
template <>
struct Orbits<45> {   // order 3, the paper's performance-table stencil (Sec. 6.3): (2,1), (3,2)
                      // eight-member orbits, four axis, three diagonal quartets, rest
  static constexpr int n8 = 2, n4 = 4, nd = 3, n1 = 1;
  static constexpr bool massless = false;
};
template <int QT>
struct OrbitStart {
  using O = Orbits<QT>;
  static constexpr int axis = 8 * O::n8, diag = axis + 4 * O::n4, rest = diag + 4 * O::nd;
  static_assert(rest + O::n1 == QT || QT == 0 || O::n8 + O::n4 == 0, "orbit composition must cover the stencil");
};

template <typename S, int QT>
__device__ __forceinline__ void moments_sym(const Tables<S>& tb, const S (&g)[QT], S (&mm)[9]) {
  using O = Orbits<QT>;
#pragma unroll
  for (int j = 0; j < 9; ++j) mm[j] = S(0);
#pragma unroll
  for (int o = 0; o < O::n8; ++o) {
    const int i = 8 * o;
    const S u0 = g[i] + g[i + 1], u1 = g[i] - g[i + 1], u2 = g[i + 2] + g[i + 3], u3 = g[i + 2] - g[i + 3];
    const S v0 = g[i + 4] + g[i + 5], v1 = g[i + 4] - g[i + 5], v2 = g[i + 6] + g[i + 7], v3 = g[i + 6] - g[i + 7];
    const S SA = u0 + u2, YA = u0 - u2, XA = u1 + u3, XYA = u1 - u3;
    const S SB = v0 + v2, YB = v0 - v2, XB = v1 + v3, XYB = v1 - v3;
    const S Sab = SA + SB;
    // c = p0, a, b, p0^2, p0 a, p0 b, a^2, a b, b^2 of the quartet-A base (a, b)
    mm[0] = fma(tb.c[i][0], Sab, mm[0]);
    mm[1] = fma(tb.c[i][1], XA, fma(tb.c[i][2], XB, mm[1]));
    mm[2] = fma(tb.c[i][2], YA, fma(tb.c[i][1], YB, mm[2]));
    mm[3] = fma(tb.c[i][3], Sab, mm[3]);
    mm[4] = fma(tb.c[i][4], XA, fma(tb.c[i][5], XB, mm[4]));
    mm[5] = fma(tb.c[i][5], YA, fma(tb.c[i][4], YB, mm[5]));
    mm[6] = fma(tb.c[i][6], SA, fma(tb.c[i][8], SB, mm[6]));
    mm[7] = fma(tb.c[i][7], XYA + XYB, mm[7]);
    mm[8] = fma(tb.c[i][8], SA, fma(tb.c[i][6], SB, mm[8]));
  }
#pragma unroll
  for (int o = 0; o < O::n4; ++o) {
    const int i = OrbitStart<QT>::axis + 4 * o;
    const S S1 = g[i] + g[i + 1], D1 = g[i] - g[i + 1], S2 = g[i + 2] + g[i + 3], D2 = g[i + 2] - g[i + 3];
    const S Sab = S1 + S2;
    // c = p0, p, 0, p0^2, p0 p, 0, p^2, 0, 0 of the base (p, 0)
    mm[0] = fma(tb.c[i][0], Sab, mm[0]);
    mm[1] = fma(tb.c[i][1], D1, mm[1]);
    mm[2] = fma(tb.c[i][1], D2, mm[2]);
    mm[3] = fma(tb.c[i][3], Sab, mm[3]);
    mm[4] = fma(tb.c[i][4], D1, mm[4]);
    mm[5] = fma(tb.c[i][4], D2, mm[5]);
    mm[6] = fma(tb.c[i][6], S1, mm[6]);
    mm[8] = fma(tb.c[i][6], S2, mm[8]);
  }
#pragma unroll
  for (int o = 0; o < O::nd; ++o) {
    const int i = OrbitStart<QT>::diag + 4 * o;
    // (a, a), (-a, a), (a, -a), (-a, -a): one sign quartet with a = b
    const S u0 = g[i] + g[i + 1], u1 = g[i] - g[i + 1], u2 = g[i + 2] + g[i + 3], u3 = g[i + 2] - g[i + 3];
    const S SA = u0 + u2, YA = u0 - u2, XA = u1 + u3, XYA = u1 - u3;
    mm[0] = fma(tb.c[i][0], SA, mm[0]);
    mm[1] = fma(tb.c[i][1], XA, mm[1]);
    mm[2] = fma(tb.c[i][1], YA, mm[2]);
    mm[3] = fma(tb.c[i][3], SA, mm[3]);
    mm[4] = fma(tb.c[i][4], XA, mm[4]);
    mm[5] = fma(tb.c[i][4], YA, mm[5]);
    mm[6] = fma(tb.c[i][6], SA, mm[6]);
    mm[7] = fma(tb.c[i][7], XYA, mm[7]);
    mm[8] = fma(tb.c[i][6], SA, mm[8]);
  }
#pragma unroll
  for (int o = 0; o < O::n1; ++o) {
    const int i = OrbitStart<QT>::rest + o;   // p = (p0, 0, 0)
    mm[0] = fma(tb.c[i][0], g[i], mm[0]);
    mm[3] = fma(tb.c[i][3], g[i], mm[3]);
  }
}

// f^eq - f_ref of the eight members of the (a, b) orbit whose first row is h.
template <typename S, int KT>
__device__ __forceinline__ void feq_orbit8(const S (&h)[kMaxK], const S (&dM)[KT], S (&f)[8]) {
  S E = S(0), OX = S(0), OY = S(0), OXY = S(0), Eb = S(0), OXb = S(0), OYb = S(0), OXYb = S(0);
#pragma unroll
  for (int k = 0; k < KT; ++k) {
    const int ax = mono_ax(k), ay = mono_ay(k);
    const S t = dM[mono_swap(k)];
    if (!ax && !ay) { E = fma(h[k], dM[k], E); Eb = fma(h[k], t, Eb); }
    else if (ax && !ay) { OX = fma(h[k], dM[k], OX); OYb = fma(h[k], t, OYb); }
    else if (!ax && ay) { OY = fma(h[k], dM[k], OY); OXb = fma(h[k], t, OXb); }
    else { OXY = fma(h[k], dM[k], OXY); OXYb = fma(h[k], t, OXYb); }
  }
  // member (sx, sy): E + sx OX + sy OY + sx sy OXY, order (+,+), (-,+), (+,-), (-,-)
  const S A = E + OXY, B = E - OXY, C = OX + OY, D = OX - OY;
  f[0] = A + C; f[1] = B - D; f[2] = B + D; f[3] = A - C;
  const S Ab = Eb + OXYb, Bb = Eb - OXYb, Cb = OXb + OYb, Db = OXb - OYb;
  f[4] = Ab + Cb; f[5] = Bb - Db; f[6] = Bb + Db; f[7] = Ab - Cb;
}

// ... of the four members (a, a), (-a, a), (a, -a), (-a, -a) of a diagonal
// quartet (their rows are the first row with the flips' column signs) ...
template <typename S, int KT>
__device__ __forceinline__ void feq_diag4(const S (&h)[kMaxK], const S (&dM)[KT], S (&f)[4]) {
  S E = S(0), OX = S(0), OY = S(0), OXY = S(0);
#pragma unroll
  for (int k = 0; k < KT; ++k) {
    const int ax = mono_ax(k), ay = mono_ay(k);
    if (!ax && !ay) E = fma(h[k], dM[k], E);
    else if (ax && !ay) OX = fma(h[k], dM[k], OX);
    else if (!ax && ay) OY = fma(h[k], dM[k], OY);
    else OXY = fma(h[k], dM[k], OXY);
  }
  const S A = E + OXY, B = E - OXY, C = OX + OY, D = OX - OY;
  f[0] = A + C; f[1] = B - D; f[2] = B + D; f[3] = A - C;
}

// ... of a rest population (its row has only px- and py-even entries) ...
template <typename S, int KT>
__device__ __forceinline__ S feq_rest(const S (&h)[kMaxK], const S (&dM)[KT]) {
  S E = S(0);
#pragma unroll
  for (int k = 0; k < KT; ++k)
    if (!mono_ax(k) && !mono_ay(k)) E = fma(h[k], dM[k], E);
  return E;
}

// ... and of the four members (p, 0), (-p, 0), (0, p), (0, -p) (the row of
// (p, 0) has no py-odd entries).
template <typename S, int KT>
__device__ __forceinline__ void feq_orbit4(const S (&h)[kMaxK], const S (&dM)[KT], S (&f)[4]) {
  S E = S(0), OX = S(0), Eb = S(0), OYb = S(0);
#pragma unroll
  for (int k = 0; k < KT; ++k) {
    const int ax = mono_ax(k), ay = mono_ay(k);
    if (ay) continue;
    const S t = dM[mono_swap(k)];
    if (!ax) { E = fma(h[k], dM[k], E); Eb = fma(h[k], t, Eb); }
    else { OX = fma(h[k], dM[k], OX); OYb = fma(h[k], t, OYb); }
  }
  f[0] = E + OX; f[1] = E - OX; f[2] = Eb + OYb; f[3] = Eb - OYb;
}

// Steps 2-8 of one cell from its streamed populations g: moments, Landau
// solve, equilibrium, relaxation, store (interior and halo images).
// DYN: plane offsets from the run-time plane size (tables shared by grids
// of different sizes), otherwise from the per-handle table tb.pl.
// MOUT (FP32 storage): also write the cell's macroscopic state to macro
// (planes of kMacroPlanes; n is NaN where the update was non-physical).
// FW (with SYM): the orbit-symmetric evaluation with the force term and the
// equilibrium walls of the generic path.
template <typename S, int QT, bool EX, int KT, bool SYM = false, bool DYN = false, bool MOUT = false, bool FW = false>
__device__ __forceinline__ void collide_store(const Tables<S>& tb, const Scalars& s, S (&g)[QT],
                                              S* __restrict__ fout, const S* __restrict__ tau_field,
                                              unsigned long long* status, int x, int y,
                                              float* __restrict__ macro = nullptr) {
  const long long si = sidx(s, x, y);
  const int Qn = EX ? QT : s.Q;
  S mm[9];
  if constexpr (SYM) moments_sym<S, QT>(tb, g, mm);
  else moments9<S, QT, EX>(tb, s.Q, g, mm);
  Macro M = landau<S, SYM ? (Orbits<QT>::massless ? 1 : 0) : -1>(s, mm);
  // no physical Landau frame: counted, and left unrelaxed (Omega = 0); the
  // frame is replaced by the reference state so that the equilibrium and
  // Omega stay finite (0 * NaN would not leave the populations unchanged)
  if (!M.ok) atomicAdd(status, 1ULL);
  unphysical_to_reference<S>(s, M);
  if constexpr (MOUT && sizeof(S) == 4) {
    const int cell = y * s.nx + x;
    const int nc = s.ncell;
    macro[cell] = M.ok ? M.fn : __int_as_float(0x7fc00000);
    macro[nc + cell] = M.fT;
    macro[2 * nc + cell] = M.fU0;
    macro[3 * nc + cell] = M.fUx;
    macro[4 * nc + cell] = M.fUy;
    macro[5 * nc + cell] = M.fdn;
    macro[6 * nc + cell] = M.fdT;
    macro[7 * nc + cell] = M.feps;
  }
  S dM[KT];
  eq_moments_of<S, KT>(s, M, dM);
  const S inv_tau = qdiv(S(1), local_tau<S>(s, tau_field, y * s.nx + x, M));
  S U0, Ux, Uy;
  if constexpr (sizeof(S) == 4) { U0 = M.fU0; Ux = M.fUx; Uy = M.fUy; }
  else { U0 = M.U0; Ux = M.Ux; Uy = M.Uy; }
  const S kt = M.ok ? inv_tau : S(0);
  S* __restrict__ obase = fout + si;
  auto plane_of = [&](int i) { return DYN ? i * s.iplane : tb.pl[i]; };
  // step 8: f* = f + Omega_i (f^eq - f), Omega_i = p_i.U / (p_i^0 tau) = (U^0 - v_i . U) / tau
  auto relax = [&](int i, S feq, S om) {
    g[i] = fma(om, feq - g[i], g[i]);
    obase[plane_of(i)] = g[i];
  };
  // Forcing scheme B (Sec. 4.4), gravity-like force K = (g.p, p^0 g):
  // F_i = (m/T) f^eq_i (U^0 g.v_i - g.U), with the full f^eq (the stored
  // shift f_ref added back).  Equilibrium walls (first and last column):
  // the cell keeps f^eq(n, U = (1, 0, 0), T_w) instead, T_w the prescribed
  // wall temperature or the cell's own T.
  S cf = S(0), gx = S(0), gy = S(0), gU = S(0);
  bool wall = false;
  S dMw[KT];
  if (!SYM || FW) {
    if (s.force && M.ok) {
      if constexpr (sizeof(S) == 4) { cf = __fdividef(s.f_m, M.fT); gx = s.f_gx; gy = s.f_gy; }
      else { cf = s.m / M.T; gx = s.gx; gy = s.gy; }
      gU = gx * Ux + gy * Uy;
    }
    wall = s.boundary == 2 && (x == 0 || x == s.nx - 1) && M.ok;
    if (wall) {
      const int side = x == 0 ? 0 : 1;
      if constexpr (sizeof(S) == 4) {
        const bool fix = s.f_wall_T[side] > 0.f;
        const float Tw = fix ? s.f_wall_T[side] : M.fT;
        const float dTw = fix ? (float)(s.wall_T[side] - s.T_ref) : M.fdT;
        eq_moments<S, KT>(M.fdn, dTw, M.fn, Tw, S(1), S(0), S(0), s.f_m, s.f_n_ref, s.f_T_ref, dMw);
      } else {
        const double Tw = s.wall_T[side] > 0.0 ? s.wall_T[side] : M.T;
        eq_moments<S, KT>(M.n - s.n_ref, Tw - s.T_ref, M.n, Tw, S(1), S(0), S(0), s.m, s.n_ref, s.T_ref, dMw);
      }
    }
  }
  if constexpr (SYM) {
    using O = Orbits<QT>;
    const S U0k = U0 * kt, Uxk = Ux * kt, Uyk = Uy * kt;
    if constexpr (FW) {
      // a wall cell evaluates the orbits at the wall state and stores f^eq
      // unrelaxed; elsewhere the force term follows the relaxation
      if (wall) {
#pragma unroll
        for (int k = 0; k < KT; ++k) dM[k] = dMw[k];
      }
    }
    auto relax_sym = [&](int i, S feq, S om) {
      if constexpr (FW) {
        if (wall) {
          g[i] = feq;
        } else {
          g[i] = fma(om, feq - g[i], g[i]);
          if (cf != S(0)) g[i] = fma(cf * (feq + tb.fref[i]), U0 * (gx * tb.vx[i] + gy * tb.vy[i]) - gU, g[i]);
        }
        obase[plane_of(i)] = g[i];
      } else {
        relax(i, feq, om);
      }
    };
    // Omega of a sign quartet with base velocity (va, vb), members (+,+), (-,+), (+,-), (-,-)
    auto quartet_om = [&](S va, S vb, S (&om)[4]) {
      const S X = Uxk * va, Y = Uyk * vb;
      const S M1 = U0k - Y, M2 = U0k + Y;
      om[0] = M1 - X; om[1] = M1 + X; om[2] = M2 - X; om[3] = M2 + X;
    };
#pragma unroll
    for (int o = 0; o < O::n8; ++o) {
      const int i0 = 8 * o;
      S f[8], oa[4], ob[4];
      feq_orbit8<S, KT>(tb.H[i0], dM, f);
      quartet_om(tb.vx[i0], tb.vy[i0], oa);
      quartet_om(tb.vx[i0 + 4], tb.vy[i0 + 4], ob);
#pragma unroll
      for (int m = 0; m < 4; ++m) relax_sym(i0 + m, f[m], oa[m]);
#pragma unroll
      for (int m = 0; m < 4; ++m) relax_sym(i0 + 4 + m, f[4 + m], ob[m]);
    }
#pragma unroll
    for (int o = 0; o < O::n4; ++o) {
      const int i0 = OrbitStart<QT>::axis + 4 * o;
      S f[4];
      feq_orbit4<S, KT>(tb.H[i0], dM, f);
      const S X = Uxk * tb.vx[i0], Y = Uyk * tb.vx[i0];   // members (v,0), (-v,0), (0,v), (0,-v)
      relax_sym(i0, f[0], U0k - X);
      relax_sym(i0 + 1, f[1], U0k + X);
      relax_sym(i0 + 2, f[2], U0k - Y);
      relax_sym(i0 + 3, f[3], U0k + Y);
    }
#pragma unroll
    for (int o = 0; o < O::nd; ++o) {
      const int i0 = OrbitStart<QT>::diag + 4 * o;
      S f[4], om[4];
      feq_diag4<S, KT>(tb.H[i0], dM, f);
      quartet_om(tb.vx[i0], tb.vy[i0], om);
#pragma unroll
      for (int m = 0; m < 4; ++m) relax_sym(i0 + m, f[m], om[m]);
    }
#pragma unroll
    for (int o = 0; o < O::n1; ++o) {
      const int i0 = OrbitStart<QT>::rest + o;
      relax_sym(i0, feq_rest<S, KT>(tb.H[i0], dM), U0k);
    }
  } else {
#pragma unroll
    for (int i = 0; i < QT; ++i) {
      if (i < Qn) {
        if (wall) {
          S fw = S(0);
#pragma unroll
          for (int k = 0; k < KT; ++k) fw = fma(tb.H[i][k], dMw[k], fw);
          g[i] = fw;
          obase[plane_of(i)] = fw;
          continue;
        }
        S feq = S(0);
#pragma unroll
        for (int k = 0; k < KT; ++k) feq = fma(tb.H[i][k], dM[k], feq);
        relax(i, feq, kt * (U0 - Ux * tb.vx[i] - Uy * tb.vy[i]));
        if (cf != S(0)) {
          g[i] = fma(cf * (feq + tb.fref[i]), U0 * (gx * tb.vx[i] + gy * tb.vy[i]) - gU, g[i]);
          obase[plane_of(i)] = g[i];
        }
      }
    }
  }
  for_each_halo_image(s, x, y, [&](long long hi) {
    S* __restrict__ hb = fout + hi;
#pragma unroll
    for (int i = 0; i < QT; ++i)
      if (i < Qn) hb[plane_of(i)] = g[i];
  });
}

// One cell of the fused step (Sec. 6.2, steps 1-8): pull-gather from global
// memory, then collide_store.
template <typename S, int QT, bool EX, int KT, int MODE, bool DYN = false, bool NC = true, bool SYM = false,
          bool FW = false>
__device__ __forceinline__ void cell_update(const Tables<S>& tb, const Scalars& s, const S* __restrict__ fin,
                                            S* __restrict__ fout, const S* __restrict__ tau_field,
                                            unsigned long long* status, int x, int y) {
  S g[QT];
  gather<S, QT, EX, MODE, DYN, NC>(tb, s, fin, sidx(s, x, y), g);
  collide_store<S, QT, EX, KT, SYM, DYN, false, FW>(tb, s, g, fout, tau_field, status, x, y);
}

// FP32 storage: 1024 resident threads per SM (eight 32 x 4 blocks, at most
// 64 registers per thread) for the on-lattice pull -- the gather latency
// needs the resident warps; 32 x 4 blocks measured 3-7 % faster than 32 x 8.
// The bilinear pull (four taps per population) runs seven blocks at up to
// 72 registers: no spill, 1-2 % faster at 512^2 to 4096^2.  The generic
// (not orbit-symmetric) on-lattice kernels, which carry the force and wall
// terms, run six blocks at up to 80 registers instead of spilling 1.6 KB at
// 64.
// FP32 storage with more than 40 populations (order 3): the orbit-symmetric
// kernels run six blocks per SM up to 49 populations (80 registers, at most
// 8 bytes spilled) and five above (96 registers, no spills), the generic
// ones four (they spill kilobytes at 96).  Paper setup (Q = 49, 512^2):
// 31.0 / 29.2 / 27.2 us at four / five / six blocks.
// FP64 storage with more than 56 populations: 256 threads per SM, so that a
// cell's 64-72 doubles stay in registers (12 % faster at Q = 65); up to 56
// populations the spills of 512 threads cost less than the lost warps (3 %).
// SYM: orbit-symmetric moments and equilibrium (built-in massless stencils).
// MOUT: also write the macroscopic state (a.macro).
// FW: SYM with the force term and the equilibrium walls (six blocks, as the
// generic kernels that otherwise carry them).
template <typename S, int QT, int MODE, bool SYM, bool FW = false>
constexpr int step_threads_per_sm() {
  return sizeof(S) == 4 ? (QT <= 40 ? (MODE == kBilinear ? 896 : (SYM && !FW ? 1024 : 768))
                                    : (SYM ? (QT <= 49 ? 768 : 640) : 512))
                        : (QT <= 56 ? 512 : 256);
}

template <typename S, int QT, bool EX, int KT, int MODE, bool SYM, bool MOUT = false, bool FW = false>
__global__ void __launch_bounds__(kThreads, step_threads_per_sm<S, QT, MODE, SYM, FW>() / kThreads) k_step(const __grid_constant__ Tables<S> tb,
                                                   const __grid_constant__ StepArgs<S> a) {
  const int x = blockIdx.x * kBX + threadIdx.x;
  const int y = blockIdx.y * kBY + threadIdx.y;
  if (x >= a.s.nx || y >= a.s.ny) return;
  if constexpr (MOUT) {
    S g[QT];
    gather<S, QT, EX, MODE>(tb, a.s, a.fin, sidx(a.s, x, y), g);
    collide_store<S, QT, EX, KT, SYM, false, true>(tb, a.s, g, a.fout, a.tau_field, a.status, x, y, a.macro);
  } else {
    cell_update<S, QT, EX, KT, MODE, false, true, SYM, FW>(tb, a.s, a.fin, a.fout, a.tau_field, a.status, x, y);
  }
}

// Fields of f(t) (steps 1-4), optionally the raw moments.  Output planes are
// row-major [ny][nx].
template <typename S, int QT, bool EX, int MODE>
__global__ void __launch_bounds__(kThreads) k_fields(const __grid_constant__ Tables<S> tb,
                                                     const __grid_constant__ MomentArgs<S> a) {
  const int x = blockIdx.x * kBX + threadIdx.x;
  const int y = blockIdx.y * kBY + threadIdx.y;
  if (x >= a.s.nx || y >= a.s.ny) return;
  const long long si = sidx(a.s, x, y);
  S g[QT];
  if (a.gather) {
    gather<S, QT, EX, MODE>(tb, a.s, a.fin, si, g);
  } else {
#pragma unroll
    for (int i = 0; i < QT; ++i) g[i] = (i < a.s.Q) ? a.fin[i * a.s.plane + si] : S(0);
  }
  S mm[9];
  moments9<S, QT, EX>(tb, a.s.Q, g, mm);
  const Macro M = landau<S>(a.s, mm);
  if (!M.ok) atomicAdd(a.status, 1ULL);
  const long long P = a.s.ncell;
  const int cell = y * a.s.nx + x;
  double* o = a.out;
  o[0 * P + cell] = M.n;
  o[1 * P + cell] = M.Ux / M.U0;
  o[2 * P + cell] = M.Uy / M.U0;
  o[3 * P + cell] = M.T;
  o[4 * P + cell] = M.eps;
  if (a.want_moments) {
    o[5 * P + cell] = a.s.N0_ref + (double)mm[0];
    o[6 * P + cell] = (double)mm[1];
    o[7 * P + cell] = (double)mm[2];
    o[8 * P + cell] = a.s.T00_ref + (double)mm[3];
    o[9 * P + cell] = (double)mm[4];
    o[10 * P + cell] = (double)mm[5];
    o[11 * P + cell] = a.s.Tii_ref + (double)mm[6];
    o[12 * P + cell] = (double)mm[7];
    o[13 * P + cell] = a.s.Tii_ref + (double)mm[8];
  }
}

// Initialisation f*(0) = f^eq(n, U, T) (Sec. 6.2), stored shifted, with halo images.
template <typename S, int KT>
__global__ void __launch_bounds__(kThreads) k_init(const __grid_constant__ Tables<S> tb,
                                                   const __grid_constant__ InitArgs<S> a) {
  const int x = blockIdx.x * kBX + threadIdx.x;
  const int y = blockIdx.y * kBY + threadIdx.y;
  if (x >= a.s.nx || y >= a.s.ny) return;
  const int cell = y * a.s.nx + x;
  const double ux = a.ux[cell], uy = a.uy[cell];
  const double u2 = ux * ux + uy * uy;
  const double n = a.n[cell], T = a.T[cell];
  const bool ok = (u2 < 1.0) && (n > 0.0) && (T > 0.0);
  if (!ok) atomicAdd(a.status, 1ULL);
  const double gam = ok ? 1.0 / sqrt(1.0 - u2) : 1.0;
  S dM[KT];
  eq_moments<S, KT>((S)(n - a.s.n_ref), (S)(T - a.s.T_ref), (S)n, (S)T, (S)gam, (S)(gam * ux),
                    (S)(gam * uy), (S)a.s.m, (S)a.s.n_ref, (S)a.s.T_ref, dM);
  const long long si = sidx(a.s, x, y);
  for (int i = 0; i < a.s.Q; ++i) {
    S feq = S(0);
#pragma unroll
    for (int k = 0; k < KT; ++k) feq = fma(tb.H[i][k], dM[k], feq);
    a.fout[i * a.s.plane + si] = feq;
    for_each_halo_image(a.s, x, y, [&](long long hi) { a.fout[i * a.s.plane + hi] = feq; });
  }
}

// Dispatch helpers --------------------------------------------------------

inline dim3 grid_for(const Scalars& s) { return dim3((s.nx + kBX - 1) / kBX, (s.ny + kBY - 1) / kBY); }
inline dim3 block_dim() { return dim3(kBX, kBY); }

// QT: population count of the instantiation; EX: the stencil has exactly QT
// populations (no per-population bounds test), otherwise Q <= QT at run time.
template <typename S, int QT, bool EX, int KT, bool SYM = false, bool MOUT = false, bool FW = false>
cudaError_t launch_step_q(const Tables<S>& tb, const StepArgs<S>& a, int mode, cudaStream_t st) {
  if (mode == kOnLattice) k_step<S, QT, EX, KT, kOnLattice, SYM, MOUT, FW><<<grid_for(a.s), block_dim(), 0, st>>>(tb, a);
  else k_step<S, QT, EX, KT, kBilinear, SYM, MOUT, FW><<<grid_for(a.s), block_dim(), 0, st>>>(tb, a);
  return cudaGetLastError();
}

template <typename S, int QT, bool EX>
cudaError_t launch_fields_q(const Tables<S>& tb, const MomentArgs<S>& a, int mode, cudaStream_t st) {
  if (mode == kOnLattice) k_fields<S, QT, EX, kOnLattice><<<grid_for(a.s), block_dim(), 0, st>>>(tb, a);
  else k_fields<S, QT, EX, kBilinear><<<grid_for(a.s), block_dim(), 0, st>>>(tb, a);
  return cudaGetLastError();
}

template <typename S, int KT>
cudaError_t launch_init_k(const Tables<S>& tb, const InitArgs<S>& a, cudaStream_t st) {
  k_init<S, KT><<<grid_for(a.s), block_dim(), 0, st>>>(tb, a);
  return cudaGetLastError();
}

}  // namespace rlbm
