// Templates of the fused RLBM kernels: pull-stream + collide (Sec. 6.2 of
// arXiv:1909.04502), initialisation to equilibrium, and the macroscopic
// field extraction.  Instantiated per precision / order in step_o2.cu and
// step_o3.cu.
#pragma once
#include "kernels.cuh"

namespace rlbm {

constexpr int kThreads = 256;

// kernel parameters are limited to 32764 bytes
static_assert(sizeof(Tables<double>) + sizeof(MomentArgs<double>) <= 32764, "kernel parameter space");

// ---------------------------------------------------------------------------
// Step 1 of the update: streaming by pull (Eq. discrete-rbe, left side).
// On-lattice: f_i(x) = f*_i(x - n_i).  Bilinear: f_i(x) = sum_ab W_ab
// f*_i(x + o_i + (a, b)) (off-lattice reading; taps and weights per
// population in the tables).  Periodic in y always; periodic or clamped
// (free-flow) in x.
// ---------------------------------------------------------------------------
template <typename S, int QT, int MODE>
__device__ __forceinline__ void gather(const Tables<S>& tb, const Scalars& s,
                                       const S* __restrict__ fin, int x, int y, S (&g)[QT]) {
#pragma unroll
  for (int i = 0; i < QT; ++i) {
    g[i] = S(0);
    if (i < s.Q) {
      const S* __restrict__ pl = fin + (long long)i * s.plane;
      if constexpr (MODE == kOnLattice) {
        int ys = y + tb.syp[i];
        ys -= (ys >= s.ny) ? s.ny : 0;
        int xs;
        if (s.boundary == 0) {
          xs = x + tb.sxp[i];
          xs -= (xs >= s.nx) ? s.nx : 0;
        } else {
          xs = min(max(x + tb.sxr[i], 0), s.nx - 1);
        }
        g[i] = __ldg(pl + ys * s.nx + xs);
      } else {
        int y0 = y + tb.oyp[i];
        y0 -= (y0 >= s.ny) ? s.ny : 0;
        int y1 = y0 + 1;
        y1 -= (y1 >= s.ny) ? s.ny : 0;
        int x0, x1;
        if (s.boundary == 0) {
          x0 = x + tb.oxp[i];
          x0 -= (x0 >= s.nx) ? s.nx : 0;
          x1 = x0 + 1;
          x1 -= (x1 >= s.nx) ? s.nx : 0;
        } else {
          x0 = min(max(x + tb.oxr[i], 0), s.nx - 1);
          x1 = min(max(x + tb.oxr[i] + 1, 0), s.nx - 1);
        }
        S v = tb.bw[i][0] * __ldg(pl + y0 * s.nx + x0);
        v = fma(tb.bw[i][1], __ldg(pl + y0 * s.nx + x1), v);
        v = fma(tb.bw[i][2], __ldg(pl + y1 * s.nx + x0), v);
        v = fma(tb.bw[i][3], __ldg(pl + y1 * s.nx + x1), v);
        g[i] = v;
      }
    }
  }
}

// Step 1: N^a = sum_i f_i p_i^a, T^ab = sum_i f_i p_i^a p_i^b (of the
// stored, possibly shifted, populations).
template <typename S, int QT>
__device__ __forceinline__ void moments9(const Tables<S>& tb, int Q, const S (&g)[QT], S (&mm)[9]) {
#pragma unroll
  for (int j = 0; j < 9; ++j) mm[j] = S(0);
#pragma unroll
  for (int i = 0; i < QT; ++i) {
    if (i < Q) {
#pragma unroll
      for (int j = 0; j < 9; ++j) mm[j] = fma(g[i], tb.c[i][j], mm[j]);
    }
  }
}

// Steps 2-4 in FP64: Landau frame eps U^a = T^ab U_b (largest eigenvalue of
// the mixed tensor T^a_b, timelike eigenvector, Sec. 4), n = U_a N^a, T from
// eps/n = T (G_2(m/T) - 1) (Eq. eos-ddim), inverted in closed form for d = 2.
//
// The eigenvalue is the largest root of p(l) = det(A - l I),
//   p(l) = a D - s^2 c - t^2 b + 2 r s t,  a = T00 - l, b = Txx + l,
//   c = Tyy + l, D = b c - r^2, s = T0x, t = T0y, r = Txy,
// and its eigenvector is v = (D, s c - r t, t b - r s).  A first guess comes
// from the ideal-fluid closed form (P = kappa eps) in FP32, refined by FP32
// Newton steps; the root is then polished by Newton steps whose residual
// p(l) is evaluated in FP64 (one step for FP32 storage, two in FP64 mode),
// and v, its normalisation, n and T are evaluated in FP64.
template <typename S>
__device__ __forceinline__ Macro landau(const Scalars& sc, const S (&mm)[9]) {
  constexpr bool F32 = sizeof(S) == 4;
  const double N0 = sc.N0_ref + (double)mm[0];
  const double Nx = (double)mm[1], Ny = (double)mm[2];
  const double T00 = sc.T00_ref + (double)mm[3];
  const double T0x = (double)mm[4], T0y = (double)mm[5];
  const double Txx = sc.Tii_ref + (double)mm[6];
  const double Txy = (double)mm[7];
  const double Tyy = sc.Tii_ref + (double)mm[8];

  float fE, fs, ft, fr, fxx, fyy;
  if constexpr (F32) {
    fE = (float)sc.T00_ref + (float)mm[3];
    fxx = (float)sc.Tii_ref + (float)mm[6];
    fyy = (float)sc.Tii_ref + (float)mm[8];
    fs = (float)mm[4]; ft = (float)mm[5]; fr = (float)mm[7];
  } else {
    fE = (float)T00; fxx = (float)Txx; fyy = (float)Tyy;
    fs = (float)T0x; ft = (float)T0y; fr = (float)Txy;
  }
  const float k = sc.kappa_guess;
  const float M2 = fs * fs + ft * ft;
  const float disc = (1.f - k) * (1.f - k) * fE * fE + 4.f * k * (fE * fE - M2);
  float lam = (-(1.f - k) * fE + sqrtf(fmaxf(disc, 0.f))) / (2.f * k);
  float dpf = 1.f;
#pragma unroll
  for (int it = 0; it < 3; ++it) {
    float a = fE - lam, b = fxx + lam, c = fyy + lam;
    float D = b * c - fr * fr;
    float p = a * D - fs * fs * c - ft * ft * b + 2.f * fr * fs * ft;
    dpf = -D + a * (b + c) - M2;
    lam -= p / dpf;
  }
  double L = (double)lam;
#pragma unroll
  for (int it = 0; it < (F32 ? 1 : 2); ++it) {
    double a = T00 - L, b = Txx + L, c = Tyy + L;
    double D = fma(b, c, -Txy * Txy);
    double p = fma(a, D, fma(-T0x * T0x, c, fma(-T0y * T0y, b, 2.0 * Txy * T0x * T0y)));
    if constexpr (F32) {
      L -= (double)((float)p / dpf);
    } else {
      double dp = -D + a * (b + c) - T0x * T0x - T0y * T0y;
      L -= p / dp;
    }
  }
  const double b = Txx + L, c = Tyy + L;
  const double D = fma(b, c, -Txy * Txy);
  const double vx = fma(T0x, c, -Txy * T0y);
  const double vy = fma(T0y, b, -Txy * T0x);
  const double nrm2 = fma(D, D, -fma(vx, vx, vy * vy));
  double inv;
  if constexpr (F32) {
    double y0 = (double)rsqrtf((float)nrm2);
    double e = fma(-nrm2, y0 * y0, 1.0);
    inv = fma(0.5 * y0, e, y0);
  } else {
    inv = rsqrt(nrm2);
  }
  Macro M;
  M.eps = L;
  M.U0 = D * inv;
  M.Ux = vx * inv;
  M.Uy = vy * inv;
  M.n = fma(M.U0, N0, -fma(M.Ux, Nx, M.Uy * Ny));
  const double m = sc.m;
  if (m == 0.0) {
    // eps = 2 P = 2 n T
    if constexpr (F32) {
      float rh = 0.5f / (float)M.n;
      double T = L * (double)rh;
      double e = fma(-2.0 * M.n, T, L);
      M.T = fma((double)rh, e, T);
    } else {
      M.T = 0.5 * L / M.n;
    }
  } else {
    // n q(T) = 2 n T^2 + (2 m n - eps) T + m (m n - eps) = 0, positive root
    if constexpr (F32) {
      float fn = (float)M.n, fl = (float)L, fm = (float)m;
      float e = fl / fn;
      float T0 = 0.25f * ((e - 2.f * fm) + sqrtf(fmaxf(e * e + 4.f * e * fm - 4.f * fm * fm, 0.f)));
      double Td = (double)T0;
      double q = fma(fma(2.0 * M.n, Td, fma(2.0 * m, M.n, -L)), Td, m * fma(m, M.n, -L));
      float dq = 4.f * fn * T0 + 2.f * fm * fn - fl;
      M.T = Td - (double)((float)q / dq);
    } else {
      double e = L / M.n;
      M.T = 0.25 * ((e - 2.0 * m) + sqrt(fma(e, e, 4.0 * m * (e - m))));
    }
  }
  M.ok = (D > 0.0) && (nrm2 > 0.0) && (M.n > 0.0) && (M.T > 0.0) && (L > 0.0) && isfinite(M.T) &&
         isfinite(M.U0);
  return M;
}

// Step 5, moment side: dM = M(n, U, T) - M(n_ref, e0, T_ref) for the basis of
// setup.h (p0^e px^a py^b, e + a + b <= N), using the App. B moments
//   <1> = n/(m+T), <p^a> = n U^a, <p^a p^b> = n (r2 U^a U^b - T eta^ab),
//   <p^a p^b p^c> = n (r3 U^a U^b U^c - T r2 (eta^ab U^c + eta^ac U^b + eta^bc U^a)),
//   r2 = (m^2 + 3mT + 3T^2)/(m+T), r3 = (m^3 + 6m^2 T + 15 m T^2 + 15 T^3)/(m+T).
// The differences from the reference are rearranged so that the FP32 result
// is accurate relative to dM itself (only dn and dT are formed in FP64).
template <typename S, int KT>
__device__ __forceinline__ void eq_moments(const Scalars& sc, const Macro& M, S (&dM)[KT]) {
  const S dn = (S)(M.n - sc.n_ref), dT = (S)(M.T - sc.T_ref);
  const S n = (S)M.n, T = (S)M.T, U0 = (S)M.U0, Ux = (S)M.Ux, Uy = (S)M.Uy;
  const S m = (S)sc.m, nr = (S)sc.n_ref, Tr = (S)sc.T_ref;
  const S U0m1 = (Ux * Ux + Uy * Uy) / (U0 + S(1));
  const S mT = m + T, mTr = m + Tr;
  const S r2 = (m * m + S(3) * m * T + S(3) * T * T) / mT;
  const S D1 = (dn * mTr - nr * dT) / (mT * mTr);
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
    const S q2 = T * r2;
    const S r3 = (m * m * m + S(6) * m * m * T + S(15) * m * T * T + S(15) * T * T * T) / mT;
    const S Nh = dT * (m * (m * m + S(3) * m * (T + Tr) + S(3) * (T * T + T * Tr + Tr * Tr)) +
                       S(3) * T * Tr * (m + T + Tr));
    const S dh = Nh / (mT * mTr);
    const S D4 = dn * q2 * U0 + nr * (q2 * U0m1 + dh);
    const S nr3 = n * r3, nq2 = n * q2;
    dM[9] = nr3 * U0 * Ux * Ux + D4;
    dM[10] = nr3 * U0 * Ux * Uy;
    dM[11] = nr3 * U0 * Uy * Uy + D4;
    dM[12] = nr3 * Ux * Ux * Ux + S(3) * nq2 * Ux;
    dM[13] = nr3 * Ux * Ux * Uy + nq2 * Uy;
    dM[14] = nr3 * Ux * Uy * Uy + nq2 * Ux;
    dM[15] = nr3 * Uy * Uy * Uy + S(3) * nq2 * Uy;
  }
}

template <typename S>
__device__ __forceinline__ S local_tau(const Scalars& sc, const S* __restrict__ tau_field, int cell,
                                       const Macro& M) {
  if (sc.tau_mode == 1) return __ldg(tau_field + cell);
  if (sc.tau_mode == 2) return (S)(sc.tau_coef / M.T);   // step 7, eta/s fixed
  return (S)sc.tau;
}

// ---------------------------------------------------------------------------
// Fused step kernel: one thread per cell.
// ---------------------------------------------------------------------------
template <typename S, int QT, int KT, int MODE>
__global__ void __launch_bounds__(kThreads) k_step(const __grid_constant__ Tables<S> tb,
                                                   const __grid_constant__ StepArgs<S> a) {
  const int cell = blockIdx.x * kThreads + threadIdx.x;
  if (cell >= a.s.ncell) return;
  const int y = cell / a.s.nx;
  const int x = cell - y * a.s.nx;
  S g[QT];
  gather<S, QT, MODE>(tb, a.s, a.fin, x, y, g);
  S mm[9];
  moments9<S, QT>(tb, a.s.Q, g, mm);
  const Macro M = landau<S>(a.s, mm);
  if (!M.ok) atomicAdd(a.status, 1ULL);
  S dM[KT];
  eq_moments<S, KT>(a.s, M, dM);
  const S inv_tau = S(1) / local_tau<S>(a.s, a.tau_field, cell, M);
  const S U0 = (S)M.U0, Ux = (S)M.Ux, Uy = (S)M.Uy;
  const S keep = M.ok ? S(1) : S(0);
#pragma unroll
  for (int i = 0; i < QT; ++i) {
    if (i < a.s.Q) {
      S feq = S(0);
#pragma unroll
      for (int k = 0; k < KT; ++k) feq = fma(tb.H[i][k], dM[k], feq);
      // step 8: Omega_i = p_i.U / (p_i^0 tau) = (U^0 - v_i . U) / tau
      const S om = keep * (U0 - Ux * tb.vx[i] - Uy * tb.vy[i]) * inv_tau;
      a.fout[(long long)i * a.s.plane + cell] = fma(om, feq - g[i], g[i]);
    }
  }
}

// Fields of f(t) (steps 1-4), optionally the raw moments.
template <typename S, int QT, int MODE>
__global__ void __launch_bounds__(kThreads) k_fields(const __grid_constant__ Tables<S> tb,
                                                     const __grid_constant__ MomentArgs<S> a) {
  const int cell = blockIdx.x * kThreads + threadIdx.x;
  if (cell >= a.s.ncell) return;
  const int y = cell / a.s.nx;
  const int x = cell - y * a.s.nx;
  S g[QT];
  if (a.gather) {
    gather<S, QT, MODE>(tb, a.s, a.fin, x, y, g);
  } else {
#pragma unroll
    for (int i = 0; i < QT; ++i) g[i] = (i < a.s.Q) ? a.fin[(long long)i * a.s.plane + cell] : S(0);
  }
  S mm[9];
  moments9<S, QT>(tb, a.s.Q, g, mm);
  const Macro M = landau<S>(a.s, mm);
  if (!M.ok) atomicAdd(a.status, 1ULL);
  const long long P = a.s.plane;
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

// Initialisation f*(0) = f^eq(n, U, T) (Sec. 6.2), stored shifted.
template <typename S, int KT>
__global__ void __launch_bounds__(kThreads) k_init(const __grid_constant__ Tables<S> tb,
                                                   const __grid_constant__ InitArgs<S> a) {
  const int cell = blockIdx.x * kThreads + threadIdx.x;
  if (cell >= a.s.ncell) return;
  const double ux = a.ux[cell], uy = a.uy[cell];
  const double u2 = ux * ux + uy * uy;
  Macro M;
  M.n = a.n[cell];
  M.T = a.T[cell];
  M.ok = (u2 < 1.0) && (M.n > 0.0) && (M.T > 0.0);
  const double gam = M.ok ? 1.0 / sqrt(1.0 - u2) : 1.0;
  M.U0 = gam;
  M.Ux = gam * ux;
  M.Uy = gam * uy;
  M.eps = 0.0;
  if (!M.ok) atomicAdd(a.status, 1ULL);
  S dM[KT];
  eq_moments<S, KT>(a.s, M, dM);
  for (int i = 0; i < a.s.Q; ++i) {
    S feq = S(0);
#pragma unroll
    for (int k = 0; k < KT; ++k) feq = fma(tb.H[i][k], dM[k], feq);
    a.fout[(long long)i * a.s.plane + cell] = feq;
  }
}

// Dispatch helpers --------------------------------------------------------

inline int blocks_for(int ncell) { return (ncell + kThreads - 1) / kThreads; }

template <typename S, int QT, int KT>
cudaError_t launch_step_q(const Tables<S>& tb, const StepArgs<S>& a, int mode, cudaStream_t st) {
  const int nb = blocks_for(a.s.ncell);
  if (mode == kOnLattice) k_step<S, QT, KT, kOnLattice><<<nb, kThreads, 0, st>>>(tb, a);
  else k_step<S, QT, KT, kBilinear><<<nb, kThreads, 0, st>>>(tb, a);
  return cudaGetLastError();
}

template <typename S, int QT>
cudaError_t launch_fields_q(const Tables<S>& tb, const MomentArgs<S>& a, int mode, cudaStream_t st) {
  const int nb = blocks_for(a.s.ncell);
  if (mode == kOnLattice) k_fields<S, QT, kOnLattice><<<nb, kThreads, 0, st>>>(tb, a);
  else k_fields<S, QT, kBilinear><<<nb, kThreads, 0, st>>>(tb, a);
  return cudaGetLastError();
}

template <typename S, int KT>
cudaError_t launch_init_k(const Tables<S>& tb, const InitArgs<S>& a, cudaStream_t st) {
  k_init<S, KT><<<blocks_for(a.s.ncell), kThreads, 0, st>>>(tb, a);
  return cudaGetLastError();
}

}  // namespace rlbm
