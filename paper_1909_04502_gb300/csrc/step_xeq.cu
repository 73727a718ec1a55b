// Order-3 massive step with FP32 storage and an extended-precision
// equilibrium (Sec. 6.2, steps 5-8, with the polynomial Maxwell-Juttner
// expansion of Eq. mj-discrete-feq at N = 3).
//
// Why: f^eq - f_ref = H dM is a contraction whose terms are up to several
// hundred times larger than its result for m~ >= 10 (the columns of H for
// the scalar-like members <p0 - m>, <px px>, <py py> nearly cancel).  FP32
// moments dM carry a rounding of 2^-24 of each term, which the contraction
// turns into population errors above 1e-5 of max f.  Rounding a member of
// dM is not a consistent change of (n, U, T), so nothing cancels it.
//
// How: the macroscopic state (n, U, T and the differences dn, dT) comes from
// the FP32 Landau solve as in the plain FP32 step and is taken as exact;
// dM(n, U, T) is evaluated from it in float-float arithmetic (about 48
// bits, fpconv.cuh), m, n_ref and T_ref enter as pairs, and the contraction
// runs as a compensated dot product (the error-free product and sum of
// every term kept in a second accumulator, Ogita, Rump and Oishi's Dot2)
// over H split into hi + lo FP32 parts.  The equilibrium then matches the
// one from exact moments to about 1e-12 of max f; the populations keep the
// FP32 storage rounding of g = f - f_ref only.  Everything runs on the
// FP32 pipe.  Orbit-symmetric built-in stencils only (the table rows of an
// orbit are its first row with signs and swapped columns, as in
// step_impl.cuh).
#include "dispatch.h"
#include "step_impl.cuh"

namespace rlbm {

namespace {

__device__ __forceinline__ ff F(float x) { return {x, 0.f}; }
__device__ __forceinline__ ff operator+(ff a, ff b) { return ff_add(a, b); }
__device__ __forceinline__ ff operator-(ff a, ff b) { return ff_sub(a, b); }
__device__ __forceinline__ ff operator*(ff a, ff b) { return ff_mul(a, b); }
__device__ __forceinline__ ff operator*(float a, ff b) { return ff_mulf(a, b); }

// 1 / b: FP32 quotient, then one correction from the float-float residual
// 1 - q b.
__device__ __forceinline__ ff ff_inv(ff b) {
  const float q1 = __fdividef(1.f, b.hi);
  const ff r = ff_sub(F(1.f), ff_mulf(q1, b));
  return ff_fast(q1, __fdividef(r.hi + r.lo, b.hi));
}

__device__ __forceinline__ ff ff_div(ff a, ff b) {
  const float q1 = __fdividef(a.hi, b.hi);
  const ff r = ff_sub(a, ff_mulf(q1, b));
  return ff_fast(q1, __fdividef(r.hi + r.lo, b.hi));
}

// dM = M(n, U, T) - M(n_ref, rest, T_ref) of the order-3 basis (the
// members and closed forms of eq_moments in step_impl.cuh, K = 16), every
// operation in float-float.
__device__ __forceinline__ void eq_moments_xeq(const Macro& M, const XeqTables& xq, ff (&dM)[16]) {
  const ff m = {xq.m[0], xq.m[1]}, nr = {xq.n_ref[0], xq.n_ref[1]}, Tr = {xq.T_ref[0], xq.T_ref[1]};
  const ff n = F(M.fn), T = F(M.fT), dn = F(M.fdn), dT = F(M.fdT);
  const ff U0 = F(M.fU0), Ux = F(M.fUx), Uy = F(M.fUy);
  const ff U0m1 = ff_div(Ux * Ux + Uy * Uy, U0 + F(1.f));       // U0 - 1 without cancellation
  const ff mT = m + T, mTr = m + Tr;
  const ff iden = ff_inv(mT * mTr), imT = iden * mTr;          // 1/((m+T)(m+T_ref)), 1/(m+T)
  const ff mm = m * m, mTp = m * T, TT = T * T;
  const ff r2 = (mm + 3.f * mTp + 3.f * TT) * imT;
  const ff D3 = dn * T + nr * dT;
  const ff nr2 = n * r2;
  dM[0] = (dn * mTr - nr * dT) * iden;
  dM[2] = n * Ux;
  dM[3] = n * Uy;
  dM[6] = nr2 * (Ux * Ux) + D3;
  dM[7] = nr2 * (Ux * Uy);
  dM[8] = nr2 * (Uy * Uy) + D3;
  const ff q2 = T * r2;
  const ff r3 = (mm * m + 6.f * (mm * T) + 15.f * (mTp * T) + 15.f * (TT * T)) * imT;
  const ff c2 = (2.f * m + 3.f * T) * imT;
  const ff c3 = 3.f * (mm + 4.f * mTp + 5.f * TT) * imT;
  const ff A2 = r2 * U0m1 + T * c2;
  const ff A3 = r3 * U0m1 + T * c3;
  dM[1] = n * U0m1 + (dn * T * mTr + nr * m * dT) * iden;
  dM[4] = n * Ux * A2;
  dM[5] = n * Uy * A2;
  const ff TTr = T * Tr, TpTr = T + Tr;
  const ff Nh = dT * (2.f * mm * TpTr + 2.f * (m * TTr) + 3.f * m * (TT + TTr + Tr * Tr) + 3.f * TTr * TpTr);
  const ff D5 = n * T * r2 * U0m1 + dn * TT * c2 + nr * Nh * iden;
  const ff nA3 = n * A3, nr3 = n * r3, nq2 = n * q2;
  dM[9] = nA3 * (Ux * Ux) + D5;
  dM[10] = nA3 * (Ux * Uy);
  dM[11] = nA3 * (Uy * Uy) + D5;
  dM[12] = nr3 * (Ux * Ux) * Ux + 3.f * (nq2 * Ux);
  dM[13] = nr3 * (Ux * Ux) * Uy + nq2 * Uy;
  dM[14] = nr3 * Ux * (Uy * Uy) + nq2 * Ux;
  dM[15] = nr3 * (Uy * Uy) * Uy + 3.f * (nq2 * Uy);
}

// Compensated accumulation of sum_k (h_k + hl_k)(x_k.hi + x_k.lo): s holds
// the FP32 sum of the products h_k x_k.hi, c the exact rounding errors of
// those products and sums plus the small cross terms.
struct acc2 {
  float s = 0.f, c = 0.f;
};

__device__ __forceinline__ void acc_term(acc2& a, float h, float hl, const ff& x) {
  const ff p = ff_prod(h, x.hi);
  const ff t = ff_sum(a.s, p.hi);
  a.s = t.hi;
  a.c += t.lo + p.lo;
  a.c = fmaf(h, x.lo, a.c);
  a.c = fmaf(hl, x.hi, a.c);
}

__device__ __forceinline__ ff acc_ff(const acc2& a) { return ff_sum(a.s, a.c); }

__device__ __forceinline__ float ff_round(ff a) { return a.hi + a.lo; }

// The four parity-class sums E, OX, OY, OXY of a row (and of its swapped
// row: px and py exponents exchanged), then the members' signs as in
// feq_orbit8 / feq_orbit4 / feq_diag4 / feq_rest of step_impl.cuh.
template <int KT>
__device__ __forceinline__ void feq_orbit8_xeq(const float (&h)[kMaxK], const float (&hl)[kMaxK],
                                               const ff (&dM)[KT], float (&f)[8]) {
  acc2 E, OX, OY, OXY, Eb, OXb, OYb, OXYb;
#pragma unroll
  for (int k = 0; k < KT; ++k) {
    const int ax = mono_ax(k), ay = mono_ay(k);
    const ff& t = dM[mono_swap(k)];
    if (!ax && !ay) { acc_term(E, h[k], hl[k], dM[k]); acc_term(Eb, h[k], hl[k], t); }
    else if (ax && !ay) { acc_term(OX, h[k], hl[k], dM[k]); acc_term(OYb, h[k], hl[k], t); }
    else if (!ax && ay) { acc_term(OY, h[k], hl[k], dM[k]); acc_term(OXb, h[k], hl[k], t); }
    else { acc_term(OXY, h[k], hl[k], dM[k]); acc_term(OXYb, h[k], hl[k], t); }
  }
  {
    const ff e = acc_ff(E), ox = acc_ff(OX), oy = acc_ff(OY), oxy = acc_ff(OXY);
    const ff A = e + oxy, B = e - oxy, C = ox + oy, D = ox - oy;
    f[0] = ff_round(A + C); f[1] = ff_round(B - D); f[2] = ff_round(B + D); f[3] = ff_round(A - C);
  }
  {
    const ff e = acc_ff(Eb), ox = acc_ff(OXb), oy = acc_ff(OYb), oxy = acc_ff(OXYb);
    const ff A = e + oxy, B = e - oxy, C = ox + oy, D = ox - oy;
    f[4] = ff_round(A + C); f[5] = ff_round(B - D); f[6] = ff_round(B + D); f[7] = ff_round(A - C);
  }
}

template <int KT>
__device__ __forceinline__ void feq_diag4_xeq(const float (&h)[kMaxK], const float (&hl)[kMaxK],
                                              const ff (&dM)[KT], float (&f)[4]) {
  acc2 E, OX, OY, OXY;
#pragma unroll
  for (int k = 0; k < KT; ++k) {
    const int ax = mono_ax(k), ay = mono_ay(k);
    if (!ax && !ay) acc_term(E, h[k], hl[k], dM[k]);
    else if (ax && !ay) acc_term(OX, h[k], hl[k], dM[k]);
    else if (!ax && ay) acc_term(OY, h[k], hl[k], dM[k]);
    else acc_term(OXY, h[k], hl[k], dM[k]);
  }
  const ff e = acc_ff(E), ox = acc_ff(OX), oy = acc_ff(OY), oxy = acc_ff(OXY);
  const ff A = e + oxy, B = e - oxy, C = ox + oy, D = ox - oy;
  f[0] = ff_round(A + C); f[1] = ff_round(B - D); f[2] = ff_round(B + D); f[3] = ff_round(A - C);
}

template <int KT>
__device__ __forceinline__ void feq_orbit4_xeq(const float (&h)[kMaxK], const float (&hl)[kMaxK],
                                               const ff (&dM)[KT], float (&f)[4]) {
  acc2 E, OX, Eb, OYb;
#pragma unroll
  for (int k = 0; k < KT; ++k) {
    const int ax = mono_ax(k), ay = mono_ay(k);
    if (ay) continue;
    const ff& t = dM[mono_swap(k)];
    if (!ax) { acc_term(E, h[k], hl[k], dM[k]); acc_term(Eb, h[k], hl[k], t); }
    else { acc_term(OX, h[k], hl[k], dM[k]); acc_term(OYb, h[k], hl[k], t); }
  }
  const ff e = acc_ff(E), ox = acc_ff(OX), eb = acc_ff(Eb), oyb = acc_ff(OYb);
  f[0] = ff_round(e + ox); f[1] = ff_round(e - ox); f[2] = ff_round(eb + oyb); f[3] = ff_round(eb - oyb);
}

template <int KT>
__device__ __forceinline__ float feq_rest_xeq(const float (&h)[kMaxK], const float (&hl)[kMaxK],
                                              const ff (&dM)[KT]) {
  acc2 E;
#pragma unroll
  for (int k = 0; k < KT; ++k)
    if (!mono_ax(k) && !mono_ay(k)) acc_term(E, h[k], hl[k], dM[k]);
  return ff_round(acc_ff(E));
}

// Steps 1-8 of one cell: the pull, moments, Landau frame and relaxation as
// in the plain FP32 step (gather, moments_sym, landau, collide_store of
// step_impl.cuh), the equilibrium as above.  512 resident threads per SM.
template <int QT, int MODE>
__global__ void __launch_bounds__(kThreads, 512 / kThreads) k_step_xeq(const __grid_constant__ Tables<float> tb,
                                                                        const __grid_constant__ XeqTables xq,
                                                                        const __grid_constant__ StepArgs<float> a) {
  using O = Orbits<QT>;
  const Scalars& s = a.s;
  const int x = blockIdx.x * kBX + threadIdx.x;
  const int y = blockIdx.y * kBY + threadIdx.y;
  if (x >= s.nx || y >= s.ny) return;
  const long long si = sidx(s, x, y);
  float g[QT];
  gather<float, QT, true, MODE>(tb, s, a.fin, si, g);
  float mm[9];
  moments_sym<float, QT>(tb, g, mm);
  Macro M = landau<float, 0>(s, mm);
  // no physical Landau frame: counted, left unrelaxed (as in collide_store)
  if (!M.ok) atomicAdd(a.status, 1ULL);
  unphysical_to_reference<float>(s, M);
  ff dM[16];
  eq_moments_xeq(M, xq, dM);
  const float inv_tau = __fdividef(1.f, local_tau<float>(s, a.tau_field, y * s.nx + x, M));
  const float kt = M.ok ? inv_tau : 0.f;
  const float U0k = M.fU0 * kt, Uxk = M.fUx * kt, Uyk = M.fUy * kt;
  float* __restrict__ obase = a.fout + si;
  // step 8: f* = f + Omega_i (f^eq - f), Omega_i = (U^0 - v_i . U) / tau
  auto relax = [&](int i, float feq, float om) {
    g[i] = fmaf(om, feq - g[i], g[i]);
    obase[tb.pl[i]] = g[i];
  };
  auto quartet_om = [&](float va, float vb, float (&om)[4]) {
    const float X = Uxk * va, Y = Uyk * vb;
    const float M1 = U0k - Y, M2 = U0k + Y;
    om[0] = M1 - X; om[1] = M1 + X; om[2] = M2 - X; om[3] = M2 + X;
  };
#pragma unroll
  for (int o = 0; o < O::n8; ++o) {
    const int i0 = 8 * o;
    float f[8], oa[4], ob[4];
    feq_orbit8_xeq<16>(tb.H[i0], xq.Hl[i0], dM, f);
    quartet_om(tb.vx[i0], tb.vy[i0], oa);
    quartet_om(tb.vx[i0 + 4], tb.vy[i0 + 4], ob);
#pragma unroll
    for (int m = 0; m < 4; ++m) relax(i0 + m, f[m], oa[m]);
#pragma unroll
    for (int m = 0; m < 4; ++m) relax(i0 + 4 + m, f[4 + m], ob[m]);
  }
#pragma unroll
  for (int o = 0; o < O::n4; ++o) {
    const int i0 = OrbitStart<QT>::axis + 4 * o;
    float f[4];
    feq_orbit4_xeq<16>(tb.H[i0], xq.Hl[i0], dM, f);
    const float X = Uxk * tb.vx[i0], Y = Uyk * tb.vx[i0];   // members (v,0), (-v,0), (0,v), (0,-v)
    relax(i0, f[0], U0k - X);
    relax(i0 + 1, f[1], U0k + X);
    relax(i0 + 2, f[2], U0k - Y);
    relax(i0 + 3, f[3], U0k + Y);
  }
#pragma unroll
  for (int o = 0; o < O::nd; ++o) {
    const int i0 = OrbitStart<QT>::diag + 4 * o;
    float f[4], om[4];
    feq_diag4_xeq<16>(tb.H[i0], xq.Hl[i0], dM, f);
    quartet_om(tb.vx[i0], tb.vy[i0], om);
#pragma unroll
    for (int m = 0; m < 4; ++m) relax(i0 + m, f[m], om[m]);
  }
#pragma unroll
  for (int o = 0; o < O::n1; ++o) {
    const int i0 = OrbitStart<QT>::rest + o;
    relax(i0, feq_rest_xeq<16>(tb.H[i0], xq.Hl[i0], dM), U0k);
  }
  for_each_halo_image(s, x, y, [&](long long hi) {
    float* __restrict__ hb = a.fout + hi;
#pragma unroll
    for (int i = 0; i < QT; ++i) hb[tb.pl[i]] = g[i];
  });
}

// f*(0) = f^eq(n, U, T) - f_ref (Sec. 6.2): the moments in FP64 and the
// contraction with H = hi + lo in FP64, rounded once to FP32.
__global__ void __launch_bounds__(kThreads) k_init_xeq(const __grid_constant__ Tables<float> tb,
                                                       const __grid_constant__ XeqTables xq,
                                                       const __grid_constant__ InitArgs<float> a) {
  const Scalars& s = a.s;
  const int x = blockIdx.x * kBX + threadIdx.x;
  const int y = blockIdx.y * kBY + threadIdx.y;
  if (x >= s.nx || y >= s.ny) return;
  const int cell = y * s.nx + x;
  const double ux = a.ux[cell], uy = a.uy[cell];
  const double u2 = ux * ux + uy * uy;
  const double n = a.n[cell], T = a.T[cell];
  const bool ok = (u2 < 1.0) && (n > 0.0) && (T > 0.0);
  if (!ok) atomicAdd(a.status, 1ULL);
  const double gam = ok ? 1.0 / sqrt(1.0 - u2) : 1.0;
  double dM[16];
  eq_moments<double, 16>(n - s.n_ref, T - s.T_ref, n, T, gam, gam * ux, gam * uy, s.m, s.n_ref, s.T_ref, dM);
  const long long si = sidx(s, x, y);
  for (int i = 0; i < s.Q; ++i) {
    double feq = 0.0;
#pragma unroll
    for (int k = 0; k < 16; ++k) feq = fma((double)tb.H[i][k] + (double)xq.Hl[i][k], dM[k], feq);
    const float v = (float)feq;
    a.fout[i * s.plane + si] = v;
    for_each_halo_image(s, x, y, [&](long long hi) { a.fout[i * s.plane + hi] = v; });
  }
}

template <int QT>
cudaError_t launch_xeq_q(const Tables<float>& tb, const XeqTables& xq, const StepArgs<float>& a, int mode,
                         cudaStream_t st) {
  if (mode == kOnLattice) k_step_xeq<QT, kOnLattice><<<grid_for(a.s), block_dim(), 0, st>>>(tb, xq, a);
  else k_step_xeq<QT, kBilinear><<<grid_for(a.s), block_dim(), 0, st>>>(tb, xq, a);
  return cudaGetLastError();
}

}  // namespace

bool xeq_supported_q(int Q) { return Q == 45 || Q == 49 || Q == 53 || Q == 57 || Q == 65; }

cudaError_t launch_step_xeq(const Tables<float>& tb, const XeqTables& xq, const StepArgs<float>& a, int mode,
                            cudaStream_t st) {
  switch (a.s.Q) {
    case 45: return launch_xeq_q<45>(tb, xq, a, mode, st);
    case 49: return launch_xeq_q<49>(tb, xq, a, mode, st);
    case 53: return launch_xeq_q<53>(tb, xq, a, mode, st);
    case 57: return launch_xeq_q<57>(tb, xq, a, mode, st);
    case 65: return launch_xeq_q<65>(tb, xq, a, mode, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_init_xeq(const Tables<float>& tb, const XeqTables& xq, const InitArgs<float>& a,
                            cudaStream_t st) {
  k_init_xeq<<<grid_for(a.s), block_dim(), 0, st>>>(tb, xq, a);
  return cudaGetLastError();
}

}  // namespace rlbm
