// (3+1)-dimensional massless RLBM step at order 3 (App. H, v0 = 1/sqrt(41),
// Q = 288, K = 30), the order-2 step of step3.cu with the 30-member basis.
// Two kernels, one thread per cell over 33 runs of 8 and 6 runs of 4 sign
// variants, the run tables as kernel parameters: k_step3qs (FP64) and
// k_step3qsf (FP32 storage of g = f - f_ref).  (Earlier forms, row by row
// with four threads per cell or with the table in shared memory, ran
// 1.6-5x slower.)
// Pull offsets are the plane offset i * plane (64-bit) plus a per-population
// shift, since 288 planes of a large grid exceed 2^31 elements.
#include <cuda_runtime.h>

#include "d3_impl.cuh"

namespace rlbm {

namespace {

constexpr int kQo3 = 288, kKo3 = 30;

// Sign-orbit form, one thread per cell: the order-2 scheme of k_step3s with
// the 30-member basis (k_step3qsf is its FP32-storage form).  Runs of
// 8: a Walsh-Hadamard transform of the pulled values gives the moment sums;
// the first H row's partial sums over the eight parity classes of the basis
// (class of member k: the parities of its x, y, z exponents), transformed
// back, give the eight equilibrium values.  Runs of 4 do the same over their
// two non-zero components (basis members odd in the zero component have H = 0
// there).  About 5 k operations per cell against 16 k row by row; the run
// tables are kernel parameters.
__device__ constexpr int kBasis3o3Par[30] = {
    // parity class (bit 0: x odd, bit 1: y odd, bit 2: z odd) of the members of
    // 1 | p0 px py pz | p0px p0py p0pz pxpx pxpy pxpz pypy pypz pzpz |
    // p0 (xx xy xz yy yz zz) | xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz
    0, 0, 1, 2, 4, 1, 2, 4, 0, 3, 5, 0, 6, 0, 0, 3, 5, 0, 6, 0, 1, 2, 4, 1, 7, 1, 2, 4, 2, 4};
__device__ constexpr int kMask4o3[kRuns4o3] = {3, 5, 3, 5, 6, 6};

template <typename S>
__global__ void __launch_bounds__(128) k_step3qs(const __grid_constant__ Tables3s3<S> tb,
                                                 const __grid_constant__ Step3qArgs<S> a) {
  const Scalars3& s = a.s;
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 4 + threadIdx.y, z = blockIdx.z;
  if (x >= s.nx || y >= s.ny || z >= s.nz) return;
  const long long si = sidx3(s, x, y, z);
  const S* __restrict__ base = a.fin + si;
  const long long P = s.plane;
  // pass 1: m = N0 Nx Ny Nz T00 T0x T0y T0z Txx Txy Txz Tyy Tyz Tzz
  S m[14];
#pragma unroll
  for (int k = 0; k < 14; ++k) m[k] = S(0);
#pragma unroll 1
  for (int r = 0; r < kRuns8o3; ++r) {
    const int i0 = tb.start8[r];
    S f[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) f[q] = __ldg(base + (long long)(i0 + q) * P + tb.off[i0 + q]);
    fwht(f);
    moments_run8(f, tb.mono8[r], m);
  }
#pragma unroll
  for (int r = 0; r < kRuns4o3; ++r) {
    const int j = kMask4o3[r] & 1 ? 0 : 1, k = kMask4o3[r] & 4 ? 2 : 1;   // the non-zero components, j < k
    const int i0 = tb.start4[r];
    S f[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) f[q] = __ldg(base + (long long)(i0 + q) * P + tb.off[i0 + q]);
    fwht(f);                      // f = (sum, sum s_j, sum s_k, sum s_j s_k)
    const S* c = tb.mono4[r];
    const int djj = j == 0 ? 8 : 11, dkk = k == 1 ? 11 : 13, djk = j == 0 ? (k == 1 ? 9 : 10) : 12;
    m[0] = fma(c[0], f[0], m[0]);
    m[4] = fma(c[4], f[0], m[4]);
    m[1 + j] = fma(c[1 + j], f[1], m[1 + j]);
    m[1 + k] = fma(c[1 + k], f[2], m[1 + k]);
    m[5 + j] = fma(c[5 + j], f[1], m[5 + j]);
    m[5 + k] = fma(c[5 + k], f[2], m[5 + k]);
    m[djj] = fma(c[djj], f[0], m[djj]);
    m[dkk] = fma(c[dkk], f[0], m[dkk]);
    m[djk] = fma(c[djk], f[3], m[djk]);
  }
  S Mm[kKo3], kU0, kU[3];
  if (!frame3(m, s, Mm, kU0, kU)) atomicAdd(a.status, 1ULL);
  long long img[26];
  const int nimg = cell_images(s, x, y, z, img);
  S* __restrict__ out = a.fout;
  // pass 2
#pragma unroll 1
  for (int r = 0; r < kRuns8o3; ++r) {
    const int i0 = tb.start8[r];
    const S* H0 = tb.H8[r];
    S C[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) C[c] = S(0);
#pragma unroll
    for (int k = 0; k < kKo3; ++k) C[kBasis3o3Par[k]] = fma(H0[k], Mm[k], C[kBasis3o3Par[k]]);
    fwht(C);                      // C[q] = f^eq of member q
    const S* vb = tb.v8[r];
    const S X = vb[0] * kU[0], Y = vb[1] * kU[1], Z = vb[2] * kU[2];
    const S r0 = kU0 - X, r1 = kU0 + X;
    const S R[4] = {r0 - Y, r1 - Y, r0 + Y, r1 + Y};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int i = i0 + q;
      const S om = (q & 4) ? R[q & 3] + Z : R[q & 3] - Z;
      const long long pl = (long long)i * P;
      const S f = __ldg(base + pl + tb.off[i]);
      const S g = fma(om, C[q] - f, f);
      out[pl + si] = g;
      for (int mm = 0; mm < nimg; ++mm) out[pl + img[mm]] = g;
    }
  }
#pragma unroll
  for (int r = 0; r < kRuns4o3; ++r) {
    const int j = kMask4o3[r] & 1 ? 0 : 1, k = kMask4o3[r] & 4 ? 2 : 1;
    const int i0 = tb.start4[r];
    const S* H0 = tb.H4[r];
    S C[4] = {S(0), S(0), S(0), S(0)};
#pragma unroll
    for (int kk = 0; kk < kKo3; ++kk) {
      const int par = kBasis3o3Par[kk];
      const int c = ((par >> j) & 1) | (((par >> k) & 1) << 1);
      C[c] = fma(H0[kk], Mm[kk], C[c]);
    }
    fwht(C);                      // C[q] = f^eq of member q (bit 0: j negated, bit 1: k negated)
    const S* vb = tb.v4[r];
    const S Xj = vb[j] * kU[j], Xk = vb[k] * kU[k];
    const S om[4] = {kU0 - Xj - Xk, kU0 + Xj - Xk, kU0 - Xj + Xk, kU0 + Xj + Xk};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = i0 + q;
      const long long pl = (long long)i * P;
      const S f = __ldg(base + pl + tb.off[i]);
      const S g = fma(om[q], C[q] - f, f);
      out[pl + si] = g;
      for (int mm = 0; mm < nimg; ++mm) out[pl + img[mm]] = g;
    }
  }
}

// FP32 storage in sign-orbit form: the arithmetic of k_step3qs on g = f -
// f_ref in FP32 with the FP32 Landau frame and FP64 polish of the order-2
// step (frame3).  The moment
// pass is unrolled three runs deep and takes each run's pull shifts by run
// and member (off8, off4); the relaxation pass, unrolled two runs deep,
// starts with the runs of 4 and takes the runs of 8 in reverse, the order
// opposite to the moment pass, so that it first rereads what is most likely
// still in L2.  Six blocks of 128 threads per SM (80 registers).  At 192^3:
// 6.4 ms per step against 10.2 ms for the row-by-row kernel it replaced (the
// 288 x 30 table in shared memory, read by broadcast 16-byte loads).
// Measured and not kept:
// the moment pass unrolled completely (5 % slower) or not at all (8 %), the
// relaxation pass unrolled completely (1.4x slower; the code grows
// several-fold), five or seven blocks per SM (1-8 % slower), the relaxation
// pass in the moment pass's order (5 % slower), image copies 4 or 16 at a
// time (3 % slower).
__global__ void __launch_bounds__(128, 6) k_step3qsf(const __grid_constant__ Tables3s3<float> tb,
                                                     const __grid_constant__ Step3qArgs<float> a) {
  const Scalars3& s = a.s;
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 4 + threadIdx.y, z = blockIdx.z;
  if (x >= s.nx || y >= s.ny || z >= s.nz) return;
  const long long si = sidx3(s, x, y, z);
  const float* __restrict__ base = a.fin + si;
  const long long P = s.plane;
  float m[14];
#pragma unroll
  for (int k = 0; k < 14; ++k) m[k] = 0.f;
#pragma unroll 3
  for (int r = 0; r < kRuns8o3; ++r) {
    const float* b = base + (long long)tb.start8[r] * P;
    float f[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) f[q] = __ldg(b + q * P + tb.off8[r][q]);
    fwht(f);
    moments_run8(f, tb.mono8[r], m);
  }
#pragma unroll
  for (int r = 0; r < kRuns4o3; ++r) {
    const int j = kMask4o3[r] & 1 ? 0 : 1, k = kMask4o3[r] & 4 ? 2 : 1;   // the non-zero components, j < k
    const float* b = base + (long long)tb.start4[r] * P;
    float f[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) f[q] = __ldg(b + q * P + tb.off4[r][q]);
    fwht(f);                      // f = (sum, sum s_j, sum s_k, sum s_j s_k)
    const float* c = tb.mono4[r];
    const int djj = j == 0 ? 8 : 11, dkk = k == 1 ? 11 : 13, djk = j == 0 ? (k == 1 ? 9 : 10) : 12;
    m[0] = fmaf(c[0], f[0], m[0]);
    m[4] = fmaf(c[4], f[0], m[4]);
    m[1 + j] = fmaf(c[1 + j], f[1], m[1 + j]);
    m[1 + k] = fmaf(c[1 + k], f[2], m[1 + k]);
    m[5 + j] = fmaf(c[5 + j], f[1], m[5 + j]);
    m[5 + k] = fmaf(c[5 + k], f[2], m[5 + k]);
    m[djj] = fmaf(c[djj], f[0], m[djj]);
    m[dkk] = fmaf(c[dkk], f[0], m[dkk]);
    m[djk] = fmaf(c[djk], f[3], m[djk]);
  }
  float Mm[kKo3], kU0, kU[3];
  if (!frame3(m, s, Mm, kU0, kU)) atomicAdd(a.status, 1ULL);
  float* ob = a.fout + si;
#pragma unroll
  for (int r = kRuns4o3 - 1; r >= 0; --r) {
    const int j = kMask4o3[r] & 1 ? 0 : 1, k = kMask4o3[r] & 4 ? 2 : 1;
    const long long p0 = (long long)tb.start4[r] * P;
    const float* H0 = tb.H4[r];
    float C[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int kk = 0; kk < kKo3; ++kk) {
      const int par = kBasis3o3Par[kk];
      const int c = ((par >> j) & 1) | (((par >> k) & 1) << 1);
      C[c] = fmaf(H0[kk], Mm[kk], C[c]);
    }
    fwht(C);                      // C[q] = f^eq of member q (bit 0: j negated, bit 1: k negated)
    const float* vb = tb.v4[r];
    const float Xj = vb[j] * kU[j], Xk = vb[k] * kU[k];
    const float om[4] = {kU0 - Xj - Xk, kU0 + Xj - Xk, kU0 - Xj + Xk, kU0 + Xj + Xk};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float g = __ldg(base + p0 + q * P + tb.off4[r][q]);
      ob[p0 + q * P] = fmaf(om[q], C[q] - g, g);
    }
  }
#pragma unroll 2
  for (int r = kRuns8o3 - 1; r >= 0; --r) {
    const long long p0 = (long long)tb.start8[r] * P;
    const float* H0 = tb.H8[r];
    float C[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) C[c] = 0.f;
#pragma unroll
    for (int k = 0; k < kKo3; ++k) C[kBasis3o3Par[k]] = fmaf(H0[k], Mm[k], C[kBasis3o3Par[k]]);
    fwht(C);                      // C[q] = f^eq of member q
    const float* vb = tb.v8[r];
    const float X = vb[0] * kU[0], Y = vb[1] * kU[1], Z = vb[2] * kU[2];
    const float r0 = kU0 - X, r1 = kU0 + X;
    const float R[4] = {r0 - Y, r1 - Y, r0 + Y, r1 + Y};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float om = (q & 4) ? R[q & 3] + Z : R[q & 3] - Z;
      const float g = __ldg(base + p0 + q * P + tb.off8[r][q]);
      ob[p0 + q * P] = fmaf(om, C[q] - g, g);
    }
  }
  images_from_stored<kQo3, 8>(s, a.fout, si, x, y, z);
}

// f*(0) = f^eq(n, U, T) (stored f, or f - f_ref for FP32), one thread per cell.
template <typename S>
__global__ void __launch_bounds__(128) k_init3q(const __grid_constant__ Init3qArgs<S> a) {
  const Scalars3& s = a.s;
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 4 + threadIdx.y, z = blockIdx.z;
  if (x >= s.nx || y >= s.ny || z >= s.nz) return;
  const long long c = ((long long)z * s.ny + y) * s.nx + x;
  const double ux = a.ux[c], uy = a.uy[c], uz = a.uz[c];
  const double g = 1.0 / sqrt(1.0 - ux * ux - uy * uy - uz * uz);
  const double U[4] = {g, g * ux, g * uy, g * uz};
  double Mm[kKo3];
  mj_full3<kKo3>(a.n[c], a.T[c], U, Mm);
  long long img[26];
  const int nimg = cell_images(s, x, y, z, img);
  const long long si = sidx3(s, x, y, z);
  for (int i = 0; i < s.Q; ++i) {
    double feq = 0.0;
    for (int k = 0; k < kKo3; ++k) feq = fma(a.H[(size_t)i * kKo3 + k], Mm[k], feq);
    const S val = (S)(sizeof(S) == 4 ? feq - a.fref[i] : feq);
    const long long pl = (long long)i * s.plane;
    a.f[pl + si] = val;
    for (int m = 0; m < nimg; ++m) a.f[pl + img[m]] = val;
  }
}

// Fields of f(t) (pulled from f*(t-1), or f*(0) in place), FP64.
template <typename S>
__global__ void __launch_bounds__(128) k_fields3q(const __grid_constant__ Fields3qArgs<S> a) {
  const Scalars3& s = a.s;
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 4 + threadIdx.y, z = blockIdx.z;
  if (x >= s.nx || y >= s.ny || z >= s.nz) return;
  const S* __restrict__ base = a.fin + sidx3(s, x, y, z);
  double N[4] = {0.0, 0.0, 0.0, 0.0}, Tm[4][4];
  for (int u = 0; u < 4; ++u)
    for (int w = 0; w < 4; ++w) Tm[u][w] = 0.0;
  for (int i = 0; i < s.Q; ++i) {
    double f = (double)base[(long long)i * s.plane + (a.pull ? a.off[i] : 0)];
    if (sizeof(S) == 4) f += a.fref[i];
    for (int u = 0; u < 4; ++u) {
      N[u] += f * a.c[4 * i + u];
      for (int w = u; w < 4; ++w) Tm[u][w] = fma(f * a.c[4 * i + u], a.c[4 * i + w], Tm[u][w]);
    }
  }
  for (int u = 0; u < 4; ++u)
    for (int w = 0; w < u; ++w) Tm[u][w] = Tm[w][u];
  const Macro3 M = landau3(N, Tm);
  const long long c = ((long long)z * s.ny + y) * s.nx + x;
  const long long nc = (long long)s.nx * s.ny * s.nz;
  a.out[c] = M.ok ? M.n : __longlong_as_double(0x7ff8000000000000LL);
  a.out[nc + c] = M.U[1] / M.U[0];
  a.out[2 * nc + c] = M.U[2] / M.U[0];
  a.out[3 * nc + c] = M.U[3] / M.U[0];
  a.out[4 * nc + c] = M.T;
  a.out[5 * nc + c] = M.eps;
}

dim3 grid3q(const Scalars3& s) { return dim3((s.nx + 31) / 32, (s.ny + 3) / 4, s.nz); }

}  // namespace

template <typename S>
cudaError_t launch_step3q_sym(const Tables3s3<S>& tb, const Step3qArgs<S>& a, cudaStream_t st) {
  if (a.s.Q != kQo3) return cudaErrorInvalidValue;
  k_step3qs<S><<<grid3q(a.s), dim3(32, 4), 0, st>>>(tb, a);
  return cudaGetLastError();
}
template cudaError_t launch_step3q_sym<double>(const Tables3s3<double>&, const Step3qArgs<double>&, cudaStream_t);
cudaError_t launch_step3q_symf(const Tables3s3<float>& tb, const Step3qArgs<float>& a, cudaStream_t st) {
  if (a.s.Q != kQo3) return cudaErrorInvalidValue;
  k_step3qsf<<<grid3q(a.s), dim3(32, 4), 0, st>>>(tb, a);
  return cudaGetLastError();
}

template <typename S>
cudaError_t launch_init3q(const Init3qArgs<S>& a, cudaStream_t st) {
  k_init3q<S><<<grid3q(a.s), dim3(32, 4), 0, st>>>(a);
  return cudaGetLastError();
}

template <typename S>
cudaError_t launch_fields3q(const Fields3qArgs<S>& a, cudaStream_t st) {
  k_fields3q<S><<<grid3q(a.s), dim3(32, 4), 0, st>>>(a);
  return cudaGetLastError();
}

template cudaError_t launch_init3q<float>(const Init3qArgs<float>&, cudaStream_t);
template cudaError_t launch_init3q<double>(const Init3qArgs<double>&, cudaStream_t);
template cudaError_t launch_fields3q<float>(const Fields3qArgs<float>&, cudaStream_t);
template cudaError_t launch_fields3q<double>(const Fields3qArgs<double>&, cudaStream_t);

}  // namespace rlbm
