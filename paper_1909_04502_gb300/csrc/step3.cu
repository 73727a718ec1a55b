// (3+1)-dimensional massless RLBM step, order 2 (Sec. 5-6 with d = 3):
// on-lattice pull, the moments N^a and T^ab, the Landau frame of the 4 x 4
// mixed tensor (Sec. 4), n = U.N, T = eps / (3n) (Eq. ultra-relativistic-eos,
// d = 3), f^eq = H M(n, U, T) (Eq. mj-discrete-feq), Anderson-Witting
// relaxation, store with the periodic halo images.  Kernels: k_step3s (FP64)
// and k_step3fs (FP32 storage of g = f - f_ref), both with the table in
// sign-orbit form.
//
// Layout: one plane per population, cell (x, y, z) at
//   (z + h) * slab + (y + h) * pitch + (x + px),  slab = (ny + 2h) * pitch,
// with a halo of h = 3 cells (the stencil length) on every side holding the
// periodic images, so that every pull is the cell index plus a constant.
#include <cuda_runtime.h>

#include "d3_impl.cuh"

namespace rlbm {

namespace {

// spatial exponents (x, y, z) of the order-2 basis members 1 | p0 px py pz |
// p0px p0py p0pz pxpx pxpy pxpz pypy pypz pzpz
__device__ constexpr int kBasis3Exp[14][3] = {{0, 0, 0}, {0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1},
                                              {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0}, {1, 1, 0},
                                              {1, 0, 1}, {0, 2, 0}, {0, 1, 1}, {0, 0, 2}};

// The FP64 step in sign-orbit form (k_step3fs is its FP32-storage form).
// Populations come in runs whose members share p0 and |p| componentwise:
// 9 runs of 8 (member s negates the components whose bit is set in s) and
// the pairs (+-3, 0, 0), (0, +-3, 0), (0, 0, +-3).  Per run of 8, a
// Walsh-Hadamard transform of the pulled values gives the sums
// F_c = sum_s chi_c(s) f_s over the sign characters c; each moment of rank
// <= 2 needs one of them times the first member's monomial (e.g. T^xy += a b
// F_xy).  The equilibrium rows of a run are the first row with the sign
// chi_k(s) of each basis member k (checked exactly on the host), so f^eq_s =
// sum over the seven characters of chi(s) C_chi, with C_chi the first row's
// partial sums over the members of that character; the relaxation rates
// follow from v_s . U = sx vx Ux + sy vy Uy + sz vz Uz.  About 110 operations
// per run of 8 against about 270 for eight rows.
template <typename S>
__device__ __forceinline__ const S* row_H(const Tables3& tb, int i) {
  if constexpr (sizeof(S) == 8) return tb.H[i];
  else return tb.Hf[i];
}
template <typename S>
__device__ __forceinline__ const S* row_v(const Tables3& tb, int i) {
  if constexpr (sizeof(S) == 8) return tb.v[i];
  else return tb.vf[i];
}
template <typename S>
__device__ __forceinline__ const S* row_mono(const Tables3& tb, int r) {
  static_assert(sizeof(S) == 8, "the monomial table is FP64");
  return tb.mono[r];
}

template <typename S>
__global__ void __launch_bounds__(128) k_step3s(const __grid_constant__ Tables3 tb,
                                                const __grid_constant__ Step3Args<S> a) {
  const Scalars3& s = a.s;
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 4 + threadIdx.y, z = blockIdx.z;
  if (x >= s.nx || y >= s.ny || z >= s.nz) return;
  const long long si = sidx3(s, x, y, z);
  const S* __restrict__ base = a.fin + si;
  // pass 1: moments m = N0 Nx Ny Nz T00 T0x T0y T0z Txx Txy Txz Tyy Tyz Tzz
  S m[14];
#pragma unroll
  for (int k = 0; k < 14; ++k) m[k] = S(0);
#pragma unroll 1
  for (int r = 0; r < 9; ++r) {
    S f[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) f[q] = __ldg(base + tb.off[8 * r + q]);
    fwht(f);
    moments_run8(f, row_mono<S>(tb, r), m);
  }
  // the axis pairs: N^a, T^0a odd, T^00, T^aa, N^0 even
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const S fp = __ldg(base + tb.off[72 + 2 * ax]), fm = __ldg(base + tb.off[73 + 2 * ax]);
    const S Sm = fp + fm, D = fp - fm;
    const S* c = row_mono<S>(tb, 9 + ax);
    const int taa = ax == 0 ? 8 : (ax == 1 ? 11 : 13);
    m[0] = fma(c[0], Sm, m[0]);
    m[4] = fma(c[4], Sm, m[4]);
    m[1 + ax] = fma(c[1 + ax], D, m[1 + ax]);
    m[5 + ax] = fma(c[5 + ax], D, m[5 + ax]);
    m[taa] = fma(c[taa], Sm, m[taa]);
  }
  S Mm[14], kU0, kU[3];
  if (!frame3(m, s, Mm, kU0, kU)) atomicAdd(a.status, 1ULL);
  long long img[26];
  const int nimg = cell_images(s, x, y, z, img);
  S* __restrict__ out = a.fout;
  // pass 2: equilibrium, relaxation, store (the pulled values are read again)
#pragma unroll 1
  for (int r = 0; r < 9; ++r) {
    const S* H0 = row_H<S>(tb, 8 * r);
    // partial sums over the basis members of each sign character, then
    // f^eq_s = sum_c chi_c(s) C_c
    S C[8];
    C[0] = fma(H0[0], Mm[0], fma(H0[1], Mm[1], fma(H0[8], Mm[8], fma(H0[11], Mm[11], H0[13] * Mm[13]))));
    C[1] = fma(H0[2], Mm[2], H0[5] * Mm[5]);
    C[2] = fma(H0[3], Mm[3], H0[6] * Mm[6]);
    C[4] = fma(H0[4], Mm[4], H0[7] * Mm[7]);
    C[3] = H0[9] * Mm[9];
    C[5] = H0[10] * Mm[10];
    C[6] = H0[12] * Mm[12];
    C[7] = S(0);
    fwht(C);
    // tau^-1 (U0 - v_s . U)
    const S* vb = row_v<S>(tb, 8 * r);
    const S X = vb[0] * kU[0], Y = vb[1] * kU[1], Z = vb[2] * kU[2];
    const S r0 = kU0 - X, r1 = kU0 + X;
    const S R[4] = {r0 - Y, r1 - Y, r0 + Y, r1 + Y};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int i = 8 * r + q;
      const S om = (q & 4) ? R[q & 3] + Z : R[q & 3] - Z;
      const S f = __ldg(base + tb.off[i]);
      const S g = fma(om, C[q] - f, f);
      const long long pl = (long long)i * s.plane;
      out[pl + si] = g;
      for (int mm = 0; mm < nimg; ++mm) out[pl + img[mm]] = g;
    }
  }
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const int i0 = 72 + 2 * ax;
    const S* H0 = row_H<S>(tb, i0);
    S Ce = S(0), Co = S(0);
#pragma unroll
    for (int k = 0; k < 14; ++k) {
      // basis members odd in component ax: p_a, p0 p_a and the mixed p_a p_b
      if (kBasis3Exp[k][ax] & 1) Co = fma(H0[k], Mm[k], Co);
      else Ce = fma(H0[k], Mm[k], Ce);
    }
    const S va = row_v<S>(tb, i0)[ax] * kU[ax];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int i = i0 + q;
      const S feq = q ? Ce - Co : Ce + Co;
      const S om = q ? kU0 + va : kU0 - va;
      const S f = __ldg(base + tb.off[i]);
      const S g = fma(om, feq - f, f);
      const long long pl = (long long)i * s.plane;
      out[pl + si] = g;
      for (int mm = 0; mm < nimg; ++mm) out[pl + img[mm]] = g;
    }
  }
}

// FP32 storage in sign-orbit form: g = f - f_ref is stored and collided in
// FP32 with the run arithmetic of k_step3s; the moments are FP32 sums of g
// (the reference moments enter in FP64); the Landau root is found in FP32
// (Newton on det(A - l I)) and corrected by one Newton step whose residual,
// the eigenvector's nu^2 = v.v, w = v.N and the numerator of dn = n - n_ref
// are evaluated in FP64 (landau3f, through frame3); the equilibrium
// differences dM = M(n, U, T) - M_ref are written so that each is accurate
// relative to itself, and the equilibrium, the relaxation and the store are
// FP32.  Every run is unrolled, so each table entry (pull shift, monomial, H
// row, velocity) is an immediate constant operand rather than a load by
// run-time index (with the runs in a loop this form was slower than the
// row-by-row kernel it replaced).  Eight blocks of 128 threads per SM
// (64 registers).  At 192^3: 1.51 ms per step against 2.20 ms row by row.
// The interior is stored in the relaxation pass; cells next to a face then
// copy their values to the periodic images, six at a time.
__global__ void __launch_bounds__(128, 8) k_step3fs(const __grid_constant__ Tables3 tb,
                                                    const __grid_constant__ Step3Args<float> a) {
  const Scalars3& s = a.s;
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 4 + threadIdx.y, z = blockIdx.z;
  if (x >= s.nx || y >= s.ny || z >= s.nz) return;
  const long long si = sidx3(s, x, y, z);
  const float* __restrict__ base = a.fin + si;
  // pass 1: m = N0 Nx Ny Nz T00 T0x T0y T0z Txx Txy Txz Tyy Tyz Tzz of g
  float m[14];
#pragma unroll
  for (int k = 0; k < 14; ++k) m[k] = 0.f;
#pragma unroll
  for (int r = 0; r < 9; ++r) {
    float f[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) f[q] = __ldg(base + tb.off[8 * r + q]);
    fwht(f);
    moments_run8(f, tb.monof[r], m);
  }
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const float fp = __ldg(base + tb.off[72 + 2 * ax]), fm = __ldg(base + tb.off[73 + 2 * ax]);
    const float Sm = fp + fm, D = fp - fm;
    const float* c = tb.monof[9 + ax];
    const int taa = ax == 0 ? 8 : (ax == 1 ? 11 : 13);
    m[0] = fmaf(c[0], Sm, m[0]);
    m[4] = fmaf(c[4], Sm, m[4]);
    m[1 + ax] = fmaf(c[1 + ax], D, m[1 + ax]);
    m[5 + ax] = fmaf(c[5 + ax], D, m[5 + ax]);
    m[taa] = fmaf(c[taa], Sm, m[taa]);
  }
  float Mm[14], kU0, kU[3];
  if (!frame3(m, s, Mm, kU0, kU)) atomicAdd(a.status, 1ULL);
  // pass 2: equilibrium differences, relaxation, interior store (order 2
  // keeps Q * plane below 2^31)
  const int ipl = (int)s.plane;
  float* ob = a.fout + si;
#pragma unroll
  for (int r = 0; r < 9; ++r) {
    const float* H0 = tb.Hf[8 * r];
    float C[8];
    C[0] = fmaf(H0[0], Mm[0], fmaf(H0[1], Mm[1], fmaf(H0[8], Mm[8], fmaf(H0[11], Mm[11], H0[13] * Mm[13]))));
    C[1] = fmaf(H0[2], Mm[2], H0[5] * Mm[5]);
    C[2] = fmaf(H0[3], Mm[3], H0[6] * Mm[6]);
    C[4] = fmaf(H0[4], Mm[4], H0[7] * Mm[7]);
    C[3] = H0[9] * Mm[9];
    C[5] = H0[10] * Mm[10];
    C[6] = H0[12] * Mm[12];
    C[7] = 0.f;
    fwht(C);
    const float* vb = tb.vf[8 * r];
    const float X = vb[0] * kU[0], Y = vb[1] * kU[1], Z = vb[2] * kU[2];
    const float r0 = kU0 - X, r1 = kU0 + X;
    const float R[4] = {r0 - Y, r1 - Y, r0 + Y, r1 + Y};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int i = 8 * r + q;
      const float om = (q & 4) ? R[q & 3] + Z : R[q & 3] - Z;
      const float g = __ldg(base + tb.off[i]);
      ob[i * ipl] = fmaf(om, C[q] - g, g);
    }
  }
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const int i0 = 72 + 2 * ax;
    const float* H0 = tb.Hf[i0];
    float Ce = 0.f, Co = 0.f;
#pragma unroll
    for (int k = 0; k < 14; ++k) {
      if (kBasis3Exp[k][ax] & 1) Co = fmaf(H0[k], Mm[k], Co);
      else Ce = fmaf(H0[k], Mm[k], Ce);
    }
    const float va = tb.vf[i0][ax] * kU[ax];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int i = i0 + q;
      const float feq = q ? Ce - Co : Ce + Co;
      const float om = q ? kU0 + va : kU0 - va;
      const float g = __ldg(base + tb.off[i]);
      ob[i * ipl] = fmaf(om, feq - g, g);
    }
  }
  images_from_stored<78, 6>(s, a.fout, si, x, y, z);
}

// f*(0) = f^eq(n, U, T) of device fields (row-major [z][y][x]), stored as f
// (FP64) or f - f_ref (FP32), written to the interior and the halo images.
template <typename S>
__global__ void __launch_bounds__(128) k_init3(const __grid_constant__ Tables3 tb,
                                               const __grid_constant__ Init3Args<S> a) {
  const Scalars3& s = a.s;
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 4 + threadIdx.y, z = blockIdx.z;
  if (x >= s.nx || y >= s.ny || z >= s.nz) return;
  const long long c = ((long long)z * s.ny + y) * s.nx + x;
  const double ux = a.ux[c], uy = a.uy[c], uz = a.uz[c];
  const double g = 1.0 / sqrt(1.0 - ux * ux - uy * uy - uz * uz);
  const double U[4] = {g, g * ux, g * uy, g * uz};
  double Mm[14];
  mj_moments3(a.n[c], a.T[c], U, Mm);
  int ix[2], iy[2], iz[2];
  const int nx2 = images1(x, s.nx, s.h, ix), ny2 = images1(y, s.ny, s.h, iy), nz2 = images1(z, s.nz, s.h, iz);
  for (int i = 0; i < s.Q; ++i) {
    double feq = 0.0;
    for (int k = 0; k < 14; ++k) feq = fma(tb.H[i][k], Mm[k], feq);
    const S val = (S)(sizeof(S) == 4 ? feq - tb.fref[i] : feq);
    const long long pl = (long long)i * s.plane;
    for (int cz = -1; cz < nz2; ++cz)
      for (int cy = -1; cy < ny2; ++cy)
        for (int cx = -1; cx < nx2; ++cx)
          a.f[pl + sidx3(s, cx < 0 ? x : ix[cx], cy < 0 ? y : iy[cy], cz < 0 ? z : iz[cz])] = val;
  }
}

// Fields of f(t): the populations pulled from f*(t-1) (after a step) or, at
// t = 0, f*(0) = f^eq itself: n, ux, uy, uz, T, eps (FP64; f = g + f_ref for
// FP32 storage).
template <typename S>
__global__ void __launch_bounds__(128) k_fields3(const __grid_constant__ Tables3 tb,
                                                 const __grid_constant__ Fields3Args<S> a) {
  const Scalars3& s = a.s;
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 4 + threadIdx.y, z = blockIdx.z;
  if (x >= s.nx || y >= s.ny || z >= s.nz) return;
  const S* __restrict__ base = a.fin + sidx3(s, x, y, z);
  double N[4] = {0.0, 0.0, 0.0, 0.0}, Tm[4][4];
  for (int u = 0; u < 4; ++u)
    for (int v = 0; v < 4; ++v) Tm[u][v] = 0.0;
  for (int i = 0; i < s.Q; ++i) {
    double f = (double)base[a.pull ? (long long)tb.off[i] : (long long)i * s.plane];
    if (sizeof(S) == 4) f += tb.fref[i];
    for (int u = 0; u < 4; ++u) {
      N[u] += f * tb.c[i][u];
      for (int v = u; v < 4; ++v) Tm[u][v] = fma(f * tb.c[i][u], tb.c[i][v], Tm[u][v]);
    }
  }
  for (int u = 0; u < 4; ++u)
    for (int v = 0; v < u; ++v) Tm[u][v] = Tm[v][u];
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

dim3 grid3(const Scalars3& s) { return dim3((s.nx + 31) / 32, (s.ny + 3) / 4, s.nz); }

}  // namespace

template <typename S>
cudaError_t launch_step3_sym(const Tables3& tb, const Step3Args<S>& a, cudaStream_t st) {
  if (a.s.Q != 78) return cudaErrorInvalidValue;
  k_step3s<S><<<grid3(a.s), dim3(32, 4), 0, st>>>(tb, a);
  return cudaGetLastError();
}
template cudaError_t launch_step3_sym<double>(const Tables3&, const Step3Args<double>&, cudaStream_t);

cudaError_t launch_step3f_sym(const Tables3& tb, const Step3Args<float>& a, cudaStream_t st) {
  if (a.s.Q != 78) return cudaErrorInvalidValue;
  k_step3fs<<<grid3(a.s), dim3(32, 4), 0, st>>>(tb, a);
  return cudaGetLastError();
}

template <typename S>
cudaError_t launch_init3(const Tables3& tb, const Init3Args<S>& a, cudaStream_t st) {
  k_init3<S><<<grid3(a.s), dim3(32, 4), 0, st>>>(tb, a);
  return cudaGetLastError();
}

template <typename S>
cudaError_t launch_fields3(const Tables3& tb, const Fields3Args<S>& a, cudaStream_t st) {
  k_fields3<S><<<grid3(a.s), dim3(32, 4), 0, st>>>(tb, a);
  return cudaGetLastError();
}

template cudaError_t launch_init3<float>(const Tables3&, const Init3Args<float>&, cudaStream_t);
template cudaError_t launch_init3<double>(const Tables3&, const Init3Args<double>&, cudaStream_t);
template cudaError_t launch_fields3<float>(const Tables3&, const Fields3Args<float>&, cudaStream_t);
template cudaError_t launch_fields3<double>(const Tables3&, const Fields3Args<double>&, cudaStream_t);

}  // namespace rlbm
