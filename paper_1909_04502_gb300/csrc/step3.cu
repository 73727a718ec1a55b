// (3+1)-dimensional massless RLBM step, order 2 (Sec. 5-6 with d = 3), FP64
// storage and arithmetic (k_step3) or FP32 storage (k_step3f):
// on-lattice pull, the moments N^a and T^ab, the Landau frame of the 4 x 4
// mixed tensor (Sec. 4), n = U.N, T = eps / (3n) (Eq. ultra-relativistic-eos,
// d = 3), f^eq = H M(n, U, T) (Eq. mj-discrete-feq), Anderson-Witting
// relaxation, store with the periodic halo images.
//
// Layout: one plane per population, cell (x, y, z) at
//   (z + h) * slab + (y + h) * pitch + (x + px),  slab = (ny + 2h) * pitch,
// with a halo of h = 3 cells (the stencil length) on every side holding the
// periodic images, so that every pull is the cell index plus a constant.
#include <cuda_runtime.h>

#include "d3_impl.cuh"

namespace rlbm {

namespace {

template <int QT>
__global__ void __launch_bounds__(128) k_step3(const __grid_constant__ Tables3 tb,
                                               const __grid_constant__ Step3Args<double> a) {
  const Scalars3& s = a.s;
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 4 + threadIdx.y, z = blockIdx.z;
  if (x >= s.nx || y >= s.ny || z >= s.nz) return;
  const long long si = sidx3(s, x, y, z);
  const double* __restrict__ base = a.fin + si;
  // pass 1: pull and moments
  double N[4] = {0.0, 0.0, 0.0, 0.0}, Tm[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) Tm[u][v] = 0.0;
#pragma unroll 6
  for (int i = 0; i < QT; ++i) {
    const double f = __ldg(base + tb.off[i]);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const double fu = f * tb.c[i][u];
      N[u] += fu;
#pragma unroll
      for (int v = u; v < 4; ++v) Tm[u][v] = fma(fu, tb.c[i][v], Tm[u][v]);
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < u; ++v) Tm[u][v] = Tm[v][u];
  const Macro3 M = landau3(N, Tm);
  if (!M.ok) atomicAdd(a.status, 1ULL);
  double Mm[14];
  mj_moments3(M.n, M.T, M.U, Mm);
  const double kt = M.ok ? 1.0 / s.tau : 0.0;
  // halo images of this cell: every side is at least h long, so each axis
  // gives at most two images (c + n, c - n) and a cell at most 3^3 - 1 = 26
  int ix[2], iy[2], iz[2];
  const int nx2 = images1(x, s.nx, s.h, ix), ny2 = images1(y, s.ny, s.h, iy), nz2 = images1(z, s.nz, s.h, iz);
  long long img[26];
  int nimg = 0;
  for (int cz = -1; cz < nz2; ++cz)
    for (int cy = -1; cy < ny2; ++cy)
      for (int cx = -1; cx < nx2; ++cx) {
        if (cx < 0 && cy < 0 && cz < 0) continue;
        img[nimg++] = sidx3(s, cx < 0 ? x : ix[cx], cy < 0 ? y : iy[cy], cz < 0 ? z : iz[cz]);
      }
  // pass 2: equilibrium, relaxation, store (the pulled value is read again)
  double* __restrict__ out = a.fout;
#pragma unroll 2
  for (int i = 0; i < QT; ++i) {
    const double f = __ldg(base + tb.off[i]);
    double feq = 0.0;
#pragma unroll
    for (int k = 0; k < 14; ++k) feq = fma(tb.H[i][k], Mm[k], feq);
    const double om = kt * (M.U[0] - tb.v[i][0] * M.U[1] - tb.v[i][1] * M.U[2] - tb.v[i][2] * M.U[3]);
    const double g = fma(om, feq - f, f);
    const long long pl = (long long)i * s.plane;
    out[pl + si] = g;
    for (int m = 0; m < nimg; ++m) out[pl + img[m]] = g;
  }
}

// FP32 storage: g = f - f_ref is stored and collided in FP32; the moments are
// FP32 sums of g (the reference moments enter in FP64); the Landau root is
// found in FP32 (Newton on det(A - l I)) and corrected by one Newton step
// whose residual, the eigenvector's nu^2 = v.v, w = v.N and the numerator of
// dn = n - n_ref are evaluated in FP64 (landau3f); the equilibrium
// differences dM = M(n, U, T) - M_ref are written so that each is accurate
// relative to itself, and the equilibrium, the relaxation and the store are
// FP32.
template <int QT>
__global__ void __launch_bounds__(128) k_step3f(const __grid_constant__ Tables3 tb,
                                                const __grid_constant__ Step3Args<float> a) {
  const Scalars3& s = a.s;
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 4 + threadIdx.y, z = blockIdx.z;
  if (x >= s.nx || y >= s.ny || z >= s.nz) return;
  const long long si = sidx3(s, x, y, z);
  const float* __restrict__ base = a.fin + si;
  float N[4] = {0.f, 0.f, 0.f, 0.f}, Tm[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) Tm[u][v] = 0.f;
#pragma unroll 6
  for (int i = 0; i < QT; ++i) {
    const float g = __ldg(base + tb.off[i]);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float gu = g * tb.cf[i][u];
      N[u] += gu;
#pragma unroll
      for (int v = u; v < 4; ++v) Tm[u][v] = fmaf(gu, tb.cf[i][v], Tm[u][v]);
    }
  }
  const Macro3f M = landau3f(N, Tm, s);
  const bool ok = M.ok;
  if (!ok) atomicAdd(a.status, 1ULL);
  const float U0 = M.U0, Ux = M.Ux, Uy = M.Uy, Uz = M.Uz;
  float dM[14];
  mj_delta3<14>(M, (float)s.n_ref, (float)s.T_ref, dM);
  const float kt = ok ? (float)(1.0 / s.tau) : 0.f;
  int ix[2], iy[2], iz[2];
  const int nx2 = images1(x, s.nx, s.h, ix), ny2 = images1(y, s.ny, s.h, iy), nz2 = images1(z, s.nz, s.h, iz);
  long long img[26];
  int nimg = 0;
  for (int cz = -1; cz < nz2; ++cz)
    for (int cy = -1; cy < ny2; ++cy)
      for (int cx = -1; cx < nx2; ++cx) {
        if (cx < 0 && cy < 0 && cz < 0) continue;
        img[nimg++] = sidx3(s, cx < 0 ? x : ix[cx], cy < 0 ? y : iy[cy], cz < 0 ? z : iz[cz]);
      }
  float* __restrict__ out = a.fout;
#pragma unroll 2
  for (int i = 0; i < QT; ++i) {
    const float g = __ldg(base + tb.off[i]);
    float geq = 0.f;
#pragma unroll
    for (int kk = 0; kk < 14; ++kk) geq = fmaf(tb.Hf[i][kk], dM[kk], geq);
    const float om = kt * (U0 - tb.vf[i][0] * Ux - tb.vf[i][1] * Uy - tb.vf[i][2] * Uz);
    const float gn = fmaf(om, geq - g, g);
    const long long pl = (long long)i * s.plane;
    out[pl + si] = gn;
    for (int m = 0; m < nimg; ++m) out[pl + img[m]] = gn;
  }
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

template <>
cudaError_t launch_step3<double>(const Tables3& tb, const Step3Args<double>& a, cudaStream_t st) {
  if (a.s.Q != 78) return cudaErrorInvalidValue;
  k_step3<78><<<grid3(a.s), dim3(32, 4), 0, st>>>(tb, a);
  return cudaGetLastError();
}

template <>
cudaError_t launch_step3<float>(const Tables3& tb, const Step3Args<float>& a, cudaStream_t st) {
  if (a.s.Q != 78) return cudaErrorInvalidValue;
  k_step3f<78><<<grid3(a.s), dim3(32, 4), 0, st>>>(tb, a);
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
