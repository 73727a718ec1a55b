// (3+1)-dimensional massless RLBM step, order 2, FP64 (Sec. 5-6 with d = 3):
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

#include "d3.h"

namespace rlbm {

namespace {

__device__ __forceinline__ long long sidx3(const Scalars3& s, int x, int y, int z) {
  return (long long)(z + s.h) * s.slab + (long long)(y + s.h) * s.pitch + (x + s.px);
}

// periodic images of coordinate c in [-h, n + h), other than c itself
__device__ __forceinline__ int images1(int c, int n, int h, int (&out)[2]) {
  int k = 0;
  if (c + n < n + h) out[k++] = c + n;
  if (c - n >= -h) out[k++] = c - n;
  return k;
}

__device__ __forceinline__ double det3(double a, double b, double c, double d, double e, double f, double g,
                                       double hh, double i) {
  return a * (e * i - f * hh) - b * (d * i - f * g) + c * (d * hh - e * g);
}

struct Macro3 {
  double n, T, eps, U[4];
  bool ok;
};

// Largest eigenvalue eps of A^a_b = T^ac eta_cb and its timelike eigenvector:
// Newton on p(l) = det(A - l I) from the ideal-fluid root for P = eps / 3,
// p'(l) = -(sum of the principal 3 x 3 minors of A - l I); U from the first
// column of adj(A - l I) (a right null vector), normalised to U.U = 1, U^0 > 0.
__device__ Macro3 landau3(const double (&N)[4], const double (&Tm)[4][4]) {
  double A[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) A[a][b] = b == 0 ? Tm[a][b] : -Tm[a][b];
  const double E = Tm[0][0], M2 = Tm[0][1] * Tm[0][1] + Tm[0][2] * Tm[0][2] + Tm[0][3] * Tm[0][3];
  const double k = 1.0 / 3.0;
  double lam = (-(1.0 - k) * E + sqrt(fmax((1.0 - k) * (1.0 - k) * E * E + 4.0 * k * (E * E - M2), 0.0))) /
               (2.0 * k);
  double B[4][4];
  for (int it = 0; it < 8; ++it) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) B[a][b] = A[a][b] - (a == b ? lam : 0.0);
    // det by complementary 2 x 2 minors of rows (0, 1) and (2, 3)
    const double s0 = B[0][0] * B[1][1] - B[1][0] * B[0][1], s1 = B[0][0] * B[1][2] - B[1][0] * B[0][2];
    const double s2 = B[0][0] * B[1][3] - B[1][0] * B[0][3], s3 = B[0][1] * B[1][2] - B[1][1] * B[0][2];
    const double s4 = B[0][1] * B[1][3] - B[1][1] * B[0][3], s5 = B[0][2] * B[1][3] - B[1][2] * B[0][3];
    const double c5 = B[2][2] * B[3][3] - B[3][2] * B[2][3], c4 = B[2][1] * B[3][3] - B[3][1] * B[2][3];
    const double c3 = B[2][1] * B[3][2] - B[3][1] * B[2][2], c2 = B[2][0] * B[3][3] - B[3][0] * B[2][3];
    const double c1 = B[2][0] * B[3][2] - B[3][0] * B[2][2], c0 = B[2][0] * B[3][1] - B[3][0] * B[2][1];
    const double p = s0 * c5 - s1 * c4 + s2 * c3 + s3 * c2 - s4 * c1 + s5 * c0;
    const double m0 = det3(B[1][1], B[1][2], B[1][3], B[2][1], B[2][2], B[2][3], B[3][1], B[3][2], B[3][3]);
    const double m1 = det3(B[0][0], B[0][2], B[0][3], B[2][0], B[2][2], B[2][3], B[3][0], B[3][2], B[3][3]);
    const double m2 = det3(B[0][0], B[0][1], B[0][3], B[1][0], B[1][1], B[1][3], B[3][0], B[3][1], B[3][3]);
    const double m3 = det3(B[0][0], B[0][1], B[0][2], B[1][0], B[1][1], B[1][2], B[2][0], B[2][1], B[2][2]);
    const double dp = -(m0 + m1 + m2 + m3);
    if (!(dp != 0.0)) break;
    const double step = p / dp;
    lam -= step;
    if (fabs(step) <= 1e-15 * fabs(lam)) break;
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) B[a][b] = A[a][b] - (a == b ? lam : 0.0);
  // v_i = (-1)^i det(B without row 0 and column i)
  double v[4];
  v[0] = det3(B[1][1], B[1][2], B[1][3], B[2][1], B[2][2], B[2][3], B[3][1], B[3][2], B[3][3]);
  v[1] = -det3(B[1][0], B[1][2], B[1][3], B[2][0], B[2][2], B[2][3], B[3][0], B[3][2], B[3][3]);
  v[2] = det3(B[1][0], B[1][1], B[1][3], B[2][0], B[2][1], B[2][3], B[3][0], B[3][1], B[3][3]);
  v[3] = -det3(B[1][0], B[1][1], B[1][2], B[2][0], B[2][1], B[2][2], B[3][0], B[3][1], B[3][2]);
  const double nu2 = v[0] * v[0] - v[1] * v[1] - v[2] * v[2] - v[3] * v[3];
  Macro3 M;
  const double inu = (v[0] > 0.0 ? 1.0 : -1.0) / sqrt(fabs(nu2));
#pragma unroll
  for (int a = 0; a < 4; ++a) M.U[a] = v[a] * inu;
  M.n = M.U[0] * N[0] - M.U[1] * N[1] - M.U[2] * N[2] - M.U[3] * N[3];
  M.eps = lam;
  M.T = lam / (3.0 * M.n);
  M.ok = nu2 > 0.0 && M.n > 0.0 && M.T > 0.0 && isfinite(M.T) && isfinite(M.U[0]);
  return M;
}

// MJ moments of the basis 1 | p0 px py pz | p0px p0py p0pz pxpx pxpy pxpz pypy
// pypz pzpz for massless particles in d = 3 (App. B): <1> = n/(2T),
// <p^a> = n U^a, <p^a p^b> = n (4T U^a U^b - T eta^ab).
__device__ __forceinline__ void mj_moments3(double n, double T, const double (&U)[4], double (&M)[14]) {
  const double q = 4.0 * n * T;
  M[0] = n / (2.0 * T);
  M[1] = n * U[0];
  M[2] = n * U[1];
  M[3] = n * U[2];
  M[4] = n * U[3];
  M[5] = q * U[0] * U[1];
  M[6] = q * U[0] * U[2];
  M[7] = q * U[0] * U[3];
  M[8] = q * U[1] * U[1] + n * T;
  M[9] = q * U[1] * U[2];
  M[10] = q * U[1] * U[3];
  M[11] = q * U[2] * U[2] + n * T;
  M[12] = q * U[2] * U[3];
  M[13] = q * U[3] * U[3] + n * T;
}

template <int QT>
__global__ void __launch_bounds__(128) k_step3(const __grid_constant__ Tables3 tb, const __grid_constant__ Step3Args a) {
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

// f*(0) = f^eq(n, U, T) of host/device fields (row-major [z][y][x]),
// written to the interior and the halo images.
__global__ void __launch_bounds__(128) k_init3(const __grid_constant__ Tables3 tb, const __grid_constant__ Init3Args a) {
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
    const long long pl = (long long)i * s.plane;
    for (int cz = -1; cz < nz2; ++cz)
      for (int cy = -1; cy < ny2; ++cy)
        for (int cx = -1; cx < nx2; ++cx)
          a.f[pl + sidx3(s, cx < 0 ? x : ix[cx], cy < 0 ? y : iy[cy], cz < 0 ? z : iz[cz])] = feq;
  }
}

// Fields of f(t): the populations pulled from f*(t-1) (after a step) or, at
// t = 0, f*(0) = f^eq itself: n, ux, uy, uz, T, eps.
__global__ void __launch_bounds__(128) k_fields3(const __grid_constant__ Tables3 tb, const __grid_constant__ Fields3Args a) {
  const Scalars3& s = a.s;
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 4 + threadIdx.y, z = blockIdx.z;
  if (x >= s.nx || y >= s.ny || z >= s.nz) return;
  const double* __restrict__ base = a.fin + sidx3(s, x, y, z);
  double N[4] = {0.0, 0.0, 0.0, 0.0}, Tm[4][4];
  for (int u = 0; u < 4; ++u)
    for (int v = 0; v < 4; ++v) Tm[u][v] = 0.0;
  for (int i = 0; i < s.Q; ++i) {
    const double f = base[a.pull ? (long long)tb.off[i] : (long long)i * s.plane];
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

cudaError_t launch_step3(const Tables3& tb, const Step3Args& a, cudaStream_t st) {
  if (a.s.Q != 78) return cudaErrorInvalidValue;
  k_step3<78><<<grid3(a.s), dim3(32, 4), 0, st>>>(tb, a);
  return cudaGetLastError();
}

cudaError_t launch_init3(const Tables3& tb, const Init3Args& a, cudaStream_t st) {
  k_init3<<<grid3(a.s), dim3(32, 4), 0, st>>>(tb, a);
  return cudaGetLastError();
}

cudaError_t launch_fields3(const Tables3& tb, const Fields3Args& a, cudaStream_t st) {
  k_fields3<<<grid3(a.s), dim3(32, 4), 0, st>>>(tb, a);
  return cudaGetLastError();
}

}  // namespace rlbm
