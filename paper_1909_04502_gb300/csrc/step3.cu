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

template <typename R>
__device__ __forceinline__ R det3(R a, R b, R c, R d, R e, R f, R g, R hh, R i) {
  return a * (e * i - f * hh) - b * (d * i - f * g) + c * (d * hh - e * g);
}

// det(B) by complementary 2 x 2 minors of rows (0, 1) and (2, 3), and
// d det(B - l I)/dl = -(sum of the principal 3 x 3 minors)
template <typename R>
__device__ __forceinline__ R det4(const R (&B)[4][4]) {
  const R s0 = B[0][0] * B[1][1] - B[1][0] * B[0][1], s1 = B[0][0] * B[1][2] - B[1][0] * B[0][2];
  const R s2 = B[0][0] * B[1][3] - B[1][0] * B[0][3], s3 = B[0][1] * B[1][2] - B[1][1] * B[0][2];
  const R s4 = B[0][1] * B[1][3] - B[1][1] * B[0][3], s5 = B[0][2] * B[1][3] - B[1][2] * B[0][3];
  const R c5 = B[2][2] * B[3][3] - B[3][2] * B[2][3], c4 = B[2][1] * B[3][3] - B[3][1] * B[2][3];
  const R c3 = B[2][1] * B[3][2] - B[3][1] * B[2][2], c2 = B[2][0] * B[3][3] - B[3][0] * B[2][3];
  const R c1 = B[2][0] * B[3][2] - B[3][0] * B[2][2], c0 = B[2][0] * B[3][1] - B[3][0] * B[2][1];
  return s0 * c5 - s1 * c4 + s2 * c3 + s3 * c2 - s4 * c1 + s5 * c0;
}

template <typename R>
__device__ __forceinline__ R ddet4(const R (&B)[4][4]) {
  const R m0 = det3(B[1][1], B[1][2], B[1][3], B[2][1], B[2][2], B[2][3], B[3][1], B[3][2], B[3][3]);
  const R m1 = det3(B[0][0], B[0][2], B[0][3], B[2][0], B[2][2], B[2][3], B[3][0], B[3][2], B[3][3]);
  const R m2 = det3(B[0][0], B[0][1], B[0][3], B[1][0], B[1][1], B[1][3], B[3][0], B[3][1], B[3][3]);
  const R m3 = det3(B[0][0], B[0][1], B[0][2], B[1][0], B[1][1], B[1][2], B[2][0], B[2][1], B[2][2]);
  return -(m0 + m1 + m2 + m3);
}

// right null vector of B from the first column of adj(B):
// v_i = (-1)^i det(B without row 0 and column i)
template <typename R>
__device__ __forceinline__ void adj_col0(const R (&B)[4][4], R (&v)[4]) {
  v[0] = det3(B[1][1], B[1][2], B[1][3], B[2][1], B[2][2], B[2][3], B[3][1], B[3][2], B[3][3]);
  v[1] = -det3(B[1][0], B[1][2], B[1][3], B[2][0], B[2][2], B[2][3], B[3][0], B[3][2], B[3][3]);
  v[2] = det3(B[1][0], B[1][1], B[1][3], B[2][0], B[2][1], B[2][3], B[3][0], B[3][1], B[3][3]);
  v[3] = -det3(B[1][0], B[1][1], B[1][2], B[2][0], B[2][1], B[2][2], B[3][0], B[3][1], B[3][2]);
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
    const double dp = ddet4(B);
    if (!(dp != 0.0)) break;
    const double step = det4(B) / dp;
    lam -= step;
    if (fabs(step) <= 1e-15 * fabs(lam)) break;
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) B[a][b] = A[a][b] - (a == b ? lam : 0.0);
  double v[4];
  adj_col0(B, v);
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
// FP32 sums of g plus the reference moments in FP64; the Landau root is
// found in FP32 (Newton on det(A - l I)) and corrected by one Newton step
// with the residual in FP64; the eigenvector (cofactors), nu^2 = v.v and
// w = v.N, and from them n, dn = n - n_ref, eps and dT = T - T_ref, are
// evaluated in FP64; the equilibrium differences dM = M(n, U, T) - M_ref are
// written so that each is accurate relative to itself, and the equilibrium,
// the relaxation and the store are FP32.
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
  const double nr = s.n_ref, Tr = s.T_ref, er = 3.0 * nr * Tr, Pr = nr * Tr;
  // full moments (reference in FP64) and the mixed tensor A = T eta
  double Nd[4] = {nr + (double)N[0], (double)N[1], (double)N[2], (double)N[3]};
  double A[4][4];
  float Af[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      double t = (double)(u <= v ? Tm[u][v] : Tm[v][u]);
      if (u == v) t += (u == 0 ? er : Pr);
      A[u][v] = v == 0 ? t : -t;
      Af[u][v] = (float)A[u][v];
    }
  // FP32 root from the ideal-fluid guess (P = eps / 3)
  const float E = Af[0][0], M2 = Af[1][0] * Af[1][0] + Af[2][0] * Af[2][0] + Af[3][0] * Af[3][0];
  const float k = 1.f / 3.f;
  float lam = (-(1.f - k) * E + sqrtf(fmaxf((1.f - k) * (1.f - k) * E * E + 4.f * k * (E * E - M2), 0.f))) /
              (2.f * k);
  float Bf[4][4];
  float dpf = -1.f;
#pragma unroll
  for (int it = 0; it < 3; ++it) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) Bf[u][v] = Af[u][v] - (u == v ? lam : 0.f);
    dpf = ddet4(Bf);
    lam -= det4(Bf) / dpf;
  }
  // FP64 residual at the FP32 root, one Newton correction
  double B[4][4];
  double ld = (double)lam;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) B[u][v] = A[u][v] - (u == v ? ld : 0.0);
  ld -= det4(B) / (double)dpf;
#pragma unroll
  for (int u = 0; u < 4; ++u) B[u][u] = A[u][u] - ld;
  double vv[4];
  adj_col0(B, vv);
  const double nu2 = vv[0] * vv[0] - vv[1] * vv[1] - vv[2] * vv[2] - vv[3] * vv[3];
  const double w = vv[0] * Nd[0] - vv[1] * Nd[1] - vv[2] * Nd[2] - vv[3] * Nd[3];
  const double nu = sqrt(fabs(nu2));
  const double sgn = vv[0] > 0.0 ? 1.0 : -1.0;
  const double n = sgn * w / nu;
  const double dn = (w * w - nr * nr * nu2) / (nu * (sgn * w + nr * nu));
  const double deps = ld - er;
  const double dT = (deps - 3.0 * Tr * dn) / (3.0 * n);
  const double T = Tr + dT;
  const bool ok = nu2 > 0.0 && n > 0.0 && T > 0.0 && isfinite(T) && isfinite(dn);
  if (!ok) atomicAdd(a.status, 1ULL);
  const float inu = (float)(sgn / nu);
  const float U0 = (float)vv[0] * inu, Ux = (float)vv[1] * inu, Uy = (float)vv[2] * inu, Uz = (float)vv[3] * inu;
  const float fn = (float)n, fT = (float)T, fdn = (float)dn, fdT = (float)dT, fnr = (float)nr, fTr = (float)Tr;
  float dM[14];
  const float U0m1 = (Ux * Ux + Uy * Uy + Uz * Uz) / (U0 + 1.f);
  const float q = 4.f * fn * fT, iso = fdn * fT + fnr * fdT;
  dM[0] = (fdn * fTr - fnr * fdT) / (2.f * fT * fTr);
  dM[1] = fdn * U0 + fnr * U0m1;
  dM[2] = fn * Ux;
  dM[3] = fn * Uy;
  dM[4] = fn * Uz;
  dM[5] = q * U0 * Ux;
  dM[6] = q * U0 * Uy;
  dM[7] = q * U0 * Uz;
  dM[8] = q * Ux * Ux + iso;
  dM[9] = q * Ux * Uy;
  dM[10] = q * Ux * Uz;
  dM[11] = q * Uy * Uy + iso;
  dM[12] = q * Uy * Uz;
  dM[13] = q * Uz * Uz + iso;
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
