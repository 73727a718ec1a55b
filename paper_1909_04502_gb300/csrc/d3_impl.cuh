// Device helpers of the (3+1)-d massless steps (step3.cu: order 2; step3q.cu:
// order 3): layout, periodic images, the 4 x 4 Landau frame (Sec. 4) in FP64
// and in FP32 with an FP64 correction, and the Maxwell-Juttner moments of the
// bases kBasis3 / kBasis3o3 (App. B, d = 3, m = 0).
#pragma once
#include <cuda_runtime.h>

#include "d3.h"
#include "fpconv.cuh"

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
// v_i = (-1)^i det(B without row 0 and column i), each 3 x 3 minor expanded
// along row 1 over the six 2 x 2 minors c_ab of rows 2 and 3; B v = det(B) e_0,
// so det(B) = sum_i B[0][i] v_i.
template <typename R>
__device__ __forceinline__ void adj_col0(const R (&B)[4][4], R (&v)[4]) {
  const R c01 = B[2][0] * B[3][1] - B[2][1] * B[3][0], c02 = B[2][0] * B[3][2] - B[2][2] * B[3][0];
  const R c03 = B[2][0] * B[3][3] - B[2][3] * B[3][0], c12 = B[2][1] * B[3][2] - B[2][2] * B[3][1];
  const R c13 = B[2][1] * B[3][3] - B[2][3] * B[3][1], c23 = B[2][2] * B[3][3] - B[2][3] * B[3][2];
  v[0] = B[1][1] * c23 - B[1][2] * c13 + B[1][3] * c12;
  v[1] = -(B[1][0] * c23 - B[1][2] * c03 + B[1][3] * c02);
  v[2] = B[1][0] * c13 - B[1][1] * c03 + B[1][3] * c01;
  v[3] = -(B[1][0] * c12 - B[1][1] * c02 + B[1][2] * c01);
}

// d v / d l for B = A - l I: each minor differentiated through the diagonal
// entries it keeps (d det / d B_rr = cofactor of B_rr).
template <typename R>
__device__ __forceinline__ void dadj_col0(const R (&B)[4][4], R (&d)[4]) {
  d[0] = -((B[2][2] * B[3][3] - B[2][3] * B[3][2]) + (B[1][1] * B[3][3] - B[1][3] * B[3][1]) +
           (B[1][1] * B[2][2] - B[1][2] * B[2][1]));
  d[1] = (B[1][0] * B[3][3] - B[1][3] * B[3][0]) + (B[1][0] * B[2][2] - B[1][2] * B[2][0]);
  d[2] = (B[2][0] * B[3][3] - B[2][3] * B[3][0]) - (B[1][0] * B[2][1] - B[1][1] * B[2][0]);
  d[3] = -((B[2][0] * B[3][2] - B[2][2] * B[3][0]) + (B[1][0] * B[3][1] - B[1][1] * B[3][0]));
}

struct Macro3 {
  double n, T, eps, U[4];
  bool ok;
};

// Largest eigenvalue eps of A^a_b = T^ac eta_cb and its timelike eigenvector:
// Newton on p(l) = det(A - l I) from the ideal-fluid root for P = eps / 3,
// p'(l) = -(sum of the principal 3 x 3 minors of A - l I); U from the first
// column of adj(A - l I) (a right null vector), normalised to U.U = 1, U^0 > 0.
__device__ __forceinline__ Macro3 landau3(const double (&N)[4], const double (&Tm)[4][4]) {
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


// FP32 storage (g = f - f_ref, f_ref at (n_ref, rest, T_ref)): the Landau root
// in FP32 (Newton on det(A - l I) from the ideal-fluid root), then one Newton
// correction whose residual is evaluated in FP64: the cofactor vector v of
// B = A - l I at the FP32 root and p(l) = B[0] . v.  The eigenvector at the
// corrected root is v + dl dv/dl (dv/dl in FP32; the remainder is O(dl^2)),
// and from it, in FP64, nu^2 = v.v, w = v.N (n = w / nu) and the numerator
// of dn = n - n_ref = (w^2 - n_ref^2 nu^2) / (nu (w + n_ref nu)); the
// quotients, U = v / nu and dT = (d_eps - 3 T_ref dn) / (3 n) (from
// eps = 3 n T) in FP32.  About 50 FP64 operations per cell; conversions on
// the integer pipe (fpconv.cuh).
struct Macro3f {
  float U0, Ux, Uy, Uz, n, T, dn, dT;
  bool ok;
};

__device__ __forceinline__ Macro3f landau3f(const float (&N)[4], const float (&Tm)[4][4], const Scalars3& s) {
  const double nr = s.n_ref, Tr = s.T_ref, er = 3.0 * nr * Tr, Pr = nr * Tr;
  const float fnr = d2f(nr), fTr = d2f(Tr), fer = d2f(er), fPr = d2f(Pr);
  // the mixed tensor A = T eta in FP32 (reference diagonal added)
  float Af[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      float t = u <= v ? Tm[u][v] : Tm[v][u];
      if (u == v) t += (u == 0 ? fer : fPr);
      Af[u][v] = v == 0 ? t : -t;
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
  // FP64 residual at the FP32 root: B = A - l I with A's entries exact from
  // the FP32 sums and the FP64 reference
  const double ld = f2d(lam);
  const double d0 = ld - er, d1 = Pr + ld;
  double B[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const double t = f2d(u <= v ? Tm[u][v] : Tm[v][u]);
      B[u][v] = v == 0 ? t : -t;
    }
  B[0][0] = f2d(Tm[0][0]) - d0;
#pragma unroll
  for (int u = 1; u < 4; ++u) B[u][u] = -(f2d(Tm[u][u]) + d1);
  double vv[4];
  adj_col0(B, vv);
  const double p = B[0][0] * vv[0] + B[0][1] * vv[1] + B[0][2] * vv[2] + B[0][3] * vv[3];
  const float dl = -__fdividef(d2f(p), dpf);
  // the eigenvector at l + dl to first order
#pragma unroll
  for (int u = 0; u < 4; ++u) Bf[u][u] = Af[u][u] - lam;
  float dv[4];
  dadj_col0(Bf, dv);
  double vc[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) vc[u] = vv[u] + f2d(dl * dv[u]);
  const double nu2 = vc[0] * vc[0] - vc[1] * vc[1] - vc[2] * vc[2] - vc[3] * vc[3];
  const double w = vc[0] * (nr + f2d(N[0])) - vc[1] * f2d(N[1]) - vc[2] * f2d(N[2]) - vc[3] * f2d(N[3]);
  const double num = fma(w, w, -(nr * nr) * nu2);
  const double deps = d0 + f2d(dl);
  // FP32 quotients
  const float fnu2 = d2f(nu2);
  const float inu = rsqrtf(fnu2);
  const float fnu = fnu2 * inu;
  const float sgn = __double2hiint(vc[0]) < 0 ? -1.f : 1.f;
  const float fw = sgn * d2f(w);
  Macro3f M;
  M.n = fw * inu;
  M.dn = __fdividef(d2f(num), fnu * (fw + fnr * fnu));
  M.dT = __fdividef(d2f(deps) - 3.f * fTr * M.dn, 3.f * M.n);
  M.T = fTr + M.dT;
  const float su = sgn * inu;
  M.U0 = d2f(vc[0]) * su;
  M.Ux = d2f(vc[1]) * su;
  M.Uy = d2f(vc[2]) * su;
  M.Uz = d2f(vc[3]) * su;
  M.ok = (__double2hiint(nu2) > 0) && (M.n > 0.f) && (M.T > 0.f) && isfinite(M.T) && isfinite(M.dn) &&
         isfinite(M.n);
  return M;
}

// The rank-3 moments <p^a p^b p^c> = n (24 T^2 U^a U^b U^c - 4 T^2 (eta^ab U^c
// + eta^ac U^b + eta^bc U^a)) for the order-3 members of kBasis3o3: p0 p^i p^j
// (i <= j) and p^i p^j p^k (i <= j <= k), spatial indices 1..3.
__device__ __forceinline__ int o3_index(int k, int e) {
  // members 14-19: p0 (xx xy xz yy yz zz); 20-29: xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz
  const int p2[6][2] = {{1, 1}, {1, 2}, {1, 3}, {2, 2}, {2, 3}, {3, 3}};
  const int p3[10][3] = {{1, 1, 1}, {1, 1, 2}, {1, 1, 3}, {1, 2, 2}, {1, 2, 3},
                         {1, 3, 3}, {2, 2, 2}, {2, 2, 3}, {2, 3, 3}, {3, 3, 3}};
  return k < 20 ? p2[k - 14][e] : p3[k - 20][e];
}

// Full moments of the basis (FP64 storage): K = 14 (order 2) or 30 (order 3).
template <int K>
__device__ __forceinline__ void mj_full3(double n, double T, const double (&U)[4], double (&M)[K]) {
  double M14[14];
  mj_moments3(n, T, U, M14);
#pragma unroll
  for (int k = 0; k < 14; ++k) M[k] = M14[k];
  if constexpr (K == 30) {
    const double q = 24.0 * n * T * T, r = 4.0 * n * T * T;
#pragma unroll
    for (int k = 14; k < 20; ++k) {
      const int i = o3_index(k, 0), j = o3_index(k, 1);
      M[k] = q * U[0] * U[i] * U[j] + (i == j ? r * U[0] : 0.0);
    }
#pragma unroll
    for (int k = 20; k < 30; ++k) {
      const int i = o3_index(k, 0), j = o3_index(k, 1), l = o3_index(k, 2);
      M[k] = q * U[i] * U[j] * U[l] + r * ((i == j ? U[l] : 0.0) + (i == l ? U[j] : 0.0) + (j == l ? U[i] : 0.0));
    }
  }
}

// Differences dM = M(n, U, T) - M(n_ref, rest, T_ref) (FP32 storage), each
// written so that it is accurate relative to itself given accurate dn, dT:
//   <1>: (dn T_ref - n_ref dT) / (2 T T_ref);  <p0>: dn U0 + n_ref (U0 - 1);
//   <p^i p^i>: 4nT (U^i)^2 + dn T + n_ref dT;
//   <p0 p^i p^i>: 24 n T^2 U0 (U^i)^2 + 4 (n T^2 (U0 - 1) + dn T^2 + n_ref dT (T + T_ref));
//   the others vanish at rest and need no rearrangement.
template <int K>
__device__ __forceinline__ void mj_delta3(const Macro3f& M, float nr, float Tr, float (&dM)[K]) {
  const float U[4] = {M.U0, M.Ux, M.Uy, M.Uz};
  const float n = M.n, T = M.T, dn = M.dn, dT = M.dT;
  const float U0m1 = (M.Ux * M.Ux + M.Uy * M.Uy + M.Uz * M.Uz) / (M.U0 + 1.f);
  const float q = 4.f * n * T, iso = dn * T + nr * dT;
  dM[0] = (dn * Tr - nr * dT) / (2.f * T * Tr);
  dM[1] = dn * M.U0 + nr * U0m1;
  dM[2] = n * M.Ux;
  dM[3] = n * M.Uy;
  dM[4] = n * M.Uz;
  dM[5] = q * M.U0 * M.Ux;
  dM[6] = q * M.U0 * M.Uy;
  dM[7] = q * M.U0 * M.Uz;
  dM[8] = q * M.Ux * M.Ux + iso;
  dM[9] = q * M.Ux * M.Uy;
  dM[10] = q * M.Ux * M.Uz;
  dM[11] = q * M.Uy * M.Uy + iso;
  dM[12] = q * M.Uy * M.Uz;
  dM[13] = q * M.Uz * M.Uz + iso;
  if constexpr (K == 30) {
    const float q3 = 24.f * n * T * T, r3 = 4.f * n * T * T;
    const float iso3 = 4.f * (n * T * T * U0m1 + dn * T * T + nr * dT * (T + Tr));
#pragma unroll
    for (int k = 14; k < 20; ++k) {
      const int i = o3_index(k, 0), j = o3_index(k, 1);
      dM[k] = q3 * M.U0 * U[i] * U[j] + (i == j ? iso3 : 0.f);
    }
#pragma unroll
    for (int k = 20; k < 30; ++k) {
      const int i = o3_index(k, 0), j = o3_index(k, 1), l = o3_index(k, 2);
      dM[k] = q3 * U[i] * U[j] * U[l] + r3 * ((i == j ? U[l] : 0.f) + (i == l ? U[j] : 0.f) + (j == l ? U[i] : 0.f));
    }
  }
}

// The collision frame from the 14 moment sums m = N0 Nx Ny Nz T00 T0x T0y
// T0z Txx Txy Txz Tyy Tyz Tzz (of f in FP64 storage, of g = f - f_ref in FP32
// storage): the moments Mk of the K-member basis that the equilibrium H Mk
// needs (full moments in FP64, differences from the reference in FP32), and
// tau^-1 U (zero where the cell has no Landau frame, which leaves it
// unrelaxed).  Returns whether the frame exists.
// A cell without a physical Landau frame is left unrelaxed (Omega = 0); its
// frame is replaced by the reference state (rest, n_ref or 1, T_ref) so
// that the equilibrium and Omega stay finite (0 * NaN is not 0).
__device__ __forceinline__ void unphysical_to_reference3(const Scalars3& s, Macro3& M) {
  M.n = s.n_ref > 0.0 ? s.n_ref : 1.0;
  M.T = s.T_ref;
  M.eps = 3.0 * M.n * M.T;
  M.U[0] = 1.0;
  M.U[1] = M.U[2] = M.U[3] = 0.0;
}
__device__ __forceinline__ void unphysical_to_reference3(const Scalars3& s, Macro3f& M) {
  M.n = (float)(s.n_ref > 0.0 ? s.n_ref : 1.0);
  M.T = s.f_T_ref;
  M.dn = M.dT = 0.f;
  M.U0 = 1.f;
  M.Ux = M.Uy = M.Uz = 0.f;
}

template <typename S, int K>
__device__ __forceinline__ bool frame3(const S (&m)[14], const Scalars3& s, S (&Mk)[K], S& kU0, S (&kU)[3]) {
  if constexpr (sizeof(S) == 8) {
    const double N[4] = {m[0], m[1], m[2], m[3]};
    const double Tm[4][4] = {{m[4], m[5], m[6], m[7]},
                             {m[5], m[8], m[9], m[10]},
                             {m[6], m[9], m[11], m[12]},
                             {m[7], m[10], m[12], m[13]}};
    Macro3 M = landau3(N, Tm);
    if (!M.ok) unphysical_to_reference3(s, M);
    mj_full3<K>(M.n, M.T, M.U, Mk);
    const double kt = M.ok ? 1.0 / s.tau : 0.0;
    kU0 = kt * M.U[0];
    kU[0] = kt * M.U[1];
    kU[1] = kt * M.U[2];
    kU[2] = kt * M.U[3];
    return M.ok;
  } else {
    const float N[4] = {m[0], m[1], m[2], m[3]};
    const float Tm[4][4] = {{m[4], m[5], m[6], m[7]},
                            {m[5], m[8], m[9], m[10]},
                            {m[6], m[9], m[11], m[12]},
                            {m[7], m[10], m[12], m[13]}};
    Macro3f M = landau3f(N, Tm, s);
    if (!M.ok) unphysical_to_reference3(s, M);
    mj_delta3<K>(M, s.f_n_ref, s.f_T_ref, Mk);
    const float kt = M.ok ? s.f_inv_tau : 0.f;
    kU0 = kt * M.U0;
    kU[0] = kt * M.Ux;
    kU[1] = kt * M.Uy;
    kU[2] = kt * M.Uz;
    return M.ok;
  }
}

// Walsh-Hadamard transform in place: v[c] <- sum_s (-1)^{popcount(c & s)} v[s]
template <typename S, int L>
__device__ __forceinline__ void fwht(S (&v)[L]) {
#pragma unroll
  for (int hb = 1; hb < L; hb <<= 1)
#pragma unroll
    for (int q = 0; q < L; ++q)
      if (!(q & hb)) {
        const S u = v[q], w = v[q | hb];
        v[q] = u + w;
        v[q | hb] = u - w;
      }
}

// the moment sums of a run of 8 from its transformed values F (F[c] = sum_s
// chi_c(s) f_s) and its first member's monomials c (Tables3::mono order)
template <typename S, typename C>
__device__ __forceinline__ void moments_run8(const S (&F)[8], const C* c, S (&m)[14]) {
  m[0] = fma((S)c[0], F[0], m[0]);
  m[1] = fma((S)c[1], F[1], m[1]);
  m[2] = fma((S)c[2], F[2], m[2]);
  m[3] = fma((S)c[3], F[4], m[3]);
  m[4] = fma((S)c[4], F[0], m[4]);
  m[5] = fma((S)c[5], F[1], m[5]);
  m[6] = fma((S)c[6], F[2], m[6]);
  m[7] = fma((S)c[7], F[4], m[7]);
  m[8] = fma((S)c[8], F[0], m[8]);
  m[9] = fma((S)c[9], F[3], m[9]);
  m[10] = fma((S)c[10], F[5], m[10]);
  m[11] = fma((S)c[11], F[0], m[11]);
  m[12] = fma((S)c[12], F[6], m[12]);
  m[13] = fma((S)c[13], F[0], m[13]);
}

// FP32 storage: the periodic images of a cell next to a face, copied from the
// values the thread has just stored for the cell itself, B populations at a
// time so that B loads are in flight (one at a time, each waits on the L2
// round trip of the one before, as the stores in between may alias them).
template <int QT, int B>
__device__ __forceinline__ void images_from_stored(const Scalars3& s, float* out, long long si, int x, int y, int z) {
  int ix[2], iy[2], iz[2];
  const int nx2 = images1(x, s.nx, s.h, ix), ny2 = images1(y, s.ny, s.h, iy), nz2 = images1(z, s.nz, s.h, iz);
  if (nx2 + ny2 + nz2 == 0) return;
  long long img[26];
  int nimg = 0;
  for (int cz = -1; cz < nz2; ++cz)
    for (int cy = -1; cy < ny2; ++cy)
      for (int cx = -1; cx < nx2; ++cx) {
        if (cx < 0 && cy < 0 && cz < 0) continue;
        img[nimg++] = sidx3(s, cx < 0 ? x : ix[cx], cy < 0 ? y : iy[cy], cz < 0 ? z : iz[cz]);
      }
  static_assert(QT % B == 0, "whole batches");
  const long long P = s.plane;
  for (int i0 = 0; i0 < QT; i0 += B) {
    float v[B];
#pragma unroll
    for (int j = 0; j < B; ++j) v[j] = out[(long long)(i0 + j) * P + si];
#pragma unroll
    for (int j = 0; j < B; ++j) {
      float* oi = out + (long long)(i0 + j) * P;
      for (int m = 0; m < nimg; ++m) oi[img[m]] = v[j];
    }
  }
}

// periodic images of a cell (every side at least h: at most 26)
__device__ __forceinline__ int cell_images(const Scalars3& s, int x, int y, int z, long long (&img)[26]) {
  int ix[2], iy[2], iz[2];
  const int nx2 = images1(x, s.nx, s.h, ix), ny2 = images1(y, s.ny, s.h, iy), nz2 = images1(z, s.nz, s.h, iz);
  int nimg = 0;
  for (int cz = -1; cz < nz2; ++cz)
    for (int cy = -1; cy < ny2; ++cy)
      for (int cx = -1; cx < nx2; ++cx) {
        if (cx < 0 && cy < 0 && cz < 0) continue;
        img[nimg++] = sidx3(s, cx < 0 ? x : ix[cx], cy < 0 ? y : iy[cy], cz < 0 ? z : iz[cz]);
      }
  return nimg;
}

}  // namespace
}  // namespace rlbm
