// (1+1)-dimensional massless RLBM step (include/rlbm.h, rlbm1_*): the d = 1
// case of Sec. 5-6.2 of arXiv:1909.04502 on the App. H "(1+1) dimensions"
// quadratures.
//
// Populations p_{j,s} = p0_j (1, s), s = +-1, on the N shells of the order-N
// table; every population moves one cell per step in direction s.  The
// equilibrium is the massless limit of the order-N expansion (Sec. 5.2, Eq.
// mj-expanded-1D-massless).  On these quadratures the Q = 2N populations and
// the 2N members phi_{a,s} = (p0)^a sign(p^x)^s (a = 1..N) of the limit basis
// form a square system, and the quadrature integrates every product the
// expansion needs exactly, so the discrete equilibrium is the unique f with
//   sum_i f_i phi_{a,s}(p_i) = M_{a,s} = int f_MJ phi_{a,s} dp/p0
//     = n (a-1)! T^(a-1) {cosh, sinh}(a theta),   U = (cosh theta, sinh theta),
// i.e. f^eq = H M with H the inverse of the matrix phi_{a,s}(p_i) (built on
// the host in double-double).  Landau frame: the largest eigenvalue of the
// 2 x 2 mixed tensor, in closed form; EOS eps = P = n T (d = 1, m = 0).
//
// Layout: one plane per population, nx interior cells with one halo cell on
// each side (a periodic image or, for free-flow ends and equilibrium walls,
// a copy of the end cell), so the pull reads base + x - s.  FP32 storage
// holds g = f - f_ref (f_ref the equilibrium of (n_ref, rest, T_ref)) and
// steps in FP32 from differences to that state (k_step1f); FP64 storage
// steps in FP64 (Q <= 10 populations per cell).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "../../include/rlbm.h"
#include "dd.h"

namespace rlbm1 {

constexpr int kMaxN = 5;               // App. H tables: orders 2 ... 5
constexpr int kMaxQ = 2 * kMaxN;
constexpr int kThreads = 128;
constexpr int kStep1CPT = 2;           // cells per thread of the FP32-storage step

// App. H, (1+1) dimensions: shells and per-direction weights.  Order 4 is
// printed with its columns exchanged (the printed weights are the roots of
// L_4); it is stored here read back.
struct Table1 {
  int N;
  double p0[kMaxN];
  double w[kMaxN];
};
const Table1 kTables[] = {
    {2, {3.414213562373095048, 0.585786437626904951}, {0.042893218813452475, 1.457106781186547524}},
    {3, {6.289945082937479196, 0.415774556783479083, 2.294280360279041719},
     {0.001651724516604877, 1.710285053107483686, 0.121396555709244769}},
    {4, {0.322547689619392311, 4.536620296921127983, 9.395070912301133129, 1.745761101158346575},
     {1.869968763544262523, 0.008571999852268322, 0.000057401877068880, 0.204735168059733606}},
    {5, {0.26356031971814091020, 3.59642577104072208122, 1.41340305910651679221, 7.08581000585883755692,
         12.6408008442757826594},
     {1.97964401902679930651, 0.02111608983931054815, 0.28206165857260368669, 0.00050971712153383997,
      0.00000184877308595198}},
};

template <typename S>
struct Tab {
  double p0[kMaxQ];       // shell energy of population i
  int s[kMaxQ];           // direction (+1 / -1)
  double H[kMaxQ][kMaxQ]; // f^eq_i - f_ref,i = sum_k H_ik dM_k  (k = 2 (a - 1) + b)
  S Hs[kMaxQ][kMaxQ];     // the same in the storage type
  // the FP32-storage step: p0 and p0^2 as FP32 (hi, lo) pairs
  float w1h[kMaxQ], w1l[kMaxQ], w2h[kMaxQ], w2l[kMaxQ];
};

struct Sc {
  int Q, N, nx, P;         // populations, order, cells, plane stride (nx + 2)
  int boundary;            // RLBM_BC_*
  double tau;
  double wall_T[2];        // equilibrium walls: first / last cell temperature (0: own T)
  double n_ref, T_ref;     // reference state of FP32 storage (n_ref = 0: none)
  double N0_ref, T00_ref;  // its moments: N^0 = n_ref, T^00 = T^xx = n_ref T_ref (eps = P)
  // FP32 copies for the FP32-storage step: n_ref, T_ref, eps_ref = n_ref T_ref,
  // 1 / tau, the wall temperatures and their differences from T_ref
  float f_n_ref, f_T_ref, f_Er, f_inv_tau;
  float f_wall_T[2], f_wall_dT[2];
};

// M_{a,b} - M_{a,b}(n_ref, rest, T_ref) for a = 1..N, b = 0, 1.
__host__ __device__ inline void moments_dM(const Sc& s, double n, double U0, double Ux, double T,
                                           double* dM) {
  const double E = U0 + Ux;               // exp(theta)
  const double Ei = 1.0 / E;              // exp(-theta) = U0 - Ux, without cancellation
  double Ea = 1.0, Eia = 1.0, fact = 1.0, Tp = 1.0, Trp = 1.0;
  for (int a = 1; a <= s.N; ++a) {
    Ea *= E;
    Eia *= Ei;
    if (a > 1) {
      fact *= (double)(a - 1);
      Tp *= T;
      Trp *= s.T_ref;
    }
    const double c = n * fact * Tp;
    dM[2 * (a - 1)] = 0.5 * c * (Ea + Eia) - s.n_ref * fact * Trp;
    dM[2 * (a - 1) + 1] = 0.5 * c * (Ea - Eia);
  }
}

struct Macro1 {
  double n, U0, Ux, T, eps, N0, Nx, T00, T0x;
  bool ok;
};

// Steps 1-4 of Sec. 6.2 from the streamed populations (shifted by f_ref in
// FP32 storage): moments, the Landau frame of the 2 x 2 mixed tensor
// A = [[T00, -T0x], [T0x, -Txx]] (largest root of
// l^2 - (T00 - Txx) l + T0x^2 - T00 Txx, eigenvector (Txx + l, T0x)),
// n = U.N and T = eps / n.
template <typename S>
__device__ inline Macro1 macro1(const Tab<S>& tb, const Sc& s, const S* g) {
  double N0 = 0.0, Nx = 0.0, T00 = 0.0, T0x = 0.0;
  for (int i = 0; i < s.Q; ++i) {
    const double f = (double)g[i], p = tb.p0[i];
    const double fp = f * p;
    N0 += fp;
    T00 += fp * p;
    if (tb.s[i] > 0) { Nx += fp; T0x += fp * p; }
    else { Nx -= fp; T0x -= fp * p; }
  }
  Macro1 M;
  M.N0 = s.N0_ref + N0;
  M.Nx = Nx;
  M.T00 = s.T00_ref + T00;
  M.T0x = T0x;
  const double Txx = M.T00;               // p^x p^x = p0 p0 on every population
  const double disc = (M.T00 + Txx) * (M.T00 + Txx) - 4.0 * M.T0x * M.T0x;
  const double l = 0.5 * ((M.T00 - Txx) + sqrt(fmax(disc, 0.0)));
  const double v0 = Txx + l, v1 = M.T0x;
  const double nu2 = v0 * v0 - v1 * v1;
  const double inu = nu2 > 0.0 ? rsqrt(nu2) : 0.0;
  M.U0 = v0 * inu;
  M.Ux = v1 * inu;
  M.eps = l;
  M.n = M.U0 * M.N0 - M.Ux * M.Nx;
  M.T = l / M.n;
  M.ok = disc > 0.0 && nu2 > 0.0 && v0 > 0.0 && l > 0.0 && M.n > 0.0 && isfinite(M.T);
  return M;
}

template <typename S>
__device__ inline S feq_i(const Tab<S>& tb, const Sc& s, int i, const double* dM) {
  if constexpr (sizeof(S) == 8) {
    double f = 0.0;
    for (int k = 0; k < s.Q; ++k) f = fma(tb.H[i][k], dM[k], f);
    return f;
  } else {
    float f = 0.f;
    for (int k = 0; k < s.Q; ++k) f = fmaf(tb.Hs[i][k], (float)dM[k], f);
    return f;
  }
}

// Store cell x of plane i and its halo image (periodic: the opposite halo
// cell; free-flow / walls: the halo cell beside an end cell).
template <typename S>
__device__ inline void store1(const Sc& s, S* out, int i, int x, S v) {
  S* row = out + (long long)i * s.P;
  row[x + 1] = v;
  if (s.boundary == RLBM_BC_PERIODIC) {
    if (x == 0) row[s.nx + 1] = v;
    if (x == s.nx - 1) row[0] = v;
  } else {
    if (x == 0) row[0] = v;
    if (x == s.nx - 1) row[s.nx + 1] = v;
  }
}

template <typename S>
__global__ void __launch_bounds__(kThreads) k_step1(const __grid_constant__ Tab<S> tb, const __grid_constant__ Sc s,
                                                    const S* __restrict__ fin, S* __restrict__ fout,
                                                    unsigned long long* status) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= s.nx) return;
  S g[kMaxQ];
  for (int i = 0; i < s.Q; ++i) g[i] = fin[(long long)i * s.P + x + 1 - tb.s[i]];   // pull
  const Macro1 M = macro1<S>(tb, s, g);
  if (!M.ok) {
    atomicAdd(status, 1ULL);                                 // left unrelaxed (Omega = 0)
    for (int i = 0; i < s.Q; ++i) store1<S>(s, fout, i, x, g[i]);
    return;
  }
  double dM[kMaxQ];
  const bool wall = s.boundary == RLBM_BC_EQWALL_X && (x == 0 || x == s.nx - 1);
  if (wall) {
    const double Tw = s.wall_T[x == 0 ? 0 : 1] > 0.0 ? s.wall_T[x == 0 ? 0 : 1] : M.T;
    moments_dM(s, M.n, 1.0, 0.0, Tw, dM);
    for (int i = 0; i < s.Q; ++i) store1<S>(s, fout, i, x, feq_i<S>(tb, s, i, dM));
    return;
  }
  moments_dM(s, M.n, M.U0, M.Ux, M.T, dM);
  const double itau = 1.0 / s.tau;
  for (int i = 0; i < s.Q; ++i) {
    const S om = (S)((M.U0 - (double)tb.s[i] * M.Ux) * itau);   // p.U / (p0 tau)
    const S fe = feq_i<S>(tb, s, i, dM);
    store1<S>(s, fout, i, x, g[i] + om * (fe - g[i]));
  }
}

// FP32 storage (g = f - f_ref): the step in FP32 throughout, with every
// quantity formed from differences to the reference state (n_ref, rest,
// T_ref), so that each FP32 rounding is of the size of the deviation, like
// the storage of g itself.  With T^xx = T^00 = E on every population the
// largest eigenvalue is l = sqrt(E^2 - T0x^2), E = eps_ref + dE, and
//   l - eps_ref = (dE (2 eps_ref + dE) - T0x^2) / (l + eps_ref),
// the eigenvector v = (E + l, T0x), nu^2 = v.v,
//   n - n_ref = (v0 dN0 - v1 Nx + n_ref v1^2 / (v0 + nu)) / nu,
//   T - T_ref = (l - eps_ref - (n - n_ref) T_ref) / n      (eps = n T),
// and the moment differences, with E_th = U0 + Ux = e^theta,
// E_th - 1 = Ux + Ux^2 / (U0 + 1) and (E_th^a - 1) = (E_th - 1) sum_{j<a} E_th^j:
//   dM_{a,0} / (a-1)! = n T^(a-1) (E_th^a - 1)^2 / (2 E_th^a) + dn T^(a-1)
//                       + n_ref (T^(a-1) - T_ref^(a-1)),
//   dM_{a,1} / (a-1)! = n T^(a-1) (E_th^a - 1)(E_th^a + 1) / (2 E_th^a),
// T^(a-1) - T_ref^(a-1) = T (T^(a-2) - T_ref^(a-2)) + T_ref^(a-2) dT.
// The FP64-storage step (k_step1<double>) keeps the FP64 arithmetic.
template <int N>
__device__ __forceinline__ void moments_dM_f32(float n, float dn, float T, float dT, float Em1, float Eth,
                                               float nr, float Tr, float (&dM)[2 * N]) {
  float Ea = 1.f, Sa = 0.f, Ta = 1.f, Tra = 1.f, DTa = 0.f, fact = 1.f;
#pragma unroll
  for (int a = 1; a <= N; ++a) {
    Sa += Ea;                              // sum_{j<a} E_th^j
    Ea *= Eth;                             // E_th^a
    if (a > 1) {
      DTa = T * DTa + Tra * dT;            // T^(a-1) - T_ref^(a-1)
      Ta *= T;
      Tra *= Tr;
      fact *= (float)(a - 1);
    }
    const float Em1a = Em1 * Sa;           // E_th^a - 1
    const float h = __fdividef(0.5f * n * Ta * Em1a, Ea);
    dM[2 * (a - 1)] = fact * (h * Em1a + dn * Ta + nr * DTa);
    dM[2 * (a - 1) + 1] = fact * h * (Ea + 1.f);
  }
}

// Store the Q values of cell x, and for an end cell its halo image (as
// store1), the image stores behind one branch that interior warps skip.
template <int Q>
__device__ __forceinline__ void store_cell1f(const Sc& s, float* out, int x, const float (&v)[Q]) {
#pragma unroll
  for (int i = 0; i < Q; ++i) out[(long long)i * s.P + x + 1] = v[i];
  if (x == 0 || x == s.nx - 1) {
    const bool per = s.boundary == RLBM_BC_PERIODIC;
    if (x == 0) {
      const int hx = per ? s.nx + 1 : 0;
#pragma unroll
      for (int i = 0; i < Q; ++i) out[(long long)i * s.P + hx] = v[i];
    }
    if (x == s.nx - 1) {
      const int hx = per ? 0 : s.nx + 1;
#pragma unroll
      for (int i = 0; i < Q; ++i) out[(long long)i * s.P + hx] = v[i];
    }
  }
}

// One cell of the FP32-storage step from its pulled populations g.
template <int N>
__device__ __forceinline__ void cell1f(const Tab<float>& tb, const Sc& s, const float (&g)[2 * N], int x,
                                       float* __restrict__ fout, unsigned long long* status) {
  constexpr int Q = 2 * N;
  // the four moment sums, compensated: every product g p0^k split exactly
  // (FMA), every addition exactly (two-sum), the errors and the lo parts of
  // p0^k summed in a second register.  Plain FP32 sums measured 2.5x the
  // error of exact ones against the oracle (their rounding is not a
  // consistent change of the state).  Population i = 2j + b is shell j
  // moving in direction +1 (b = 0) or -1 (b = 1) (build_tables), so the sums
  // run separately over the two directions -- A: sum g p0, B: sum g p0^2 --
  // and N^0 = A+ + A-, N^x = A+ - A-, T^00 = B+ + B-, T^0x = B+ - B- are
  // formed at the end, each in one two-sum.
  float m[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};   // A+, A-, B+, B-
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int b = i & 1;
    const float p1 = __fmul_rn(g[i], tb.w1h[i]);   // not contracted into the sums below
    const float p2 = __fmul_rn(g[i], tb.w2h[i]);
    const float r1 = fmaf(g[i], tb.w1l[i], fmaf(g[i], tb.w1h[i], -p1));   // p1's error + the lo part
    const float r2 = fmaf(g[i], tb.w2l[i], fmaf(g[i], tb.w2h[i], -p2));
    const float p[2] = {p1, p2};
    const float r[2] = {r1, r2};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int a = 2 * k + b;
      const float t = m[a] + p[k];
      const float bb = t - m[a];
      const float err = (m[a] - (t - bb)) + (p[k] - bb);
      m[a] = t;
      c[a] += err + r[k];
    }
  }
  // (hi_a + lo_a) + sgn (hi_b + lo_b), the hi parts added exactly
  auto combine = [](float ha, float la, float hb, float lb) {
    const float t = ha + hb;
    const float bb = t - ha;
    const float err = (ha - (t - bb)) + (hb - bb);
    return t + (err + (la + lb));
  };
  const float dN0 = combine(m[0], c[0], m[1], c[1]), Nx = combine(m[0], c[0], -m[1], -c[1]);
  const float dE = combine(m[2], c[2], m[3], c[3]), T0x = combine(m[2], c[2], -m[3], -c[3]);
  const float Er = s.f_Er, nr = s.f_n_ref, Tr = s.f_T_ref;
  const float E = Er + dE;
  const float q = (E - T0x) * (E + T0x);
  const float l = sqrtf(fmaxf(q, 0.f));
  const float dl = __fdividef(fmaf(dE, 2.f * Er + dE, -T0x * T0x), l + Er);
  const float v0 = E + l, v1 = T0x;
  const float nu2 = (v0 - v1) * (v0 + v1);
  const float inu = rsqrtf(nu2);
  const float nu = nu2 * inu;
  const float dn = (v0 * dN0 - v1 * Nx + __fdividef(nr * v1 * v1, v0 + nu)) * inu;
  const float n = nr + dn;
  const float dT = __fdividef(dl - dn * Tr, n);
  const float T = Tr + dT;
  const float U0 = v0 * inu, Ux = v1 * inu;
  const bool ok = q > 0.f && nu2 > 0.f && v0 > 0.f && l > 0.f && n > 0.f && T > 0.f && isfinite(T) &&
                  isfinite(U0) && isfinite(dn);
  if (!ok) {
    atomicAdd(status, 1ULL);                                 // left unrelaxed (Omega = 0)
    store_cell1f<Q>(s, fout, x, g);
    return;
  }
  // f^eq of the pair (shell j, +1), (shell j, -1) from the first row: the
  // rows differ by the sign of the odd members (phi_{a,1} changes sign with
  // the direction; exact in the table, checked on the host), so
  // f^eq = E +- O with E, O the even- and odd-member partial sums
  auto feq_pair = [&](int j, const float (&dM)[Q], float& fp, float& fm) {
    float E = 0.f, O = 0.f;
#pragma unroll
    for (int k = 0; k < Q; k += 2) E = fmaf(tb.Hs[2 * j][k], dM[k], E);
#pragma unroll
    for (int k = 1; k < Q; k += 2) O = fmaf(tb.Hs[2 * j][k], dM[k], O);
    fp = E + O;
    fm = E - O;
  };
  float dM[Q], o[Q];
  const bool wall = s.boundary == RLBM_BC_EQWALL_X && (x == 0 || x == s.nx - 1);
  if (wall) {
    // f^eq(n, rest, T_w): theta = 0, T_w the prescribed wall temperature or the cell's own
    const int side = x == 0 ? 0 : 1;
    const bool fix = s.f_wall_T[side] > 0.f;
    const float Tw = fix ? s.f_wall_T[side] : T, dTw = fix ? s.f_wall_dT[side] : dT;
    moments_dM_f32<N>(n, dn, Tw, dTw, 0.f, 1.f, nr, Tr, dM);
#pragma unroll
    for (int j = 0; j < N; ++j) feq_pair(j, dM, o[2 * j], o[2 * j + 1]);
    store_cell1f<Q>(s, fout, x, o);
    return;
  }
  const float Em1 = Ux + __fdividef(Ux * Ux, U0 + 1.f);     // e^theta - 1
  moments_dM_f32<N>(n, dn, T, dT, Em1, 1.f + Em1, nr, Tr, dM);
  const float kt = s.f_inv_tau;
  const float omp = kt * (U0 - Ux), omm = kt * (U0 + Ux);   // p.U / (p0 tau), directions +1 and -1
#pragma unroll
  for (int j = 0; j < N; ++j) {
    float fp, fm;
    feq_pair(j, dM, fp, fm);
    o[2 * j] = fmaf(omp, fp - g[2 * j], g[2 * j]);
    o[2 * j + 1] = fmaf(omm, fm - g[2 * j + 1], g[2 * j + 1]);
  }
  store_cell1f<Q>(s, fout, x, o);
}

// CPT cells per thread, kThreads apart: every thread issues the pulls of
// all its cells before it computes, so that more loads are in flight.  On
// 2^24 cells two cells per thread were 2-5 % faster than one (orders 2-5),
// four and eight slower; the step is bound by the compensated sums' issue
// rather than by loads in flight.
template <int N, int CPT>
__global__ void __launch_bounds__(kThreads) k_step1f(const __grid_constant__ Tab<float> tb,
                                                     const __grid_constant__ Sc s, const float* __restrict__ fin,
                                                     float* __restrict__ fout, unsigned long long* status) {
  constexpr int Q = 2 * N;
  const int x0 = blockIdx.x * (kThreads * CPT) + threadIdx.x;
  float g[CPT][Q];
#pragma unroll
  for (int c = 0; c < CPT; ++c) {
    const int x = x0 + c * kThreads;
    if (x < s.nx) {
#pragma unroll
      for (int i = 0; i < Q; ++i) g[c][i] = __ldg(fin + (long long)i * s.P + x + 2 * (i & 1));   // pull from x - s
    }
  }
#pragma unroll
  for (int c = 0; c < CPT; ++c) {
    const int x = x0 + c * kThreads;
    if (x < s.nx) cell1f<N>(tb, s, g[c], x, fout, status);
  }
}

template <typename S>
__global__ void __launch_bounds__(kThreads) k_init1(const __grid_constant__ Tab<S> tb, const __grid_constant__ Sc s,
                                                    const double* n, const double* ux, const double* T, S* fout,
                                                    unsigned long long* status) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= s.nx) return;
  const double u = ux[x];
  const bool ok = u * u < 1.0 && n[x] > 0.0 && T[x] > 0.0;
  if (!ok) atomicAdd(status, 1ULL);
  const double gam = ok ? rsqrt(1.0 - u * u) : 1.0;
  double dM[kMaxQ];
  moments_dM(s, n[x], gam, gam * u, T[x], dM);
  for (int i = 0; i < s.Q; ++i) store1<S>(s, fout, i, x, feq_i<S>(tb, s, i, dM));
}

// Fields of the streamed populations (pull = 1) or of the stored ones:
// out[8][nx] = n, ux, T, eps, N0, Nx, T00, T0x (n NaN without a Landau frame).
template <typename S>
__global__ void __launch_bounds__(kThreads) k_fields1(const __grid_constant__ Tab<S> tb, const __grid_constant__ Sc s,
                                                      const S* __restrict__ fin, int pull, double* out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= s.nx) return;
  S g[kMaxQ];
  for (int i = 0; i < s.Q; ++i) g[i] = fin[(long long)i * s.P + x + 1 - (pull ? tb.s[i] : 0)];
  const Macro1 M = macro1<S>(tb, s, g);
  const int nx = s.nx;
  out[x] = M.ok ? M.n : __longlong_as_double(0x7ff8000000000000LL);
  out[nx + x] = M.Ux / M.U0;
  out[2 * nx + x] = M.T;
  out[3 * nx + x] = M.eps;
  out[4 * nx + x] = M.N0;
  out[5 * nx + x] = M.Nx;
  out[6 * nx + x] = M.T00;
  out[7 * nx + x] = M.T0x;
}

// Host: the order-N table and H = inverse of phi_{a,b}(p_i) in double-double.
bool build_tables(int order, std::vector<double>* p0, std::vector<int>* sgn, std::vector<double>* w,
                  std::vector<double>* H) {
  const Table1* t = nullptr;
  for (const auto& tt : kTables)
    if (tt.N == order) t = &tt;
  if (!t) return false;
  const int Q = 2 * order;
  p0->clear();
  sgn->clear();
  w->clear();
  // population 2j + b: shell j, direction +1 (b = 0) or -1 (b = 1); the
  // FP32-storage step takes this order as given
  for (int j = 0; j < order; ++j)
    for (int s : {1, -1}) {
      p0->push_back(t->p0[j]);
      sgn->push_back(s);
      w->push_back(0.5 * t->w[j]);
    }
  // A[k][i] = phi_k(p_i), k = 2 (a - 1) + b; H = A^-1 by Gauss-Jordan with
  // partial pivoting
  using rlbm::dd;
  std::vector<dd> A((size_t)Q * 2 * Q);
  for (int k = 0; k < Q; ++k) {
    const int a = k / 2 + 1, b = k % 2;
    for (int i = 0; i < Q; ++i) {
      dd v(1.0);
      for (int e = 0; e < a; ++e) v = v * dd((*p0)[i]);
      if (b && (*sgn)[i] < 0) v = -v;
      A[(size_t)k * 2 * Q + i] = v;
    }
    for (int i = 0; i < Q; ++i) A[(size_t)k * 2 * Q + Q + i] = dd(i == k ? 1.0 : 0.0);
  }
  for (int c = 0; c < Q; ++c) {
    int piv = c;
    for (int r = c + 1; r < Q; ++r)
      if (std::fabs(A[(size_t)r * 2 * Q + c].hi) > std::fabs(A[(size_t)piv * 2 * Q + c].hi)) piv = r;
    if (A[(size_t)piv * 2 * Q + c].hi == 0.0) return false;
    if (piv != c)
      for (int j = 0; j < 2 * Q; ++j) std::swap(A[(size_t)c * 2 * Q + j], A[(size_t)piv * 2 * Q + j]);
    const dd d = A[(size_t)c * 2 * Q + c];
    for (int j = 0; j < 2 * Q; ++j) A[(size_t)c * 2 * Q + j] = A[(size_t)c * 2 * Q + j] / d;
    for (int r = 0; r < Q; ++r) {
      if (r == c) continue;
      const dd f = A[(size_t)r * 2 * Q + c];
      if (f.hi == 0.0) continue;
      for (int j = 0; j < 2 * Q; ++j) A[(size_t)r * 2 * Q + j] = A[(size_t)r * 2 * Q + j] - f * A[(size_t)c * 2 * Q + j];
    }
  }
  // A = [I | Phi^-1] with Phi[k][i]; f = Phi^-1 M, so H[i][k] = (Phi^-1)[i][k]
  H->assign((size_t)Q * Q, 0.0);
  for (int i = 0; i < Q; ++i)
    for (int k = 0; k < Q; ++k) (*H)[(size_t)i * Q + k] = A[(size_t)i * 2 * Q + Q + k].to_double();
  return true;
}

}  // namespace rlbm1

using namespace rlbm1;

struct rlbm1_handle {
  Sc sc{};
  std::unique_ptr<Tab<float>> tf;
  std::unique_ptr<Tab<double>> td;
  std::vector<double> p0, w, fref;
  std::vector<int> sgn;
  size_t elem = 8;
  void* buf[2] = {nullptr, nullptr};
  int cur = 0;
  bool have_prev = false;
  double* fields = nullptr;          // [8][nx]
  double* staging = nullptr;         // [3][nx] init input from host
  unsigned long long* status = nullptr;
  cudaStream_t stream = nullptr;
  std::string err = "no error";
  ~rlbm1_handle() {
    for (void* b : buf) cudaFree(b);
    cudaFree(fields);
    cudaFree(staging);
    cudaFree(status);
  }
};

namespace {

thread_local std::string g_err1 = "no error";

int fail1(rlbm1_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  else g_err1 = msg;
  return code;
}

int cuda_fail1(rlbm1_handle* h, cudaError_t e, const char* what) {
  return fail1(h, RLBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

template <typename S>
void fill(const rlbm1_handle* h, const std::vector<double>& H, Tab<S>* t) {
  std::memset(t, 0, sizeof(Tab<S>));
  const int Q = h->sc.Q;
  for (int i = 0; i < Q; ++i) {
    t->p0[i] = h->p0[i];
    const double p2 = h->p0[i] * h->p0[i];
    t->w1h[i] = (float)h->p0[i];
    t->w1l[i] = (float)(h->p0[i] - (double)t->w1h[i]);
    t->w2h[i] = (float)p2;
    t->w2l[i] = (float)(p2 - (double)t->w2h[i]);
    t->s[i] = h->sgn[i];
    for (int k = 0; k < Q; ++k) {
      t->H[i][k] = H[(size_t)i * Q + k];
      t->Hs[i][k] = (S)H[(size_t)i * Q + k];
    }
  }
}

dim3 grid1(int nx) { return dim3((nx + kThreads - 1) / kThreads); }

}  // namespace

extern "C" {

const char* rlbm1_last_error(const rlbm1_handle* h) { return h ? h->err.c_str() : g_err1.c_str(); }

int rlbm1_plan(int order, int* Q, int* nvec, double* p, double* w, double* H) {
  if (!Q) return fail1(nullptr, RLBM_ERR_INVALID_ARG, "null argument");
  std::vector<double> p0, wv, Hm;
  std::vector<int> sg;
  if (!build_tables(order, &p0, &sg, &wv, &Hm)) return fail1(nullptr, RLBM_ERR_INVALID_ARG, "order must be 2 ... 5");
  const int q = 2 * order;
  *Q = q;
  for (int i = 0; i < q; ++i) {
    if (nvec) nvec[i] = sg[i];
    if (p) { p[2 * i] = p0[i]; p[2 * i + 1] = sg[i] * p0[i]; }
    if (w) w[i] = wv[i];
  }
  if (H) std::memcpy(H, Hm.data(), sizeof(double) * q * q);
  return RLBM_OK;
}

int rlbm1_create(int nx, int order, double tau, int boundary, const double* wall_T, int precision, void* stream,
                 rlbm1_handle** out) {
  if (!out) return fail1(nullptr, RLBM_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (nx < 1 || nx > (1 << 28)) return fail1(nullptr, RLBM_ERR_INVALID_ARG, "nx out of range");
  if (!(tau > 0.5)) return fail1(nullptr, RLBM_ERR_INVALID_ARG, "tau must exceed 1/2");
  if (boundary != RLBM_BC_PERIODIC && boundary != RLBM_BC_FREEFLOW_X && boundary != RLBM_BC_EQWALL_X)
    return fail1(nullptr, RLBM_ERR_INVALID_ARG, "boundary");
  if (precision != RLBM_FP64 && precision != RLBM_FP32_STORE) return fail1(nullptr, RLBM_ERR_INVALID_ARG, "precision");
  std::unique_ptr<rlbm1_handle> h(new rlbm1_handle());
  std::vector<double> H;
  if (!build_tables(order, &h->p0, &h->sgn, &h->w, &H)) return fail1(nullptr, RLBM_ERR_INVALID_ARG, "order must be 2 ... 5");
  // the FP32-storage step takes each pair's second row as the first with the
  // odd members' signs flipped, and the directions as +1, -1 alternating
  for (int j = 0; j < order; ++j)
    for (int k = 0; k < 2 * order; ++k)
      if (h->sgn[2 * j] != 1 || h->sgn[2 * j + 1] != -1 ||
          H[(size_t)(2 * j + 1) * 2 * order + k] != ((k & 1) ? -1.0 : 1.0) * H[(size_t)2 * j * 2 * order + k])
        return fail1(nullptr, RLBM_ERR_QUADRATURE, "1-d equilibrium matrix without the direction symmetry");
  Sc& s = h->sc;
  s.N = order;
  s.Q = 2 * order;
  s.nx = nx;
  s.P = nx + 2;
  s.boundary = boundary;
  s.tau = tau;
  s.wall_T[0] = wall_T ? wall_T[0] : 0.0;
  s.wall_T[1] = wall_T ? wall_T[1] : 0.0;
  s.n_ref = precision == RLBM_FP32_STORE ? 1.0 : 0.0;
  s.T_ref = 1.0;
  s.N0_ref = s.n_ref;
  s.T00_ref = s.n_ref * s.T_ref;
  s.f_n_ref = (float)s.n_ref;
  s.f_T_ref = (float)s.T_ref;
  s.f_Er = (float)s.T00_ref;
  s.f_inv_tau = (float)(1.0 / tau);
  for (int k = 0; k < 2; ++k) {
    s.f_wall_T[k] = (float)s.wall_T[k];
    s.f_wall_dT[k] = (float)(s.wall_T[k] - s.T_ref);
  }
  h->elem = precision == RLBM_FP32_STORE ? 4 : 8;
  h->stream = (cudaStream_t)stream;
  // reference populations f_ref = H M(n_ref, rest, T_ref) (the shift of FP32 storage)
  h->fref.assign(s.Q, 0.0);
  if (s.n_ref > 0.0) {
    Sc z = s;
    z.n_ref = 0.0;
    double M[kMaxQ];
    moments_dM(z, s.n_ref, 1.0, 0.0, s.T_ref, M);
    for (int i = 0; i < s.Q; ++i)
      for (int k = 0; k < s.Q; ++k) h->fref[i] += H[(size_t)i * s.Q + k] * M[k];
  }
  if (h->elem == 4) { h->tf.reset(new Tab<float>()); fill(h.get(), H, h->tf.get()); }
  else { h->td.reset(new Tab<double>()); fill(h.get(), H, h->td.get()); }
  const size_t bytes = (size_t)s.Q * s.P * h->elem;
  for (int b = 0; b < 2; ++b)
    if (cudaMalloc(&h->buf[b], bytes) != cudaSuccess) { cudaGetLastError(); return fail1(nullptr, RLBM_ERR_OOM, "population buffers"); }
  if (cudaMalloc(&h->fields, sizeof(double) * 8 * nx) != cudaSuccess ||
      cudaMalloc(&h->staging, sizeof(double) * 3 * nx) != cudaSuccess ||
      cudaMalloc(&h->status, sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    return fail1(nullptr, RLBM_ERR_OOM, "field buffers");
  }
  cudaError_t e = cudaMemsetAsync(h->status, 0, sizeof(unsigned long long), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->buf[0], 0, bytes, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->buf[1], 0, bytes, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail1(nullptr, e, "rlbm1_create");
  *out = h.release();
  return RLBM_OK;
}

void rlbm1_destroy(rlbm1_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  delete h;
}

int rlbm1_stencil(const rlbm1_handle* h, int* Q, int* nvec, double* p, double* w) {
  if (!h || !Q) return RLBM_ERR_INVALID_ARG;
  *Q = h->sc.Q;
  for (int i = 0; i < h->sc.Q; ++i) {
    if (nvec) nvec[i] = h->sgn[i];
    if (p) { p[2 * i] = h->p0[i]; p[2 * i + 1] = h->sgn[i] * h->p0[i]; }
    if (w) w[i] = h->w[i];
  }
  return RLBM_OK;
}

int rlbm1_init(rlbm1_handle* h, const double* n, const double* ux, const double* T, int on_device) {
  if (!h || !n || !ux || !T) return RLBM_ERR_INVALID_ARG;
  const int nx = h->sc.nx;
  const double* dn = n;
  const double* du = ux;
  const double* dT = T;
  cudaError_t e = cudaSuccess;
  if (!on_device) {
    e = cudaMemcpyAsync(h->staging, n, sizeof(double) * nx, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->staging + nx, ux, sizeof(double) * nx, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->staging + 2 * nx, T, sizeof(double) * nx, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail1(h, e, "rlbm1_init copy");
    dn = h->staging;
    du = h->staging + nx;
    dT = h->staging + 2 * nx;
  }
  if (h->elem == 4)
    k_init1<float><<<grid1(nx), kThreads, 0, h->stream>>>(*h->tf, h->sc, dn, du, dT, (float*)h->buf[h->cur], h->status);
  else
    k_init1<double><<<grid1(nx), kThreads, 0, h->stream>>>(*h->td, h->sc, dn, du, dT, (double*)h->buf[h->cur], h->status);
  e = cudaGetLastError();
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail1(h, e, "rlbm1_init");
  h->have_prev = false;
  return RLBM_OK;
}

int rlbm1_step(rlbm1_handle* h, int nsteps) {
  if (!h || nsteps < 0) return RLBM_ERR_INVALID_ARG;
  for (int it = 0; it < nsteps; ++it) {
    if (h->elem == 4) {
      const float* in = (const float*)h->buf[h->cur];
      float* o = (float*)h->buf[h->cur ^ 1];
      const dim3 gr((h->sc.nx + kThreads * kStep1CPT - 1) / (kThreads * kStep1CPT));
      switch (h->sc.N) {
        case 2: k_step1f<2, kStep1CPT><<<gr, kThreads, 0, h->stream>>>(*h->tf, h->sc, in, o, h->status); break;
        case 3: k_step1f<3, kStep1CPT><<<gr, kThreads, 0, h->stream>>>(*h->tf, h->sc, in, o, h->status); break;
        case 4: k_step1f<4, kStep1CPT><<<gr, kThreads, 0, h->stream>>>(*h->tf, h->sc, in, o, h->status); break;
        default: k_step1f<5, kStep1CPT><<<gr, kThreads, 0, h->stream>>>(*h->tf, h->sc, in, o, h->status); break;
      }
    } else
      k_step1<double><<<grid1(h->sc.nx), kThreads, 0, h->stream>>>(*h->td, h->sc, (const double*)h->buf[h->cur],
                                                                    (double*)h->buf[h->cur ^ 1], h->status);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail1(h, e, "rlbm1_step");
    h->cur ^= 1;
    h->have_prev = true;
  }
  return RLBM_OK;
}

int rlbm1_moments(rlbm1_handle* h, double* out, int on_device) {
  if (!h || !out) return RLBM_ERR_INVALID_ARG;
  const int nx = h->sc.nx;
  const void* src = h->have_prev ? h->buf[h->cur ^ 1] : h->buf[h->cur];
  const int pull = h->have_prev ? 1 : 0;
  double* dst = on_device ? out : h->fields;
  if (h->elem == 4)
    k_fields1<float><<<grid1(nx), kThreads, 0, h->stream>>>(*h->tf, h->sc, (const float*)src, pull, dst);
  else
    k_fields1<double><<<grid1(nx), kThreads, 0, h->stream>>>(*h->td, h->sc, (const double*)src, pull, dst);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && !on_device) {
    e = cudaMemcpyAsync(out, h->fields, sizeof(double) * 8 * nx, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  }
  if (e != cudaSuccess) return cuda_fail1(h, e, "rlbm1_moments");
  return RLBM_OK;
}

int rlbm1_get_populations(rlbm1_handle* h, double* f) {
  if (!h || !f) return RLBM_ERR_INVALID_ARG;
  const Sc& s = h->sc;
  std::vector<unsigned char> raw((size_t)s.Q * s.P * h->elem);
  cudaError_t e = cudaMemcpyAsync(raw.data(), h->buf[h->cur], raw.size(), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail1(h, e, "rlbm1_get_populations");
  for (int i = 0; i < s.Q; ++i)
    for (int x = 0; x < s.nx; ++x) {
      const size_t at = (size_t)i * s.P + x + 1;
      const double v = h->elem == 4 ? (double)((const float*)raw.data())[at] : ((const double*)raw.data())[at];
      f[(size_t)i * s.nx + x] = v + h->fref[i];
    }
  return RLBM_OK;
}

int rlbm1_sync_status(rlbm1_handle* h, long long* count) {
  if (!h) return RLBM_ERR_INVALID_ARG;
  unsigned long long c = 0;
  cudaError_t e = cudaMemcpyAsync(&c, h->status, sizeof(c), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->status, 0, sizeof(c), h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail1(h, e, "rlbm1_sync_status");
  if (count) *count = (long long)c;
  return c ? fail1(h, RLBM_ERR_NONPHYSICAL, "non-physical cell updates") : RLBM_OK;
}

}  // extern "C"
