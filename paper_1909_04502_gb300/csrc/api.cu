// C ABI of the RLBM library (declared in include/rlbm.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "../../include/rlbm.h"
#include "dispatch.h"
#include "handle.h"
#include "step_impl.cuh"
#include "setup.h"

using namespace rlbm;

namespace {

thread_local std::string g_create_error = "no error";

int fail(rlbm_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_error = msg;
  return code;
}

int cuda_fail(rlbm_handle* h, cudaError_t e, const char* where) {
  return fail(h, RLBM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define RLBM_CUDA(h, call)                                   \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, #call); \
  } while (0)

// Off-lattice pull taps for velocity (vx, vy) and lambda: the departure point
// is x - lambda v; o = floor of it, phi = its fractional part.  A displacement
// within 1e-12 of a whole number of cells is that number.
void bilinear_base(double lambda, double vx, double vy, int o[2], double phi[2]) {
  double src[2] = {-lambda * vx, -lambda * vy};
  for (int d = 0; d < 2; ++d) {
    double r = std::nearbyint(src[d]);
    if (std::fabs(src[d] - r) < 1e-12) src[d] = r;
    double fl = std::floor(src[d]);
    o[d] = (int)fl;
    if (phi) phi[d] = src[d] - fl;
  }
}

// Device kernels converting between stored (shifted, storage precision,
// padded) populations and FP64 unshifted populations [Q][ny][nx].  The import
// also fills the halo images.
template <typename S>
__global__ void k_export(const S* __restrict__ src, double* __restrict__ dst, const Scalars s,
                         const double* __restrict__ fref) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)s.Q * s.ncell) return;
  int i = (int)(idx / s.ncell), c = (int)(idx - (long long)i * s.ncell);
  int y = c / s.nx, x = c - y * s.nx;
  dst[idx] = (double)src[i * s.plane + sidx(s, x, y)] + fref[i];
}

template <typename S>
__global__ void k_import(const double* __restrict__ src, S* __restrict__ dst, const Scalars s,
                         const double* __restrict__ fref) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)s.Q * s.ncell) return;
  int i = (int)(idx / s.ncell), c = (int)(idx - (long long)i * s.ncell);
  int y = c / s.nx, x = c - y * s.nx;
  const S v = (S)(src[idx] - fref[i]);
  dst[i * s.plane + sidx(s, x, y)] = v;
  for_each_halo_image(s, x, y, [&](long long hi) { dst[i * s.plane + hi] = v; });
}

template <typename S>
__global__ void k_tau_import(const double* __restrict__ src, S* __restrict__ dst, int ncell) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < ncell) dst[idx] = (S)src[idx];
}

// Derived scalars: FP32 copies, flags, the int plane stride.
void finish_scalars(Scalars* s) {
  s->PE_ref = s->Tii_ref + s->T00_ref;
  s->n_ref2 = s->n_ref * s->n_ref;
  s->force = (s->m > 0.0 && (s->gx != 0.0 || s->gy != 0.0)) ? 1 : 0;
  s->f_gx = (float)s->gx;
  s->f_gy = (float)s->gy;
  s->f_wall_T[0] = (float)s->wall_T[0];
  s->f_wall_T[1] = (float)s->wall_T[1];
  s->massless = (s->m == 0.0) ? 1 : 0;
  s->iplane = (int)s->plane;
  s->f_tau = (float)s->tau;
  s->f_tau_coef = (float)s->tau_coef;
  s->f_m = (float)s->m;
  s->f_n_ref = (float)s->n_ref;
  s->f_T_ref = (float)s->T_ref;
  s->f_T00_ref = (float)s->T00_ref;
  s->f_Tii_ref = (float)s->Tii_ref;
  s->f_PE_hi = (float)s->PE_ref;
  s->f_PE_lo = (float)(s->PE_ref - (double)s->f_PE_hi);
}

// Halo widths and padded layout of the population planes (kernels.cuh).
void compute_layout(const Quadrature& q, const rlbm_params& p, size_t elem, Scalars* s) {
  int hx = 0, hy = 0;
  for (int i = 0; i < q.Q; ++i) {
    if (p.stream_mode == RLBM_ONLATTICE) {
      hx = std::max(hx, std::abs(q.nx[i]));
      hy = std::max(hy, std::abs(q.ny[i]));
    } else {
      int o[2];
      bilinear_base(p.lambda, q.px[i] / q.p0[i], q.py[i] / q.p0[i], o, nullptr);
      hx = std::max(hx, std::max(-o[0], o[0] + 1));
      hy = std::max(hy, std::max(-o[1], o[1] + 1));
    }
  }
  const int align = (int)(32 / elem);                 // 32-byte row alignment
  s->hx = hx;
  s->hy = hy;
  s->px = (hx + align - 1) / align * align;
  s->pitch = (s->px + p.nx + hx + align - 1) / align * align;
  s->plane = ((long long)(p.ny + 2 * hy) * s->pitch + 31) / 32 * 32;
}

// Bilinear weights in the storage type whose exact sum is one: each weight
// becomes a multiple of 2^-b (b = 24 for float, 52 for double; every such
// value in [0, 1] is exact in R) and the largest takes the remainder.
// Rounding each weight on its own leaves the sum off by up to a few units in
// the last place, which multiplies the streamed populations by that factor
// every step and drifts the global sums of N^0 and T^{0a}.
// True when the kernels' orbit-symmetric evaluation applies: the stencil has
// one of the compiled orbit compositions (massless Q = 28, 44; the built-in
// massive Q = 33, 29, 25 at order 2 and 65, 57, 49, 53 at order 3; the
// 45-vector stencil of the paper's performance table at order 3) in orbit
// order (setup.cpp), every member's momentum
// and weight are the signed / swapped image of its orbit's first member, and
// every row of H is exactly the first row with the matching column signs and
// (for a swapped member) swapped columns; axis, diagonal and rest rows have
// the zero or symmetric entries the kernels skip.
bool orbit_symmetric(const rlbm_handle* h) {
  const Quadrature& q = h->q;
  int n8, n4, nd, n1;
  if (q.Q == 28 && h->K == 9 && q.m == 0.0) { n8 = 3; n4 = 1; nd = 0; n1 = 0; }
  else if (q.Q == 44 && h->K == 16 && q.m == 0.0) { n8 = 4; n4 = 3; nd = 0; n1 = 0; }
  else if (q.Q == 33 && h->K == 9) { n8 = 3; n4 = 1; nd = 1; n1 = 1; }
  else if (q.Q == 29 && h->K == 9) { n8 = 2; n4 = 1; nd = 2; n1 = 1; }
  else if (q.Q == 25 && h->K == 9) { n8 = 1; n4 = 2; nd = 2; n1 = 1; }
  else if (q.Q == 65 && h->K == 16 && q.m > 0.0) { n8 = 7; n4 = 0; nd = 2; n1 = 1; }
  else if (q.Q == 57 && h->K == 16 && q.m > 0.0) { n8 = 5; n4 = 1; nd = 3; n1 = 1; }
  else if (q.Q == 49 && h->K == 16 && q.m > 0.0) { n8 = 3; n4 = 4; nd = 2; n1 = 1; }
  else if (q.Q == 53 && h->K == 16 && q.m > 0.0) { n8 = 4; n4 = 3; nd = 2; n1 = 1; }
  else if (q.Q == 45 && h->K == 16 && q.m > 0.0) { n8 = 2; n4 = 4; nd = 3; n1 = 1; }
  else return false;
  const int K = h->K;
  auto row = [&](int i, int k) { return h->H[(size_t)i * K + k]; };
  auto check = [&](int i0, int i, int sx, int sy, bool swap) {
    const double bx = swap ? q.py[i0] : q.px[i0], by = swap ? q.px[i0] : q.py[i0];
    if (q.p0[i] != q.p0[i0] || q.px[i] != sx * bx || q.py[i] != sy * by || q.w[i] != q.w[i0]) return false;
    for (int k = 0; k < K; ++k) {
      const double sgn = (mono_ax(k) && sx < 0 ? -1.0 : 1.0) * (mono_ay(k) && sy < 0 ? -1.0 : 1.0);
      if (row(i, k) != sgn * row(i0, swap ? mono_swap(k) : k)) return false;
    }
    return true;
  };
  const int sg[4][2] = {{1, 1}, {-1, 1}, {1, -1}, {-1, -1}};
  int i0 = 0;
  for (int o = 0; o < n8; ++o, i0 += 8) {
    if (q.px[i0] == 0.0 || q.py[i0] == 0.0 || std::fabs(q.px[i0]) == std::fabs(q.py[i0])) return false;
    for (int m = 0; m < 8; ++m)
      if (!check(i0, i0 + m, sg[m & 3][0], sg[m & 3][1], m >= 4)) return false;
  }
  for (int o = 0; o < n4; ++o, i0 += 4) {
    if (q.py[i0] != 0.0 || q.px[i0] == 0.0) return false;
    for (int k = 0; k < K; ++k)
      if (mono_ay(k) && row(i0, k) != 0.0) return false;
    const int sgn4[4][3] = {{1, 1, 0}, {-1, 1, 0}, {1, 1, 1}, {1, -1, 1}};   // (sx, sy, swap)
    for (int m = 0; m < 4; ++m)
      if (!check(i0, i0 + m, sgn4[m][0], sgn4[m][1], sgn4[m][2] != 0)) return false;
  }
  for (int o = 0; o < nd; ++o, i0 += 4) {
    if (q.px[i0] != q.py[i0] || q.px[i0] == 0.0) return false;
    for (int m = 0; m < 4; ++m)
      if (!check(i0, i0 + m, sg[m][0], sg[m][1], false)) return false;
  }
  for (int o = 0; o < n1; ++o, ++i0) {
    if (q.px[i0] != 0.0 || q.py[i0] != 0.0) return false;
    for (int k = 0; k < K; ++k)
      if ((mono_ax(k) || mono_ay(k)) && row(i0, k) != 0.0) return false;
  }
  return i0 == q.Q;
}

// Step kernel a handle uses: the caller's choice, else the direct-load
// kernel (on GB300 the TMA-staged kernels are slower at every grid size: the
// shared-memory stages cut residency from 32 to 16-24 warps per SM, and the
// collision's FP64 chains need those warps more than the pull needs staging).
int effective_step_kernel(const rlbm_handle* h) {
  if (h->step_kernel != RLBM_KERNEL_AUTO) return h->step_kernel;
  return RLBM_KERNEL_DIRECT;
}

template <typename R>
void quantize_unit_sum(const double (&w)[4], R (&out)[4]) {
  const int bits = sizeof(R) == 4 ? 24 : 52;
  const long long one = 1LL << bits;
  long long k[4];
  int big = 0;
  for (int j = 0; j < 4; ++j) {
    k[j] = std::llround(std::ldexp(w[j], bits));
    if (w[j] > w[big]) big = j;
  }
  long long rest = one;
  for (int j = 0; j < 4; ++j)
    if (j != big) rest -= k[j];
  k[big] = rest;
  for (int j = 0; j < 4; ++j) out[j] = (R)std::ldexp((double)k[j], -bits);
}

// Reference populations of the shifted FP32 storage:
// f_ref,i = sum_k H_ik M_k(n_ref, e0, T_ref) (zero when n_ref = 0).
void reference_populations(rlbm_handle* h, int order, double m, double nr, double Tr) {
  std::vector<double> Mref(h->K);
  const double e0[3] = {1.0, 0.0, 0.0};
  mj_moments(order, m, nr, e0, Tr, Mref.data());
  h->fref.assign(h->q.Q, 0.0);
  for (int i = 0; i < h->q.Q; ++i)
    for (int k = 0; k < h->K; ++k) h->fref[i] += h->H[(size_t)i * h->K + k] * Mref[k];
}

template <typename R>
void fill_tables(const rlbm_handle* h, const Scalars& s, Tables<R>* t) {
  std::memset(t, 0, sizeof(Tables<R>));
  const Quadrature& q = h->q;
  for (int i = 0; i < q.Q; ++i) {
    const double p0 = q.p0[i], px = q.px[i], py = q.py[i];
    const double c[9] = {p0, px, py, p0 * p0, p0 * px, p0 * py, px * px, px * py, py * py};
    for (int j = 0; j < 9; ++j) t->c[i][j] = (R)c[j];
    t->vx[i] = (R)(px / p0);
    t->vy[i] = (R)(py / p0);
    for (int k = 0; k < h->K; ++k) t->H[i][k] = (R)h->H[(size_t)i * h->K + k];
    if (h->p.stream_mode == RLBM_ONLATTICE) {
      t->off[i] = -q.ny[i] * s.pitch - q.nx[i];
      t->dx[i] = (short)(-q.nx[i]);
      t->dy[i] = (short)(-q.ny[i]);
      t->roff[i] = q.ny[i] * s.pitch + q.nx[i];
      t->bw[i][0] = (R)1.0;
    } else {
      int o[2];
      double phi[2];
      bilinear_base(h->p.lambda, px / p0, py / p0, o, phi);
      t->off[i] = o[1] * s.pitch + o[0];
      t->dx[i] = (short)o[0];
      t->dy[i] = (short)o[1];
      t->roff[i] = (-o[1] - 1) * s.pitch + (-o[0] - 1);
      const double w[4] = {(1.0 - phi[0]) * (1.0 - phi[1]), phi[0] * (1.0 - phi[1]), (1.0 - phi[0]) * phi[1],
                           phi[0] * phi[1]};
      quantize_unit_sum<R>(w, t->bw[i]);
    }
    t->pl[i] = i * (int)s.plane;
    t->offp[i] = t->pl[i] + t->off[i];
    t->offr[i] = t->offp[i] + s.pitch;
    t->roff[i] += t->pl[i];
    t->fref[i] = (R)(i < (int)h->fref.size() ? h->fref[i] : 0.0);
  }
}

// FP32 storage at order 3 with m~ >= kXeqMinMass on an orbit-symmetric
// table runs the extended-precision equilibrium of step_xeq.cu: there the
// contraction H dM cancels so strongly that FP32 moments lose the 1e-5 bar
// (at m~ = 10-20 by 10-55 %; at m~ = 7 they keep 3-4e-6).
constexpr double kXeqMinMass = 6.0;

bool use_xeq(const rlbm_handle* h, const Scalars& s) {
  return h->p.precision == RLBM_FP32_STORE && h->p.order == 3 && h->p.m >= kXeqMinMass && s.sym &&
         xeq_supported_q(h->q.Q);
}

void split_pair(double v, float (&out)[2]) {
  out[0] = (float)v;
  out[1] = (float)(v - (double)out[0]);
}

// The low parts of the FP32 equilibrium matrix (fill_tables rounds H to
// FP32) and the reference scalars as pairs.
void fill_xeq_tables(const rlbm_handle* h, const Scalars& s, XeqTables* t) {
  std::memset(t, 0, sizeof(XeqTables));
  for (int i = 0; i < h->q.Q; ++i)
    for (int k = 0; k < h->K; ++k) {
      const double v = h->H[(size_t)i * h->K + k];
      t->Hl[i][k] = (float)(v - (double)(float)v);
    }
  split_pair(s.m, t->m);
  split_pair(s.n_ref, t->n_ref);
  split_pair(s.T_ref, t->T_ref);
}

int build_quadrature(const rlbm_params* p, Quadrature* q, std::string* err) {
  if (p->quadrature == RLBM_QUAD_MASSLESS) {
    if (p->m != 0.0) { *err = "RLBM_QUAD_MASSLESS needs m = 0"; return RLBM_ERR_INVALID_ARG; }
    return massless_quadrature(p->order, q, err) ? RLBM_OK : RLBM_ERR_INVALID_ARG;
  }
  if (p->quadrature == RLBM_QUAD_MASSIVE) {
    if (!(p->m > 0.0)) { *err = "RLBM_QUAD_MASSIVE needs m > 0"; return RLBM_ERR_INVALID_ARG; }
    if (p->groups == nullptr || p->n_groups <= 0) {
      if (p->v0 != 0.0) { *err = "v0 given without groups"; return RLBM_ERR_INVALID_ARG; }
      return builtin_massive(p->m, p->order, q, err) ? RLBM_OK : RLBM_ERR_QUADRATURE;
    }
    std::vector<int> g(p->groups, p->groups + 2 * p->n_groups);
    double v0 = p->v0;
    if (v0 == 0.0 && !search_v0(g, p->m, p->order, &v0, nullptr, nullptr)) {
      *err = "no v0 gives non-negative weights on this stencil";
      return RLBM_ERR_QUADRATURE;
    }
    double res;
    if (!massive_quadrature(g, p->m, v0, p->order, q, &res, nullptr, true) || res > 1e-9) {
      *err = "orthonormality conditions not satisfied on this stencil";
      return RLBM_ERR_QUADRATURE;
    }
    return RLBM_OK;
  }
  if (p->quadrature == RLBM_QUAD_CUSTOM) {
    if (!p->custom_table || p->custom_Q <= 0) { *err = "custom table missing"; return RLBM_ERR_INVALID_ARG; }
    *q = Quadrature();
    q->m = p->m;
    q->order = p->order;
    for (int i = 0; i < p->custom_Q; ++i) {
      const double* r = p->custom_table + 6 * i;
      q->nx.push_back((int)std::lround(r[0]));
      q->ny.push_back((int)std::lround(r[1]));
      q->p0.push_back(r[2]);
      q->px.push_back(r[3]);
      q->py.push_back(r[4]);
      q->w.push_back(r[5]);
    }
    q->Q = p->custom_Q;
    return RLBM_OK;
  }
  *err = "unknown quadrature";
  return RLBM_ERR_INVALID_ARG;
}

}  // namespace

extern "C" {

void rlbm_default_params(rlbm_params* p) {
  std::memset(p, 0, sizeof(*p));
  p->d = 2;
  p->m = 0.0;
  p->order = 2;
  p->quadrature = RLBM_QUAD_MASSLESS;
  p->tau_mode = RLBM_TAU_CONST;
  p->tau = 1.0;
  p->boundary = RLBM_BC_PERIODIC;
  p->nx = p->ny = 0;
  p->precision = RLBM_FP32_STORE;
  p->stream_mode = RLBM_ONLATTICE;
  p->lambda = 0.0;
  p->n_ref = 1.0;
  p->T_ref = 1.0;
}

const char* rlbm_strerror(int code) {
  switch (code) {
    case RLBM_OK: return "ok";
    case RLBM_ERR_INVALID_ARG: return "invalid argument";
    case RLBM_ERR_UNSUPPORTED: return "unsupported";
    case RLBM_ERR_CUDA: return "CUDA error";
    case RLBM_ERR_NONPHYSICAL: return "non-physical cell state";
    case RLBM_ERR_TIMEOUT: return "device wait timed out";
    case RLBM_ERR_OOM: return "out of device memory";
    case RLBM_ERR_QUADRATURE: return "no quadrature";
  }
  return "unknown error";
}

const char* rlbm_last_error(const rlbm_handle* h) { return h ? h->err.c_str() : g_create_error.c_str(); }

// Dimension of the stencils and of the gas they carry: d = 1 problems run on
// a d = 2 stencil over an nx x 1 grid (the paper's own practice for its
// one-dimensional tests), so the EOS and eta/s -> tau use d = 2.
constexpr int kStencilDim = 2;

// Checks shared by rlbm_create and the allocation-free step.
static int validate_params(const rlbm_params* p, std::string* err) {
  auto bad = [err](int code, const char* msg) { *err = msg; return code; };
  if (p->d == 3) return bad(RLBM_ERR_UNSUPPORTED, "d = 3 runs through rlbm3_create");
  if (p->d != 1 && p->d != 2) return bad(RLBM_ERR_INVALID_ARG, "d must be 1 or 2");
  if (p->order != 2 && p->order != 3) return bad(RLBM_ERR_INVALID_ARG, "order must be 2 or 3");
  if (p->nx <= 0 || p->ny <= 0 || (long long)p->nx * p->ny > (1LL << 30))
    return bad(RLBM_ERR_INVALID_ARG, "grid size out of range");
  if (p->d == 1 && p->ny != 1) return bad(RLBM_ERR_INVALID_ARG, "d = 1 needs ny = 1");
  if (p->precision != RLBM_FP64 && p->precision != RLBM_FP32_STORE) return bad(RLBM_ERR_INVALID_ARG, "precision");
  if (p->boundary != RLBM_BC_PERIODIC && p->boundary != RLBM_BC_FREEFLOW_X && p->boundary != RLBM_BC_EQWALL_X)
    return bad(RLBM_ERR_INVALID_ARG, "boundary");
  if (p->stream_mode != RLBM_ONLATTICE && p->stream_mode != RLBM_BILINEAR)
    return bad(RLBM_ERR_INVALID_ARG, "stream_mode");
  if (p->stream_mode == RLBM_BILINEAR && !(p->lambda > 0.0))
    return bad(RLBM_ERR_INVALID_ARG, "bilinear streaming needs lambda > 0");
  if (p->tau_mode < 0 || p->tau_mode > 2) return bad(RLBM_ERR_INVALID_ARG, "tau_mode");
  if (p->tau_mode == RLBM_TAU_CONST && !(p->tau > 0.5)) return bad(RLBM_ERR_INVALID_ARG, "tau must exceed 1/2");
  if (p->tau_mode == RLBM_TAU_ETA_OVER_S && !(p->eta_over_s > 0.0 && p->kappa > 0.0))
    return bad(RLBM_ERR_INVALID_ARG, "eta_over_s and kappa must be positive");
  if (!(p->T_ref > 0.0) || !(p->n_ref >= 0.0)) return bad(RLBM_ERR_INVALID_ARG, "reference state");
  return RLBM_OK;
}

int rlbm_plan(const rlbm_params* p, int* Q, int* K, int* nvec, double* pmom, double* w, double* H,
              double* v0) {
  if (!p || !Q || !K) return fail(nullptr, RLBM_ERR_INVALID_ARG, "null argument");
  if (p->order != 2 && p->order != 3) return fail(nullptr, RLBM_ERR_INVALID_ARG, "order must be 2 or 3");
  Quadrature q;
  std::string err;
  int rc = build_quadrature(p, &q, &err);
  if (rc != RLBM_OK) return fail(nullptr, rc, err);
  if (q.Q > kMaxQ) return fail(nullptr, RLBM_ERR_UNSUPPORTED, "too many populations");
  std::vector<double> Hm;
  if (!equilibrium_matrix(q, &Hm, &err)) return fail(nullptr, RLBM_ERR_QUADRATURE, err);
  *Q = q.Q;
  *K = (int)moment_basis(p->order).size();
  for (int i = 0; i < q.Q; ++i) {
    if (nvec) { nvec[2 * i] = q.nx[i]; nvec[2 * i + 1] = q.ny[i]; }
    if (pmom) { pmom[3 * i] = q.p0[i]; pmom[3 * i + 1] = q.px[i]; pmom[3 * i + 2] = q.py[i]; }
    if (w) w[i] = q.w[i];
  }
  if (H) std::copy(Hm.begin(), Hm.end(), H);
  if (v0) *v0 = q.v0;
  return RLBM_OK;
}

int rlbm_create(const rlbm_params* p, rlbm_handle** out) {
  if (!p || !out) return fail(nullptr, RLBM_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  {
    std::string verr;
    const int vrc = validate_params(p, &verr);
    if (vrc != RLBM_OK) return fail(nullptr, vrc, verr);
  }

  std::unique_ptr<rlbm_handle> h(new rlbm_handle());
  h->p = *p;
  h->p.groups = nullptr;
  h->p.custom_table = nullptr;
  std::string err;
  int rc = build_quadrature(p, &h->q, &err);
  if (rc != RLBM_OK) return fail(nullptr, rc, err);
  if (h->q.Q > kMaxQ) return fail(nullptr, RLBM_ERR_UNSUPPORTED, "too many populations");
  h->K = (int)moment_basis(p->order).size();
  if (!equilibrium_matrix(h->q, &h->H, &err)) return fail(nullptr, RLBM_ERR_QUADRATURE, err);

  const double m = p->m;
  const double nr = (p->precision == RLBM_FP32_STORE) ? p->n_ref : 0.0;
  const double Tr = p->T_ref;
  Scalars& s = h->sc;
  std::memset(&s, 0, sizeof(s));
  s.Q = h->q.Q;
  s.K = h->K;
  s.order = p->order;
  s.nx = p->nx;
  s.ny = p->ny;
  s.ncell = p->nx * p->ny;
  h->elem = (p->precision == RLBM_FP32_STORE) ? 4 : 8;
  compute_layout(h->q, *p, h->elem, &s);
  s.boundary = p->boundary;
  s.tau_mode = p->tau_mode;
  s.tau = p->tau;
  s.tau_coef = p->eta_over_s * (kStencilDim + 2) * p->kappa;
  s.m = m;
  s.n_ref = nr;
  s.T_ref = Tr;
  s.N0_ref = nr;
  s.T00_ref = nr * (m * m + 2.0 * m * Tr + 2.0 * Tr * Tr) / (m + Tr);
  s.Tii_ref = nr * Tr;
  s.kappa_guess = (float)(Tr * (m + Tr) / (m * m + 2.0 * m * Tr + 2.0 * Tr * Tr));
  s.gx = p->gx;
  s.gy = p->gy;
  s.wall_T[0] = p->wall_T[0];
  s.wall_T[1] = p->wall_T[1];
  finish_scalars(&s);
  // sym: the orbit-symmetric kernels without force or walls (the batched,
  // adjoint and extended-precision kernels take only these); sym_fw: the
  // order-2 orbit-symmetric kernels with the force term or the walls
  {
    const bool orb = orbit_symmetric(h.get()), fw = s.force || s.boundary == RLBM_BC_EQWALL_X;
    s.sym = (orb && !fw) ? 1 : 0;
    s.sym_fw = (orb && fw && s.K == 9) ? 1 : 0;
  }
  if ((long long)h->q.Q * s.plane >= (1LL << 31))
    return fail(nullptr, RLBM_ERR_UNSUPPORTED, "grid too large: Q * plane must stay below 2^31 elements");
  reference_populations(h.get(), p->order, m, nr, Tr);

  h->stream = (cudaStream_t)p->stream;
  if (h->elem == 4) {
    h->tf.reset(new Tables<float>());
    fill_tables(h.get(), s, h->tf.get());
    if (use_xeq(h.get(), s)) {
      h->txq.reset(new XeqTables());
      fill_xeq_tables(h.get(), s, h->txq.get());
    }
  } else {
    h->td.reset(new Tables<double>());
    fill_tables(h.get(), s, h->td.get());
  }
  // device buffers
  const size_t pop_bytes = (size_t)h->q.Q * s.plane * h->elem;
  cudaError_t e;
  for (int b = 0; b < 2; ++b) {
    e = cudaMalloc(&h->buf[b], pop_bytes);
    if (e != cudaSuccess) { cudaGetLastError(); return fail(nullptr, RLBM_ERR_OOM, "population buffers"); }
  }
  e = cudaMalloc(&h->fields, (size_t)14 * s.ncell * sizeof(double));
  if (e != cudaSuccess) { cudaGetLastError(); return fail(nullptr, RLBM_ERR_OOM, "field buffer"); }
  e = cudaMalloc(&h->tau_field, (size_t)s.ncell * h->elem);
  if (e != cudaSuccess) { cudaGetLastError(); return fail(nullptr, RLBM_ERR_OOM, "tau buffer"); }
  e = cudaMalloc(&h->status, 2 * sizeof(unsigned long long));
  if (e != cudaSuccess) { cudaGetLastError(); return fail(nullptr, RLBM_ERR_OOM, "status word"); }
  e = cudaMalloc(&h->fref_dev, kMaxQ * sizeof(double));
  if (e != cudaSuccess) { cudaGetLastError(); return fail(nullptr, RLBM_ERR_OOM, "reference"); }
  cudaMemset(h->buf[0], 0, pop_bytes);
  cudaMemset(h->buf[1], 0, pop_bytes);
  cudaMemset(h->status, 0, 2 * sizeof(unsigned long long));
  cudaMemcpy(h->fref_dev, h->fref.data(), h->q.Q * sizeof(double), cudaMemcpyHostToDevice);
  // tensor maps for the TMA-staged step kernel (where it applies)
  if (tma_supported(h.get())) {
    std::unique_ptr<TmaMaps> maps(new TmaMaps());
    const int mode = p->stream_mode == RLBM_BILINEAR ? kBilinear : kOnLattice;
    bool ok = true;
    std::string why;
    for (int b = 0; b < 2 && ok; ++b)
      for (int v = 0; v < 2 && ok; ++v)
        ok = tma_encode(h.get(), h->buf[b], tma_box_rows(mode, v == 0 ? 8 : 4), &maps->m[b][v], &why);
    if (ok) h->tma = std::move(maps);
  }
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(nullptr, RLBM_ERR_CUDA, cudaGetErrorString(e));
  *out = h.release();
  return RLBM_OK;
}

void rlbm_destroy(rlbm_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  cudaFree(h->buf[0]);
  cudaFree(h->buf[1]);
  cudaFree(h->fields);
  cudaFree(h->tau_field);
  cudaFree(h->status);
  cudaFree(h->fref_dev);
  if (h->staging) cudaFree(h->staging);
  delete h;
}

int rlbm_set_stream(rlbm_handle* h, void* stream) {
  if (!h) return RLBM_ERR_INVALID_ARG;
  h->stream = (cudaStream_t)stream;
  return RLBM_OK;
}

long long rlbm_time(const rlbm_handle* h) { return h ? h->t : -1; }

int rlbm_stencil(const rlbm_handle* h, int* Q, int* nvec, double* p, double* w) {
  if (!h || !Q) return RLBM_ERR_INVALID_ARG;
  *Q = h->q.Q;
  for (int i = 0; i < h->q.Q; ++i) {
    if (nvec) { nvec[2 * i] = h->q.nx[i]; nvec[2 * i + 1] = h->q.ny[i]; }
    if (p) { p[3 * i] = h->q.p0[i]; p[3 * i + 1] = h->q.px[i]; p[3 * i + 2] = h->q.py[i]; }
    if (w) w[i] = h->q.w[i];
  }
  return RLBM_OK;
}

int rlbm_init(rlbm_handle* h, const double* n, const double* ux, const double* uy, const double* T,
              int on_device) {
  if (!h || !n || !ux || !uy || !T) return RLBM_ERR_INVALID_ARG;
  const Scalars& s = h->sc;
  const size_t bytes = (size_t)s.ncell * sizeof(double);
  const double* src[4] = {n, ux, uy, T};
  const double* dev[4];
  for (int k = 0; k < 4; ++k) {
    if (on_device) {
      dev[k] = src[k];
    } else {
      double* d = h->fields + (size_t)k * s.ncell;   // the field planes double as staging
      RLBM_CUDA(h, cudaMemcpyAsync(d, src[k], bytes, cudaMemcpyHostToDevice, h->stream));
      dev[k] = d;
    }
  }
  cudaError_t e;
  if (h->elem == 4) {
    InitArgs<float> a{s, dev[0], dev[1], dev[2], dev[3], (float*)h->buf[h->cur], h->status};
    e = h->txq ? launch_init_xeq(*h->tf, *h->txq, a, h->stream) : launch_init<float>(*h->tf, a, h->stream);
  } else {
    InitArgs<double> a{s, dev[0], dev[1], dev[2], dev[3], (double*)h->buf[h->cur], h->status};
    e = launch_init<double>(*h->td, a, h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "init kernel");
  if (!on_device) RLBM_CUDA(h, cudaStreamSynchronize(h->stream));
  h->t = 0;
  h->have_prev = false;
  return RLBM_OK;
}

int rlbm_set_tau_field(rlbm_handle* h, const double* tau, int on_device) {
  if (!h || !tau) return RLBM_ERR_INVALID_ARG;
  const Scalars& s = h->sc;
  const double* d = tau;
  if (!on_device) {
    double* st = h->fields;
    RLBM_CUDA(h, cudaMemcpyAsync(st, tau, (size_t)s.ncell * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    d = st;
  }
  const int nb = (s.ncell + 255) / 256;
  if (h->elem == 4) k_tau_import<float><<<nb, 256, 0, h->stream>>>(d, (float*)h->tau_field, s.ncell);
  else k_tau_import<double><<<nb, 256, 0, h->stream>>>(d, (double*)h->tau_field, s.ncell);
  RLBM_CUDA(h, cudaGetLastError());
  if (!on_device) RLBM_CUDA(h, cudaStreamSynchronize(h->stream));
  return RLBM_OK;
}

int rlbm_set_step_kernel(rlbm_handle* h, int kernel) {
  if (!h || kernel < RLBM_KERNEL_AUTO || kernel > RLBM_KERNEL_TMA_32X4) return RLBM_ERR_INVALID_ARG;
  if ((kernel == RLBM_KERNEL_TMA_32X8 || kernel == RLBM_KERNEL_TMA_32X4) && !h->tma)
    return fail(h, RLBM_ERR_UNSUPPORTED, "the TMA-staged kernel needs FP32 storage, the massless Q = 28 order-2 "
                                         "stencil and a padded row of at least 36 elements");
  h->step_kernel = kernel;
  return RLBM_OK;
}

int rlbm_step_kernel(const rlbm_handle* h) { return h ? effective_step_kernel(h) : RLBM_ERR_INVALID_ARG; }

int rlbm_step(rlbm_handle* h, int nsteps) {
  if (!h || nsteps < 0) return RLBM_ERR_INVALID_ARG;
  const int mode = h->p.stream_mode == RLBM_BILINEAR ? kBilinear : kOnLattice;
  for (int it = 0; it < nsteps; ++it) {
    cudaError_t e;
    if (h->elem == 4) {
      StepArgs<float> a{h->sc, (const float*)h->buf[h->cur], (float*)h->buf[h->cur ^ 1],
                        (const float*)h->tau_field, h->status};
      const int k = effective_step_kernel(h);
      if (h->txq)
        e = launch_step_xeq(*h->tf, *h->txq, a, mode, h->stream);
      else if (k == RLBM_KERNEL_TMA_32X8 || k == RLBM_KERNEL_TMA_32X4)
        e = launch_step_tma(*h->tf, a, mode, k == RLBM_KERNEL_TMA_32X8 ? 8 : 4,
                            h->tma->m[h->cur][k == RLBM_KERNEL_TMA_32X8 ? 0 : 1], h->stream);
      else
        e = launch_step<float>(*h->tf, a, mode, h->stream);
    } else {
      StepArgs<double> a{h->sc, (const double*)h->buf[h->cur], (double*)h->buf[h->cur ^ 1],
                         (const double*)h->tau_field, h->status};
      e = launch_step<double>(*h->td, a, mode, h->stream);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "step kernel");
    h->cur ^= 1;
    h->t += 1;
    h->have_prev = true;
  }
  return RLBM_OK;
}

int rlbm_moments(rlbm_handle* h, double* n, double* ux, double* uy, double* T, double* eps, double* Nab,
                 double* Tab, int on_device) {
  if (!h) return RLBM_ERR_INVALID_ARG;
  const Scalars& s = h->sc;
  const int mode = h->p.stream_mode == RLBM_BILINEAR ? kBilinear : kOnLattice;
  const int want = (Nab || Tab) ? 1 : 0;
  const void* fin = h->have_prev ? h->buf[h->cur ^ 1] : h->buf[h->cur];
  cudaError_t e;
  if (h->elem == 4) {
    MomentArgs<float> a{s, (const float*)fin, h->have_prev ? 1 : 0, h->fields, want, h->status};
    e = launch_fields<float>(*h->tf, a, mode, h->stream);
  } else {
    MomentArgs<double> a{s, (const double*)fin, h->have_prev ? 1 : 0, h->fields, want, h->status};
    e = launch_fields<double>(*h->td, a, mode, h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "fields kernel");
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const size_t bytes = (size_t)s.ncell * sizeof(double);
  double* outs[5] = {n, ux, uy, T, eps};
  for (int k = 0; k < 5; ++k)
    if (outs[k]) RLBM_CUDA(h, cudaMemcpyAsync(outs[k], h->fields + (size_t)k * s.ncell, bytes, kind, h->stream));
  for (int k = 0; k < 3; ++k)
    if (Nab) RLBM_CUDA(h, cudaMemcpyAsync(Nab + (size_t)k * s.ncell, h->fields + (size_t)(5 + k) * s.ncell, bytes, kind, h->stream));
  for (int k = 0; k < 6; ++k)
    if (Tab) RLBM_CUDA(h, cudaMemcpyAsync(Tab + (size_t)k * s.ncell, h->fields + (size_t)(8 + k) * s.ncell, bytes, kind, h->stream));
  if (!on_device) RLBM_CUDA(h, cudaStreamSynchronize(h->stream));
  return RLBM_OK;
}

static int ensure_staging(rlbm_handle* h) {
  if (h->staging) return RLBM_OK;
  cudaError_t e = cudaMalloc(&h->staging, (size_t)h->q.Q * h->sc.ncell * sizeof(double));
  if (e != cudaSuccess) { cudaGetLastError(); return fail(h, RLBM_ERR_OOM, "staging buffer"); }
  return RLBM_OK;
}

int rlbm_get_populations(rlbm_handle* h, double* f, int on_device) {
  if (!h || !f) return RLBM_ERR_INVALID_ARG;
  const Scalars& s = h->sc;
  double* dst = f;
  if (!on_device) {
    int rc = ensure_staging(h);
    if (rc) return rc;
    dst = h->staging;
  }
  const long long total = (long long)s.Q * s.ncell;
  const int nb = (int)((total + 255) / 256);
  if (h->elem == 4) k_export<float><<<nb, 256, 0, h->stream>>>((const float*)h->buf[h->cur], dst, s, h->fref_dev);
  else k_export<double><<<nb, 256, 0, h->stream>>>((const double*)h->buf[h->cur], dst, s, h->fref_dev);
  RLBM_CUDA(h, cudaGetLastError());
  if (!on_device) {
    RLBM_CUDA(h, cudaMemcpyAsync(f, dst, total * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    RLBM_CUDA(h, cudaStreamSynchronize(h->stream));
  }
  return RLBM_OK;
}

int rlbm_set_populations(rlbm_handle* h, const double* f, int on_device) {
  if (!h || !f) return RLBM_ERR_INVALID_ARG;
  const Scalars& s = h->sc;
  const long long total = (long long)s.Q * s.ncell;
  const double* src = f;
  if (!on_device) {
    int rc = ensure_staging(h);
    if (rc) return rc;
    RLBM_CUDA(h, cudaMemcpyAsync(h->staging, f, total * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    src = h->staging;
  }
  const int nb = (int)((total + 255) / 256);
  if (h->elem == 4) k_import<float><<<nb, 256, 0, h->stream>>>(src, (float*)h->buf[h->cur], s, h->fref_dev);
  else k_import<double><<<nb, 256, 0, h->stream>>>(src, (double*)h->buf[h->cur], s, h->fref_dev);
  RLBM_CUDA(h, cudaGetLastError());
  if (!on_device) RLBM_CUDA(h, cudaStreamSynchronize(h->stream));
  h->have_prev = false;
  return RLBM_OK;
}

int rlbm_sync_status(rlbm_handle* h, long long* count) {
  if (!h) return RLBM_ERR_INVALID_ARG;
  RLBM_CUDA(h, cudaStreamSynchronize(h->stream));
  unsigned long long st[2] = {0, 0};
  RLBM_CUDA(h, cudaMemcpy(st, h->status, sizeof(st), cudaMemcpyDeviceToHost));
  RLBM_CUDA(h, cudaMemset(h->status, 0, sizeof(st)));
  if (count) *count = (long long)st[0];
  if (st[1]) return fail(h, RLBM_ERR_TIMEOUT, "a device-side wait timed out");
  if (st[0]) return fail(h, RLBM_ERR_NONPHYSICAL, std::to_string(st[0]) + " non-physical cell updates");
  return RLBM_OK;
}

int rlbm_buffers(rlbm_handle* h, void** cur, void** prev, int* elem_size, long long* plane, int* layout) {
  if (!h) return RLBM_ERR_INVALID_ARG;
  if (cur) *cur = h->buf[h->cur];
  if (prev) *prev = h->buf[h->cur ^ 1];
  if (elem_size) *elem_size = (int)h->elem;
  if (plane) *plane = h->sc.plane;
  if (layout) {
    layout[0] = h->sc.pitch;
    layout[1] = h->sc.hx;
    layout[2] = h->sc.hy;
    layout[3] = h->sc.px;
  }
  return RLBM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Host-only helpers for the allocation-free entry point (noalloc.cu).
// ---------------------------------------------------------------------------

void rlbm_internal_set_error(const std::string& msg) { g_create_error = msg; }

int rlbm_internal_prepare(const rlbm_params* p, Scalars* sc, Tables<float>* tf, Tables<double>* td,
                          std::unique_ptr<XeqTables>* txq, std::string* err) {
  {
    const int vrc = validate_params(p, err);
    if (vrc != RLBM_OK) return vrc;
  }
  rlbm_handle h;                      // host-side description only: no device buffers
  h.p = *p;
  h.p.groups = nullptr;
  h.p.custom_table = nullptr;
  int rc = build_quadrature(p, &h.q, err);
  if (rc != RLBM_OK) return rc;
  if (h.q.Q > kMaxQ) { *err = "too many populations"; return RLBM_ERR_UNSUPPORTED; }
  h.K = (int)moment_basis(p->order).size();
  if (!equilibrium_matrix(h.q, &h.H, err)) return RLBM_ERR_QUADRATURE;
  const double m = p->m;
  const double nr = (p->precision == RLBM_FP32_STORE) ? p->n_ref : 0.0;
  const double Tr = p->T_ref;
  Scalars& s = *sc;
  std::memset(&s, 0, sizeof(s));
  s.Q = h.q.Q;
  s.K = h.K;
  s.order = p->order;
  s.nx = p->nx;
  s.ny = p->ny;
  s.ncell = p->nx * p->ny;
  compute_layout(h.q, *p, p->precision == RLBM_FP32_STORE ? 4 : 8, &s);
  s.boundary = p->boundary;
  s.tau_mode = p->tau_mode;
  s.tau = p->tau;
  s.tau_coef = p->eta_over_s * (kStencilDim + 2) * p->kappa;
  s.m = m;
  s.n_ref = nr;
  s.T_ref = Tr;
  s.N0_ref = nr;
  s.T00_ref = nr * (m * m + 2.0 * m * Tr + 2.0 * Tr * Tr) / (m + Tr);
  s.Tii_ref = nr * Tr;
  s.kappa_guess = (float)(Tr * (m + Tr) / (m * m + 2.0 * m * Tr + 2.0 * Tr * Tr));
  s.gx = p->gx;
  s.gy = p->gy;
  s.wall_T[0] = p->wall_T[0];
  s.wall_T[1] = p->wall_T[1];
  finish_scalars(&s);
  // as in rlbm_create
  {
    const bool orb = orbit_symmetric(&h), fw = s.force || s.boundary == RLBM_BC_EQWALL_X;
    s.sym = (orb && !fw) ? 1 : 0;
    s.sym_fw = (orb && fw && s.K == 9) ? 1 : 0;
  }
  if ((long long)h.q.Q * s.plane >= (1LL << 31)) {
    *err = "grid too large: Q * plane must stay below 2^31 elements";
    return RLBM_ERR_UNSUPPORTED;
  }
  reference_populations(&h, p->order, m, nr, Tr);
  if (p->precision == RLBM_FP32_STORE) {
    fill_tables(&h, s, tf);
    if (use_xeq(&h, s)) {
      txq->reset(new XeqTables());
      fill_xeq_tables(&h, s, txq->get());
    }
  } else {
    fill_tables(&h, s, td);
  }
  return RLBM_OK;
}
