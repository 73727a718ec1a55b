// C ABI of the (3+1)-d massless step (include/rlbm.h, rlbm3_*).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "../../include/rlbm.h"
#include "d3.h"

using namespace rlbm;

struct rlbm3_handle {
  Quadrature3 q;
  Scalars3 sc{};
  std::unique_ptr<Tables3> tb;
  size_t elem = 8;                // bytes per stored population (8: f, 4: g = f - f_ref)
  void* buf[2] = {nullptr, nullptr};
  int cur = 0;                    // buf[cur] holds f*(t)
  bool have_prev = false;         // buf[cur ^ 1] holds f*(t-1)
  double* fields = nullptr;       // [6][ncell]
  double* staging = nullptr;      // 5 input fields on the device (init from host)
  unsigned long long* status = nullptr;
  cudaStream_t stream = nullptr;
  std::vector<double> fref;       // reference populations (FP32 storage)
  bool sym = false;               // order 2 in sign-orbit form (the steps need it)
  // order 3 run tables in sign-orbit form for the FP64 or the FP32-storage step, or null
  std::unique_ptr<Tables3s3<double>> ts3d;
  std::unique_ptr<Tables3s3<float>> ts3f;
  // order 3: tables in device memory (init, fields)
  double* dHd = nullptr;          // Q x 30 FP64 (init)
  double* dcd = nullptr;          // Q x 4 FP64 (fields)
  double* dfref = nullptr;        // Q
  int* doff = nullptr;            // Q
  std::string err = "no error";
  ~rlbm3_handle() {
    for (void* b : buf) cudaFree(b);
    cudaFree(fields);
    cudaFree(staging);
    cudaFree(status);
    cudaFree(dHd);
    cudaFree(dcd);
    cudaFree(dfref);
    cudaFree(doff);
  }
};

namespace {

thread_local std::string g_err3 = "no error";

int fail3(rlbm3_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  else g_err3 = msg;
  return code;
}

int cuda_fail3(rlbm3_handle* h, cudaError_t e, const char* what) {
  return fail3(h, RLBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// MJ moments of the basis at rest (n, T): <1> = n/(2T), <p0> = n,
// <p^i p^i> = nT, <p0 p^i p^i> = 4 n T^2 (order 3), the others zero.
std::vector<double> rest_moments(int K, double n, double T) {
  std::vector<double> M(K, 0.0);
  M[0] = n / (2.0 * T);
  M[1] = n;
  M[8] = M[11] = M[13] = n * T;
  if (K == 30) M[14] = M[17] = M[19] = 4.0 * n * T * T;
  return M;
}

template <typename T>
int upload(void** dst, const std::vector<T>& v) {
  if (cudaMalloc(dst, v.size() * sizeof(T)) != cudaSuccess) { cudaGetLastError(); return RLBM_ERR_OOM; }
  if (cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) return RLBM_ERR_CUDA;
  return RLBM_OK;
}

// The order-3 run tables (sign-orbit form): 33 runs of 8 and 6 runs of 4
// with the non-zero components x y, x z, x y, x z, y z, y z; null when the
// table has another layout.
template <typename S>
std::unique_ptr<Tables3s3<S>> order3_runs(const Quadrature3& q, const std::vector<int>& offs) {
  static const int kMask4[kRuns4o3] = {3, 5, 3, 5, 6, 6};
  std::unique_ptr<Tables3s3<S>> t(new Tables3s3<S>());
  std::memset(t.get(), 0, sizeof(Tables3s3<S>));
  int n8 = 0, n4 = 0, i0 = 0;
  for (int mask : q.orbit_mask) {
    const int size = mask == 7 ? 8 : 4;
    if (i0 + size > q.Q || q.K != 30) return nullptr;
    const double* p = &q.p[4 * i0];
    const double mono[14] = {p[0], p[1], p[2], p[3], p[0] * p[0], p[0] * p[1], p[0] * p[2],
                             p[0] * p[3], p[1] * p[1], p[1] * p[2], p[1] * p[3], p[2] * p[2],
                             p[2] * p[3], p[3] * p[3]};
    S *H, *mo, *v;
    if (mask == 7 && n8 < kRuns8o3) {
      t->start8[n8] = i0;
      H = t->H8[n8], mo = t->mono8[n8], v = t->v8[n8];
      ++n8;
    } else if (mask != 7 && n4 < kRuns4o3 && mask == kMask4[n4]) {
      t->start4[n4] = i0;
      H = t->H4[n4], mo = t->mono4[n4], v = t->v4[n4];
      ++n4;
    } else {
      return nullptr;
    }
    for (int k = 0; k < 30; ++k) H[k] = (S)q.H[(size_t)i0 * 30 + k];
    for (int k = 0; k < 14; ++k) mo[k] = (S)mono[k];
    for (int k = 0; k < 3; ++k) v[k] = (S)(p[1 + k] / p[0]);
    i0 += size;
  }
  if (n8 != kRuns8o3 || n4 != kRuns4o3 || i0 != q.Q || (int)offs.size() != q.Q) return nullptr;
  for (int i = 0; i < q.Q; ++i) t->off[i] = offs[i];
  for (int r = 0; r < kRuns8o3; ++r)
    for (int k = 0; k < 8; ++k) t->off8[r][k] = offs[t->start8[r] + k];
  for (int r = 0; r < kRuns4o3; ++r)
    for (int k = 0; k < 4; ++k) t->off4[r][k] = offs[t->start4[r] + k];
  return t;
}

}  // namespace

extern "C" {

const char* rlbm3_last_error(const rlbm3_handle* h) { return h ? h->err.c_str() : g_err3.c_str(); }

int rlbm3_plan(int order, int* Q, int* K, int* nvec, double* p, double* w, double* H) {
  if (!Q || !K) return fail3(nullptr, RLBM_ERR_INVALID_ARG, "null argument");
  Quadrature3 q;
  std::string err;
  if (!massless3_tables(order, &q, &err)) return fail3(nullptr, RLBM_ERR_INVALID_ARG, err);
  *Q = q.Q;
  *K = q.K;
  for (int i = 0; i < q.Q; ++i) {
    if (nvec) for (int k = 0; k < 3; ++k) nvec[3 * i + k] = q.n[3 * i + k];
    if (p) for (int k = 0; k < 4; ++k) p[4 * i + k] = q.p[4 * i + k];
    if (w) w[i] = q.w[i];
    if (H) for (int k = 0; k < q.K; ++k) H[(size_t)q.K * i + k] = q.H[(size_t)i * q.K + k];
  }
  return RLBM_OK;
}

int rlbm3_create(int nx, int ny, int nz, double tau, int order, int precision, void* stream,
                 rlbm3_handle** out) {
  if (!out) return fail3(nullptr, RLBM_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (precision != RLBM_FP64 && precision != RLBM_FP32_STORE) return fail3(nullptr, RLBM_ERR_INVALID_ARG, "precision");
  if (order != 2 && order != 3) return fail3(nullptr, RLBM_ERR_INVALID_ARG, "order must be 2 or 3");
  // halo: the largest stencil component (3 at order 2, 6 at order 3); every
  // side at least that long, so that each halo cell is the image of exactly
  // one interior cell
  const int halo = order == 2 ? 3 : 6;
  if (nx < halo || ny < halo || nz < halo || (long long)nx * ny * nz > (1LL << 28))
    return fail3(nullptr, RLBM_ERR_INVALID_ARG, "grid size out of range (each side at least the halo width)");
  if (!(tau > 0.5)) return fail3(nullptr, RLBM_ERR_INVALID_ARG, "tau must exceed 1/2");
  std::unique_ptr<rlbm3_handle> h(new rlbm3_handle());
  std::string err;
  if (!massless3_tables(order, &h->q, &err)) return fail3(nullptr, RLBM_ERR_QUADRATURE, err);
  Scalars3& s = h->sc;
  s.Q = h->q.Q;
  s.nx = nx; s.ny = ny; s.nz = nz;
  s.h = halo;
  s.px = order == 2 ? 4 : 8;                         // 32-byte aligned interior rows, >= h
  s.pitch = ((s.px + nx + s.h) + 3) / 4 * 4;
  s.slab = (long long)(ny + 2 * s.h) * s.pitch;
  s.plane = ((long long)(nz + 2 * s.h) * s.slab + 31) / 32 * 32;
  s.tau = tau;
  h->elem = precision == RLBM_FP32_STORE ? 4 : 8;
  s.n_ref = h->elem == 4 ? 1.0 : 0.0;
  s.T_ref = h->elem == 4 ? 1.0 : 0.0;
  s.f_n_ref = (float)s.n_ref;
  s.f_T_ref = (float)s.T_ref;
  s.f_inv_tau = (float)(1.0 / s.tau);
  // order 2 keeps 32-bit pull offsets i * plane - shift; order 3 adds the
  // plane offset in 64 bits and keeps only the shift
  if (order == 2 && (long long)s.Q * s.plane >= (1LL << 31))
    return fail3(nullptr, RLBM_ERR_UNSUPPORTED, "grid too large for the order-2 table");
  const int K = h->q.K;
  h->fref.assign(s.Q, 0.0);
  if (h->elem == 4) {
    const std::vector<double> Mr = rest_moments(K, s.n_ref, s.T_ref);
    for (int i = 0; i < s.Q; ++i)
      for (int k = 0; k < K; ++k) h->fref[i] += h->q.H[(size_t)i * K + k] * Mr[k];
  }
  std::vector<int> offs(s.Q);
  for (int i = 0; i < s.Q; ++i) {
    const int* n = &h->q.n[3 * i];
    const long long shift = (long long)n[2] * s.slab + (long long)n[1] * s.pitch + n[0];
    offs[i] = (int)(order == 2 ? (long long)i * s.plane - shift : -shift);
  }
  h->tb.reset(new Tables3());
  std::memset(h->tb.get(), 0, sizeof(Tables3));
  if (order == 3) {
    std::vector<double> c(4 * s.Q);
    for (int i = 0; i < s.Q; ++i)
      for (int u = 0; u < 4; ++u) c[4 * i + u] = h->q.p[4 * i + u];
    int rc = RLBM_OK;           // (the steps take their run tables as kernel parameters)
    if (!rc) rc = upload((void**)&h->dHd, h->q.H);
    if (!rc) rc = upload((void**)&h->dcd, c);
    if (!rc) rc = upload((void**)&h->dfref, h->fref);
    if (!rc) rc = upload((void**)&h->doff, offs);
    if (rc) return fail3(nullptr, rc, "order-3 tables");
  }
  if (order == 3 && h->q.sym && h->elem == 8) h->ts3d = order3_runs<double>(h->q, offs);
  if (order == 3 && h->q.sym && h->elem == 4) h->ts3f = order3_runs<float>(h->q, offs);
  if (order == 2) {
    // sign-orbit form: 9 runs of 8, then the axis pairs along x, y and z
    static const int kMasks[kRuns3] = {7, 7, 7, 7, 7, 7, 7, 7, 7, 1, 2, 4};
    h->sym = h->q.sym && (int)h->q.orbit_mask.size() == kRuns3 &&
             std::equal(h->q.orbit_mask.begin(), h->q.orbit_mask.end(), kMasks);
    for (int r = 0; r < kRuns3 && h->sym; ++r) {
      const double* p = &h->q.p[4 * (r < 9 ? 8 * r : 72 + 2 * (r - 9))];
      const double mono[14] = {p[0], p[1], p[2], p[3], p[0] * p[0], p[0] * p[1], p[0] * p[2],
                               p[0] * p[3], p[1] * p[1], p[1] * p[2], p[1] * p[3], p[2] * p[2],
                               p[2] * p[3], p[3] * p[3]};
      for (int k = 0; k < 14; ++k) h->tb->mono[r][k] = mono[k];
      for (int k = 0; k < 14; ++k) h->tb->monof[r][k] = (float)mono[k];
    }
  }
  // the steps take the table in sign-orbit form (checked exactly above)
  if (order == 2 ? !h->sym : !(h->elem == 8 ? (bool)h->ts3d : (bool)h->ts3f))
    return fail3(nullptr, RLBM_ERR_QUADRATURE, "3-d table not in sign-orbit form");
  for (int i = 0; i < s.Q && order == 2; ++i) {
    for (int u = 0; u < 4; ++u) h->tb->c[i][u] = h->q.p[4 * i + u];
    for (int u = 0; u < 3; ++u) h->tb->v[i][u] = h->q.p[4 * i + 1 + u] / h->q.p[4 * i];
    for (int k = 0; k < 14; ++k) h->tb->H[i][k] = h->q.H[(size_t)i * 14 + k];
    for (int u = 0; u < 3; ++u) h->tb->vf[i][u] = (float)h->tb->v[i][u];
    for (int k = 0; k < 14; ++k) h->tb->Hf[i][k] = (float)h->tb->H[i][k];
    h->tb->fref[i] = h->fref[i];
    h->tb->off[i] = offs[i];
  }
  h->stream = (cudaStream_t)stream;
  const size_t bytes = (size_t)s.Q * s.plane * h->elem;
  const size_t nc = (size_t)nx * ny * nz;
  for (int b = 0; b < 2; ++b) {
    cudaError_t e = cudaMalloc(&h->buf[b], bytes);
    if (e != cudaSuccess) { cudaGetLastError(); return fail3(nullptr, RLBM_ERR_OOM, "population buffers"); }
  }
  if (cudaMalloc(&h->fields, 6 * nc * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&h->status, sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    return fail3(nullptr, RLBM_ERR_OOM, "field buffers");
  }
  cudaError_t e = cudaMemsetAsync(h->status, 0, sizeof(unsigned long long), h->stream);
  if (e != cudaSuccess) return cuda_fail3(nullptr, e, "status");
  *out = h.release();
  return RLBM_OK;
}

void rlbm3_destroy(rlbm3_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  delete h;
}

int rlbm3_stencil(const rlbm3_handle* h, int* Q, int* nvec, double* p, double* w) {
  if (!h || !Q) return RLBM_ERR_INVALID_ARG;
  *Q = h->q.Q;
  for (int i = 0; i < h->q.Q; ++i) {
    if (nvec) for (int k = 0; k < 3; ++k) nvec[3 * i + k] = h->q.n[3 * i + k];
    if (p) for (int k = 0; k < 4; ++k) p[4 * i + k] = h->q.p[4 * i + k];
    if (w) w[i] = h->q.w[i];
  }
  return RLBM_OK;
}

int rlbm3_init(rlbm3_handle* h, const double* n, const double* ux, const double* uy, const double* uz,
               const double* T, int on_device) {
  if (!h || !n || !ux || !uy || !uz || !T) return fail3(h, RLBM_ERR_INVALID_ARG, "null argument");
  const size_t nc = (size_t)h->sc.nx * h->sc.ny * h->sc.nz;
  const double* fp[5] = {n, ux, uy, uz, T};
  if (!on_device) {
    if (!h->staging) {
      cudaError_t e = cudaMalloc(&h->staging, 5 * nc * sizeof(double));
      if (e != cudaSuccess) { cudaGetLastError(); return fail3(h, RLBM_ERR_OOM, "staging"); }
    }
    const double* src[5] = {n, ux, uy, uz, T};
    for (int k = 0; k < 5; ++k) {
      cudaError_t e = cudaMemcpyAsync(h->staging + k * nc, src[k], nc * sizeof(double), cudaMemcpyHostToDevice,
                                      h->stream);
      if (e != cudaSuccess) return cuda_fail3(h, e, "copy of the initial fields");
    }
    for (int k = 0; k < 5; ++k) fp[k] = h->staging + k * nc;
  }
  cudaError_t e;
  if (h->q.order == 3) {
    if (h->elem == 4) {
      Init3qArgs<float> a{(float*)h->buf[h->cur], fp[0], fp[1], fp[2], fp[3], fp[4], h->sc, h->dHd, h->dfref};
      e = launch_init3q<float>(a, h->stream);
    } else {
      Init3qArgs<double> a{(double*)h->buf[h->cur], fp[0], fp[1], fp[2], fp[3], fp[4], h->sc, h->dHd, h->dfref};
      e = launch_init3q<double>(a, h->stream);
    }
  } else if (h->elem == 4) {
    Init3Args<float> a{(float*)h->buf[h->cur], fp[0], fp[1], fp[2], fp[3], fp[4], h->sc};
    e = launch_init3<float>(*h->tb, a, h->stream);
  } else {
    Init3Args<double> a{(double*)h->buf[h->cur], fp[0], fp[1], fp[2], fp[3], fp[4], h->sc};
    e = launch_init3<double>(*h->tb, a, h->stream);
  }
  if (e != cudaSuccess) return cuda_fail3(h, e, "init kernel");
  h->have_prev = false;
  if (!on_device) {
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail3(h, e, "init");
  }
  return RLBM_OK;
}

int rlbm3_step(rlbm3_handle* h, int nsteps) {
  if (!h || nsteps < 0) return fail3(h, RLBM_ERR_INVALID_ARG, "bad argument");
  for (int t = 0; t < nsteps; ++t) {
    cudaError_t e;
    if (h->q.order == 3) {
      if (h->elem == 4) {
        Step3qArgs<float> a{(const float*)h->buf[h->cur], (float*)h->buf[h->cur ^ 1], h->status, h->sc};
        e = launch_step3q_symf(*h->ts3f, a, h->stream);
      } else {
        Step3qArgs<double> a{(const double*)h->buf[h->cur], (double*)h->buf[h->cur ^ 1], h->status, h->sc};
        e = launch_step3q_sym(*h->ts3d, a, h->stream);
      }
    } else if (h->elem == 4) {
      Step3Args<float> a{(const float*)h->buf[h->cur], (float*)h->buf[h->cur ^ 1], h->status, h->sc};
      e = launch_step3f_sym(*h->tb, a, h->stream);
    } else {
      Step3Args<double> a{(const double*)h->buf[h->cur], (double*)h->buf[h->cur ^ 1], h->status, h->sc};
      e = launch_step3_sym(*h->tb, a, h->stream);
    }
    if (e != cudaSuccess) return cuda_fail3(h, e, "step kernel");
    h->cur ^= 1;
    h->have_prev = true;
  }
  return RLBM_OK;
}

int rlbm3_moments(rlbm3_handle* h, double* out, int on_device) {
  if (!h || !out) return fail3(h, RLBM_ERR_INVALID_ARG, "null argument");
  const size_t nc = (size_t)h->sc.nx * h->sc.ny * h->sc.nz;
  const void* fin = h->have_prev ? h->buf[h->cur ^ 1] : h->buf[h->cur];
  double* dst = on_device ? out : h->fields;
  const int pull = h->have_prev ? 1 : 0;
  cudaError_t e;
  if (h->q.order == 3) {
    if (h->elem == 4) {
      Fields3qArgs<float> a{(const float*)fin, pull, dst, h->sc, h->dcd, h->doff, h->dfref};
      e = launch_fields3q<float>(a, h->stream);
    } else {
      Fields3qArgs<double> a{(const double*)fin, pull, dst, h->sc, h->dcd, h->doff, h->dfref};
      e = launch_fields3q<double>(a, h->stream);
    }
  } else if (h->elem == 4) {
    Fields3Args<float> a{(const float*)fin, pull, dst, h->sc};
    e = launch_fields3<float>(*h->tb, a, h->stream);
  } else {
    Fields3Args<double> a{(const double*)fin, pull, dst, h->sc};
    e = launch_fields3<double>(*h->tb, a, h->stream);
  }
  if (e != cudaSuccess) return cuda_fail3(h, e, "fields kernel");
  if (!on_device) {
    e = cudaMemcpyAsync(out, h->fields, 6 * nc * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail3(h, e, "fields copy");
  }
  return RLBM_OK;
}

int rlbm3_get_populations(rlbm3_handle* h, double* f) {
  if (!h || !f) return fail3(h, RLBM_ERR_INVALID_ARG, "null argument");
  const Scalars3& s = h->sc;
  std::vector<unsigned char> host((size_t)s.Q * s.plane * h->elem);
  cudaError_t e = cudaMemcpyAsync(host.data(), h->buf[h->cur], host.size(), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail3(h, e, "population copy");
  const float* hf = (const float*)host.data();
  const double* hd = (const double*)host.data();
  size_t o = 0;
  for (int i = 0; i < s.Q; ++i)
    for (int z = 0; z < s.nz; ++z)
      for (int y = 0; y < s.ny; ++y)
        for (int x = 0; x < s.nx; ++x) {
          const size_t j = (size_t)i * s.plane + (size_t)(z + s.h) * s.slab + (size_t)(y + s.h) * s.pitch + x + s.px;
          f[o++] = h->elem == 4 ? (double)hf[j] + h->fref[i] : hd[j];
        }
  return RLBM_OK;
}

int rlbm3_sync_status(rlbm3_handle* h, long long* count) {
  if (!h) return RLBM_ERR_INVALID_ARG;
  unsigned long long v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, h->status, sizeof(v), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->status, 0, sizeof(v), h->stream);
  if (e != cudaSuccess) return cuda_fail3(h, e, "status");
  if (count) *count = (long long)v;
  return v ? RLBM_ERR_NONPHYSICAL : RLBM_OK;
}

}  // extern "C"
