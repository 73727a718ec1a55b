// C ABI of the (3+1)-d massless step (include/rlbm.h, rlbm3_*).
#include <cuda_runtime.h>

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
  double* buf[2] = {nullptr, nullptr};
  int cur = 0;                    // buf[cur] holds f*(t)
  bool have_prev = false;         // buf[cur ^ 1] holds f*(t-1)
  double* fields = nullptr;       // [6][ncell]
  double* staging = nullptr;      // 5 input fields on the device (init from host)
  unsigned long long* status = nullptr;
  cudaStream_t stream = nullptr;
  std::string err = "no error";
  ~rlbm3_handle() {
    for (double* b : buf) cudaFree(b);
    cudaFree(fields);
    cudaFree(staging);
    cudaFree(status);
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

}  // namespace

extern "C" {

const char* rlbm3_last_error(const rlbm3_handle* h) { return h ? h->err.c_str() : g_err3.c_str(); }

int rlbm3_plan(int* Q, int* nvec, double* p, double* w, double* H) {
  if (!Q) return fail3(nullptr, RLBM_ERR_INVALID_ARG, "null argument");
  Quadrature3 q;
  std::string err;
  if (!massless3_tables(&q, &err)) return fail3(nullptr, RLBM_ERR_QUADRATURE, err);
  *Q = q.Q;
  for (int i = 0; i < q.Q; ++i) {
    if (nvec) for (int k = 0; k < 3; ++k) nvec[3 * i + k] = q.n[3 * i + k];
    if (p) for (int k = 0; k < 4; ++k) p[4 * i + k] = q.p[4 * i + k];
    if (w) w[i] = q.w[i];
    if (H) for (int k = 0; k < 14; ++k) H[14 * i + k] = q.H[(size_t)i * 14 + k];
  }
  return RLBM_OK;
}

int rlbm3_create(int nx, int ny, int nz, double tau, void* stream, rlbm3_handle** out) {
  if (!out) return fail3(nullptr, RLBM_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  // every side at least the stencil length 3, so that each halo cell is the
  // image of exactly one interior cell
  if (nx < 3 || ny < 3 || nz < 3 || (long long)nx * ny * nz > (1LL << 28))
    return fail3(nullptr, RLBM_ERR_INVALID_ARG, "grid size out of range (each side 3 ... )");
  if (!(tau > 0.5)) return fail3(nullptr, RLBM_ERR_INVALID_ARG, "tau must exceed 1/2");
  std::unique_ptr<rlbm3_handle> h(new rlbm3_handle());
  std::string err;
  if (!massless3_tables(&h->q, &err)) return fail3(nullptr, RLBM_ERR_QUADRATURE, err);
  Scalars3& s = h->sc;
  s.Q = h->q.Q;
  s.nx = nx; s.ny = ny; s.nz = nz;
  s.h = 3;
  s.px = 4;                                          // 32-byte aligned interior rows
  s.pitch = ((s.px + nx + s.h) + 3) / 4 * 4;
  s.slab = (long long)(ny + 2 * s.h) * s.pitch;
  s.plane = ((long long)(nz + 2 * s.h) * s.slab + 31) / 32 * 32;
  s.tau = tau;
  if ((long long)s.Q * s.plane >= (1LL << 31)) return fail3(nullptr, RLBM_ERR_UNSUPPORTED, "grid too large");
  h->tb.reset(new Tables3());
  std::memset(h->tb.get(), 0, sizeof(Tables3));
  for (int i = 0; i < s.Q; ++i) {
    for (int u = 0; u < 4; ++u) h->tb->c[i][u] = h->q.p[4 * i + u];
    for (int u = 0; u < 3; ++u) h->tb->v[i][u] = h->q.p[4 * i + 1 + u] / h->q.p[4 * i];
    for (int k = 0; k < 14; ++k) h->tb->H[i][k] = h->q.H[(size_t)i * 14 + k];
    const int* n = &h->q.n[3 * i];
    h->tb->off[i] = (int)((long long)i * s.plane - ((long long)n[2] * s.slab + (long long)n[1] * s.pitch + n[0]));
  }
  h->stream = (cudaStream_t)stream;
  const size_t bytes = (size_t)s.Q * s.plane * sizeof(double);
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
  Init3Args a{};
  a.f = h->buf[h->cur];
  a.s = h->sc;
  if (on_device) {
    a.n = n; a.ux = ux; a.uy = uy; a.uz = uz; a.T = T;
  } else {
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
    a.n = h->staging; a.ux = h->staging + nc; a.uy = h->staging + 2 * nc; a.uz = h->staging + 3 * nc;
    a.T = h->staging + 4 * nc;
  }
  cudaError_t e = launch_init3(*h->tb, a, h->stream);
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
    Step3Args a{};
    a.fin = h->buf[h->cur];
    a.fout = h->buf[h->cur ^ 1];
    a.status = h->status;
    a.s = h->sc;
    cudaError_t e = launch_step3(*h->tb, a, h->stream);
    if (e != cudaSuccess) return cuda_fail3(h, e, "step kernel");
    h->cur ^= 1;
    h->have_prev = true;
  }
  return RLBM_OK;
}

int rlbm3_moments(rlbm3_handle* h, double* out, int on_device) {
  if (!h || !out) return fail3(h, RLBM_ERR_INVALID_ARG, "null argument");
  const size_t nc = (size_t)h->sc.nx * h->sc.ny * h->sc.nz;
  Fields3Args a{};
  a.fin = h->have_prev ? h->buf[h->cur ^ 1] : h->buf[h->cur];
  a.pull = h->have_prev ? 1 : 0;
  a.out = on_device ? out : h->fields;
  a.s = h->sc;
  cudaError_t e = launch_fields3(*h->tb, a, h->stream);
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
  std::vector<double> host((size_t)s.Q * s.plane);
  cudaError_t e = cudaMemcpyAsync(host.data(), h->buf[h->cur], host.size() * sizeof(double),
                                  cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail3(h, e, "population copy");
  size_t o = 0;
  for (int i = 0; i < s.Q; ++i)
    for (int z = 0; z < s.nz; ++z)
      for (int y = 0; y < s.ny; ++y)
        for (int x = 0; x < s.nx; ++x)
          f[o++] = host[(size_t)i * s.plane + (size_t)(z + s.h) * s.slab + (size_t)(y + s.h) * s.pitch + x + s.px];
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
