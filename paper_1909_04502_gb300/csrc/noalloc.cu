// rlbm_step_noalloc: the fused step for callers that cannot allocate device
// memory.  Some callers run inside another runtime that owns the device
// memory (a plugin whose buffers come from the host application's pool), or
// must not allocate while they record or replay work, or cannot afford the
// device-wide synchronisation that cudaMalloc/cudaFree imply.  They pass the
// population buffers themselves; the only scratch the step kernel needs (the
// per-step count of non-physical cell updates) lives in a file-scope device
// array instead of a handle-owned allocation.
#include <cuda_runtime.h>

#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/rlbm.h"
#include "dispatch.h"
#include "setup.h"

// Provided by api.cu (host only, no device work): kernel tables and scalars
// for a parameter set, and the thread's error message of rlbm_last_error(NULL).
int rlbm_internal_prepare(const rlbm_params* p, rlbm::Scalars* sc, rlbm::Tables<float>* tf,
                          rlbm::Tables<double>* td, std::unique_ptr<rlbm::XeqTables>* txq, std::string* err);
void rlbm_internal_set_error(const std::string& msg);

namespace rlbm {
namespace {

// Largest nsteps of one call: one 8-byte counter per step.
constexpr int kNoallocMaxSteps = 1024;

// Shared by every call on a device (every GPU that loads the library holds
// its own copy until the process exits).  Host code must not use this name
// as a device address; it uses the address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned long long g_noalloc_counts[kNoallocMaxSteps];

std::mutex g_mutex;
std::map<int, unsigned long long*> g_scratch;        // device -> address of g_noalloc_counts

struct Prepared {
  Scalars sc;
  std::unique_ptr<Tables<float>> tf;
  std::unique_ptr<Tables<double>> td;
  std::unique_ptr<XeqTables> txq;   // extended-precision equilibrium (order 3, m~ >= 6, FP32), or null
};
std::map<std::string, std::shared_ptr<Prepared>> g_prepared;   // host-side tables per configuration

int set_error(int code, const std::string& msg) {
  rlbm_internal_set_error(msg);     // readable through rlbm_last_error(NULL)
  return code;
}

// Once per device, with that device current.
int scratch_address(unsigned long long** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(RLBM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  std::lock_guard<std::mutex> lock(g_mutex);
  auto it = g_scratch.find(dev);
  if (it != g_scratch.end()) {
    *out = it->second;
    return RLBM_OK;
  }
  unsigned long long* ptr = nullptr;
  e = cudaGetSymbolAddress((void**)&ptr, g_noalloc_counts);
  if (e != cudaSuccess || ptr == nullptr)
    return set_error(RLBM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  g_scratch[dev] = ptr;
  *out = ptr;
  return RLBM_OK;
}

// The key holds every field of rlbm_params that rlbm_internal_prepare reads
// (all of them but the stream), and the arrays that groups and custom_table
// point to.  The size check below fails to compile when a field is added to
// rlbm_params, so that the key is extended with it.
static_assert(sizeof(rlbm_params) == 176, "rlbm_params changed: extend config_key with the new field");

std::string config_key(const rlbm_params* p) {
  std::string k;
  auto add = [&k](const void* d, size_t n) { k.append((const char*)d, n); };
  add(&p->d, sizeof(p->d));
  add(&p->m, sizeof(p->m));
  add(&p->order, sizeof(p->order));
  add(&p->quadrature, sizeof(p->quadrature));
  add(&p->n_groups, sizeof(p->n_groups));
  if (p->groups && p->n_groups > 0) add(p->groups, sizeof(int) * 2 * p->n_groups);
  add(&p->v0, sizeof(p->v0));
  add(&p->custom_Q, sizeof(p->custom_Q));
  if (p->custom_table && p->custom_Q > 0) add(p->custom_table, sizeof(double) * 6 * p->custom_Q);
  add(&p->tau_mode, sizeof(p->tau_mode));
  add(&p->tau, sizeof(p->tau));
  add(&p->eta_over_s, sizeof(p->eta_over_s));
  add(&p->kappa, sizeof(p->kappa));
  add(&p->boundary, sizeof(p->boundary));
  add(&p->nx, sizeof(p->nx));
  add(&p->ny, sizeof(p->ny));
  add(&p->precision, sizeof(p->precision));
  add(&p->stream_mode, sizeof(p->stream_mode));
  add(&p->lambda, sizeof(p->lambda));
  add(&p->n_ref, sizeof(p->n_ref));
  add(&p->T_ref, sizeof(p->T_ref));
  add(&p->gx, sizeof(p->gx));             // the force decides Scalars::force and the kernel
  add(&p->gy, sizeof(p->gy));
  add(&p->wall_T[0], sizeof(p->wall_T));  // both wall temperatures
  return k;
}

// Host-side tables (quadrature, equilibrium matrix, kernel scalars), laid
// out exactly as rlbm_create lays them out, cached per configuration (host
// memory only).
int prepare(const rlbm_params* p, std::shared_ptr<Prepared>* out) {
  const std::string key = config_key(p);
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    auto it = g_prepared.find(key);
    if (it != g_prepared.end()) {
      *out = it->second;
      return RLBM_OK;
    }
  }
  auto pr = std::make_shared<Prepared>();
  if (p->precision == RLBM_FP32_STORE) pr->tf.reset(new Tables<float>());
  else pr->td.reset(new Tables<double>());
  std::string err;
  int rc = rlbm_internal_prepare(p, &pr->sc, pr->tf.get(), pr->td.get(), &pr->txq, &err);
  if (rc != RLBM_OK) return set_error(rc, err);
  std::lock_guard<std::mutex> lock(g_mutex);
  g_prepared[key] = pr;
  *out = pr;
  return RLBM_OK;
}

}  // namespace
}  // namespace rlbm

extern "C" int rlbm_step_noalloc(const rlbm_params* p, void* f_a, void* f_b, const void* tau_field,
                                 int nsteps, long long* counts) {
  using namespace rlbm;
  if (!p || !f_a || !f_b) return set_error(RLBM_ERR_INVALID_ARG, "null argument");
  if (nsteps < 1 || nsteps > kNoallocMaxSteps)
    return set_error(RLBM_ERR_INVALID_ARG, "nsteps must be in [1, 1024] (one scratch counter per step)");
  if (p->tau_mode == RLBM_TAU_FIELD && !tau_field)
    return set_error(RLBM_ERR_INVALID_ARG, "tau_mode RLBM_TAU_FIELD needs tau_field");
  std::shared_ptr<Prepared> pr;
  int rc = prepare(p, &pr);
  if (rc != RLBM_OK) return rc;
  unsigned long long* scratch = nullptr;
  rc = scratch_address(&scratch);
  if (rc != RLBM_OK) return rc;
  cudaStream_t st = (cudaStream_t)p->stream;
  cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(unsigned long long) * nsteps, st);
  if (e != cudaSuccess) return set_error(RLBM_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  const int mode = p->stream_mode == RLBM_BILINEAR ? kBilinear : kOnLattice;
  void* buf[2] = {f_a, f_b};
  for (int s = 0; s < nsteps; ++s) {
    const void* in = buf[s & 1];
    void* outp = buf[(s + 1) & 1];
    if (pr->tf) {
      StepArgs<float> a{pr->sc, (const float*)in, (float*)outp, (const float*)tau_field, scratch + s};
      e = pr->txq ? launch_step_xeq(*pr->tf, *pr->txq, a, mode, st) : launch_step<float>(*pr->tf, a, mode, st);
    } else {
      StepArgs<double> a{pr->sc, (const double*)in, (double*)outp, (const double*)tau_field, scratch + s};
      e = launch_step<double>(*pr->td, a, mode, st);
    }
    if (e != cudaSuccess) return set_error(RLBM_ERR_CUDA, std::string("step kernel: ") + cudaGetErrorString(e));
  }
  if (counts) {
    std::vector<unsigned long long> host(nsteps);
    e = cudaMemcpyAsync(host.data(), scratch, sizeof(unsigned long long) * nsteps, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_error(RLBM_ERR_CUDA, std::string("status copy: ") + cudaGetErrorString(e));
    bool bad = false;
    for (int s = 0; s < nsteps; ++s) {
      counts[s] = (long long)host[s];
      bad = bad || host[s] != 0;
    }
    if (bad) return set_error(RLBM_ERR_NONPHYSICAL, "non-physical cell updates (see counts)");
  }
  return RLBM_OK;
}

