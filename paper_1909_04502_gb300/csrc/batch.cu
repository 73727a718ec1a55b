// Batched RLBM: many independent simulations (different grid sizes, tau and
// stencils) advanced by persistent cooperative kernels, one per stencil kind
// present, captured together in one CUDA graph.  The per-cell update is the
// fused step of step_impl.cuh.
//
// Work decomposition: every instance's grid is cut into tiles of BX x BY
// cells, numbered consecutively over all instances with the tiles of each
// kind contiguous; block b of a kind's persistent grid of G blocks takes the
// b-th of G equal contiguous chunks of that kind's tiles in each time step,
// then waits at a grid-wide barrier before the next step.  The barrier spins a
// bounded number of times; on timeout it records RLBM_ERR_TIMEOUT and every
// block leaves.
//
// Second schedule (kChains): each instance's own single-grid step kernels,
// nsteps in a row, captured on one stream per instance so that the graph holds
// independent chains: an instance waits only on its own previous step, never
// on a grid-wide barrier, and the chains of different instances run
// concurrently.  The tuner picks whichever schedule is faster.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <utility>
#include <vector>

#include "../../include/rlbm.h"
#include "handle.h"
#include "step_impl.cuh"

namespace rlbm {

// Stencil kinds the batched kernel is compiled for (FP32 storage, order 2):
// the tables of each kind live in constant memory so that every constant is
// an instruction operand, as in the single-grid kernel.
enum BatchKind { kKindMassless = 0, kKindQ33 = 1, kKindQ25 = 2, kKindQ29 = 3, kKindMasslessBilinear = 4, kNumKinds = 5 };

__constant__ Tables<float> c_btab[kNumKinds];

struct BatchInst {
  Scalars s;
  float* buf[2];
  const float* tau_field;
  unsigned long long* status;
  int kind;
  int tiles_x;
  int tile_begin;
  int cur;               // buf[cur] holds f*(t) when a launch starts (updated by the kernel)
};

struct BarrierState {
  unsigned int count;
  unsigned int gen;
  unsigned int error;    // non-zero: a wait timed out
  unsigned int pad;
};

struct BatchArgs {
  BatchInst* inst;
  const int* tile_inst;  // instance of each tile
  int tile_lo, tile_hi;  // tiles of this launch's kind
  int nsteps;
  BarrierState* bar;
  unsigned long long* timeouts;
  long long spin_limit;  // iterations of the bounded barrier wait
};

// Grid-wide barrier for a cooperative launch, with a bounded wait.
// Returns false when the wait gave up or another block reported a timeout.
__device__ __forceinline__ bool grid_barrier(BarrierState* bar, unsigned long long* timeouts,
                                             long long spin_limit) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    volatile unsigned int* vgen = &bar->gen;
    volatile unsigned int* verr = &bar->error;
    const unsigned int gen = *vgen;
    __threadfence();
    const unsigned int arrived = atomicAdd(&bar->count, 1u);
    int ok = 1;
    if (arrived == gridDim.x - 1) {
      bar->count = 0;
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      long long it = 0;
      while (*vgen == gen) {
        if (*verr != 0u || ++it > spin_limit) {
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    if (!ok && atomicExch(&bar->error, 1u) == 0u) atomicAdd(timeouts, 1ULL);
    if (*verr != 0u) ok = 0;
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <int BX, int BY, int KIND>
__device__ __forceinline__ void batch_tile(const BatchInst& I, int tile, int step) {
  const int lt = tile - I.tile_begin;
  const int ty = lt / I.tiles_x, tx = lt - ty * I.tiles_x;
  const int x = tx * BX + (int)threadIdx.x;
  const int y = ty * BY + (int)threadIdx.y;
  if (x >= I.s.nx || y >= I.s.ny) return;
  const int c = (I.cur + step) & 1;
  const float* fin = I.buf[c];
  float* fout = I.buf[c ^ 1];
  if constexpr (KIND == kKindMassless)
    cell_update<float, 28, true, 9, kOnLattice, true, false, true>(c_btab[KIND], I.s, fin, fout, I.tau_field, I.status, x, y);
  else if constexpr (KIND == kKindQ33)
    cell_update<float, 33, true, 9, kOnLattice, true, false, true>(c_btab[KIND], I.s, fin, fout, I.tau_field, I.status, x, y);
  else if constexpr (KIND == kKindQ25)
    cell_update<float, 25, true, 9, kOnLattice, true, false, true>(c_btab[KIND], I.s, fin, fout, I.tau_field, I.status, x, y);
  else if constexpr (KIND == kKindQ29)
    cell_update<float, 29, true, 9, kOnLattice, true, false, true>(c_btab[KIND], I.s, fin, fout, I.tau_field, I.status, x, y);
  else
    cell_update<float, 28, true, 9, kBilinear, true, false, true>(c_btab[KIND], I.s, fin, fout, I.tau_field, I.status, x, y);
}

// One persistent kernel per stencil kind: a kernel compiled for a single
// population count keeps a per-kind register budget (a kernel holding every
// kind's cell update spills).  768 resident threads per SM (80 registers):
// the run-time offsets and the loop state need more registers than the
// single-grid kernel's 64, and at 1024 threads the spills cost more than the
// lost occupancy (measured 3-10 % slower).  The tiles of the kind's instances
// are the contiguous range [tile_lo, tile_hi).
template <int BX, int BY, int KIND>
__global__ void __launch_bounds__(BX * BY, 768 / (BX * BY)) k_batch(const __grid_constant__ BatchArgs a) {
  __shared__ BatchInst s_inst;
  constexpr int kWords = (int)(sizeof(BatchInst) / sizeof(int));
  static_assert(sizeof(BatchInst) % sizeof(int) == 0, "descriptor copied as words");
  const int tid = threadIdx.y * BX + threadIdx.x;
  // block b takes the contiguous chunk [lo, hi) of this kind's tiles, so the
  // instance (and its descriptor) changes only at chunk or instance boundaries
  const long long n = a.tile_hi - a.tile_lo;
  const int lo = a.tile_lo + (int)(n * blockIdx.x / gridDim.x);
  const int hi = a.tile_lo + (int)(n * (blockIdx.x + 1) / gridDim.x);
  int have = -1;                      // instance held in s_inst (the same in every thread)
  for (int step = 0; step < a.nsteps; ++step) {
    for (int t = lo; t < hi; ++t) {
      const int idx = __ldg(a.tile_inst + t);
      if (idx != have) {              // block-uniform
        __syncthreads();              // every thread is done with the previous descriptor
        const int* src = reinterpret_cast<const int*>(a.inst + idx);
        int* dst = reinterpret_cast<int*>(&s_inst);
        for (int w = tid; w < kWords; w += BX * BY) dst[w] = src[w];
        __syncthreads();
        have = idx;
      }
      batch_tile<BX, BY, KIND>(s_inst, t, step);
    }
    if (!grid_barrier(a.bar, a.timeouts, a.spin_limit)) return;
  }
}

// After a launch: instance cur flips by nsteps parity (run as a tiny kernel
// on the same stream, ordered after the persistent kernel).
__global__ void k_batch_flip(BatchInst* inst, int ninst, int nsteps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ninst) inst[i].cur ^= (nsteps & 1);
}

}  // namespace rlbm

using namespace rlbm;

struct rlbm_batch {
  std::vector<rlbm_handle*> h;
  std::vector<int> kind;
  std::vector<int> tile_begin, tiles_x;
  int total_tiles = 0;
  int kind_lo[kNumKinds] = {}, kind_hi[kNumKinds] = {};   // tile range of each kind (grouped by kind)
  cudaStream_t stream = nullptr;          // the user's stream (graphs are launched on it)
  cudaStream_t cap_stream = nullptr;      // private stream the graphs are captured on
  Tables<float>* tab_host = nullptr;     // pinned copy of the constant tables (graph memcpy source)
  BatchInst* inst_host = nullptr;        // pinned descriptor staging
  BatchInst* inst_dev = nullptr;
  int* tile_inst_dev = nullptr;
  BarrierState* bar = nullptr;
  unsigned long long* timeouts = nullptr;
  long long spin_limit = 1LL << 24;
  int tile_shape = 0;                     // 0: 32 x 8, 1: 32 x 4, 2: per-instance chains (autotuned)
  int grid = 0;                           // persistent grid size (autotuned)
  int grid_max[2] = {0, 0};               // co-resident limit per tile shape (smallest over the kinds present)
  // graphs by (nsteps, schedule, and for chains the buffer parity of every
  // instance, which the captured launches bake in)
  std::map<std::pair<long long, std::string>, cudaGraphExec_t> graphs;
  std::vector<cudaStream_t> chain_streams;  // one per instance (kChains capture)
  std::vector<cudaEvent_t> chain_events;    // fork, then one join per instance
  std::string err = "no error";
};

namespace {

int batch_fail(rlbm_batch* b, int code, const std::string& msg) {
  if (b) b->err = msg;
  return code;
}

int kind_of(const rlbm_handle* h, int* kind) {
  if (h->p.precision != RLBM_FP32_STORE || h->p.order != 2 || h->p.tau_mode == RLBM_TAU_FIELD) return -1;
  if (h->p.stream_mode == RLBM_BILINEAR) {
    if (h->q.Q == 28 && h->sc.sym) { *kind = kKindMasslessBilinear; return 0; }
    return -1;
  }
  if (h->q.Q == 28 && h->sc.sym) { *kind = kKindMassless; return 0; }
  if (h->q.Q == 33 && h->sc.sym) { *kind = kKindQ33; return 0; }
  if (h->q.Q == 25 && h->sc.sym) { *kind = kKindQ25; return 0; }
  if (h->q.Q == 29 && h->sc.sym) { *kind = kKindQ29; return 0; }
  return -1;
}

// Two handles share a kind's constant table only if their stencil tables agree.
bool same_stencil(const rlbm_handle* a, const rlbm_handle* b) {
  if (a->q.Q != b->q.Q || a->p.m != b->p.m || a->p.lambda != b->p.lambda || a->p.n_ref != b->p.n_ref ||
      a->p.T_ref != b->p.T_ref)
    return false;
  for (int i = 0; i < a->q.Q; ++i)
    if (a->q.p0[i] != b->q.p0[i] || a->q.px[i] != b->q.px[i] || a->q.py[i] != b->q.py[i] || a->q.w[i] != b->q.w[i])
      return false;
  return true;
}

template <int BX, int BY, int KIND>
cudaError_t launch_kind(rlbm_batch* b, int nsteps, int grid, cudaStream_t st) {
  BatchArgs a{b->inst_dev, b->tile_inst_dev, b->kind_lo[KIND], b->kind_hi[KIND], nsteps, b->bar, b->timeouts,
              b->spin_limit};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(BX, BY);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_batch<BX, BY, KIND>, a);
}

template <int BX, int BY>
cudaError_t launch_batch(rlbm_batch* b, int kind, int nsteps, int grid, cudaStream_t st) {
  switch (kind) {
    case kKindMassless: return launch_kind<BX, BY, kKindMassless>(b, nsteps, grid, st);
    case kKindQ33: return launch_kind<BX, BY, kKindQ33>(b, nsteps, grid, st);
    case kKindQ25: return launch_kind<BX, BY, kKindQ25>(b, nsteps, grid, st);
    case kKindQ29: return launch_kind<BX, BY, kKindQ29>(b, nsteps, grid, st);
    default: return launch_kind<BX, BY, kKindMasslessBilinear>(b, nsteps, grid, st);
  }
}

template <int BX, int BY>
int blocks_per_sm(int kind) {
  int nb = 0;
  const int threads = BX * BY;
  switch (kind) {
    case kKindMassless: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<BX, BY, kKindMassless>, threads, 0); break;
    case kKindQ33: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<BX, BY, kKindQ33>, threads, 0); break;
    case kKindQ25: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<BX, BY, kKindQ25>, threads, 0); break;
    case kKindQ29: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<BX, BY, kKindQ29>, threads, 0); break;
    default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<BX, BY, kKindMasslessBilinear>, threads, 0); break;
  }
  return nb;
}

constexpr int kChains = 2;

// kChains: fork from st into one stream per instance, enqueue each instance's
// nsteps single-grid steps there (rlbm_step on a borrowed stream; the handle's
// host state is restored, rlbm_batch_step advances it after the launch), join.
cudaError_t enqueue_chains(rlbm_batch* b, int nsteps, cudaStream_t st) {
  cudaError_t e = cudaEventRecord(b->chain_events[0], st);
  for (size_t i = 0; i < b->h.size() && e == cudaSuccess; ++i) {
    rlbm_handle* h = b->h[i];
    cudaStream_t ws = b->chain_streams[i];
    e = cudaStreamWaitEvent(ws, b->chain_events[0], 0);
    if (e != cudaSuccess) break;
    const cudaStream_t own = h->stream;
    const int cur = h->cur;
    const long long t = h->t;
    const bool have_prev = h->have_prev;
    h->stream = ws;
    const int rc = rlbm_step(h, nsteps);
    h->stream = own;
    h->cur = cur;
    h->t = t;
    h->have_prev = have_prev;
    if (rc != RLBM_OK) return cudaErrorLaunchFailure;
    e = cudaEventRecord(b->chain_events[1 + i], ws);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, b->chain_events[1 + i], 0);
  }
  return e;
}

// The kinds run one after another (each a cooperative launch of its own
// tiles); a kind with fewer tiles than the grid gets a grid of its tile count.
// The descriptors' buffer parity flips at the end under both schedules.
cudaError_t enqueue(rlbm_batch* b, int nsteps, cudaStream_t st) {
  if (b->tile_shape == kChains) {
    cudaError_t e = enqueue_chains(b, nsteps, st);
    if (e != cudaSuccess) return e;
    k_batch_flip<<<(int)((b->h.size() + 127) / 128), 128, 0, st>>>(b->inst_dev, (int)b->h.size(), nsteps);
    return cudaGetLastError();
  }
  cudaError_t e = cudaMemcpyToSymbolAsync(c_btab, b->tab_host, sizeof(Tables<float>) * kNumKinds, 0,
                                          cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  for (int k = 0; k < kNumKinds; ++k) {
    const int tiles = b->kind_hi[k] - b->kind_lo[k];
    if (tiles <= 0) continue;
    const int grid = std::min(b->grid, tiles);
    e = (b->tile_shape == 0) ? launch_batch<32, 8>(b, k, nsteps, grid, st) : launch_batch<32, 4>(b, k, nsteps, grid, st);
    if (e != cudaSuccess) return e;
  }
  k_batch_flip<<<(int)((b->h.size() + 127) / 128), 128, 0, st>>>(b->inst_dev, (int)b->h.size(), nsteps);
  return cudaGetLastError();
}

// Tile map for tile height by: the tiles of each kind form one contiguous
// range (kinds in enum order, instances in batch order inside a kind).
std::vector<int> build_tile_map(rlbm_batch* b, int by) {
  std::vector<int> tile_inst;
  int tiles = 0;
  for (int k = 0; k < kNumKinds; ++k) {
    b->kind_lo[k] = tiles;
    for (size_t i = 0; i < b->h.size(); ++i) {
      if (b->kind[i] != k) continue;
      const rlbm_handle* h = b->h[i];
      const int nt = ((h->p.nx + 31) / 32) * ((h->p.ny + by - 1) / by);
      b->tile_begin[i] = tiles;
      b->inst_host[i].tile_begin = tiles;
      for (int t = 0; t < nt; ++t) tile_inst.push_back((int)i);
      tiles += nt;
    }
    b->kind_hi[k] = tiles;
  }
  b->total_tiles = tiles;
  return tile_inst;
}

// Upload descriptors (instance buffers, current-buffer index) when the
// handles were stepped or re-initialised outside the batch.
int sync_descriptors(rlbm_batch* b) {
  bool dirty = false;
  for (size_t i = 0; i < b->h.size(); ++i) {
    const rlbm_handle* h = b->h[i];
    BatchInst& I = b->inst_host[i];
    if (I.cur != h->cur) { I.cur = h->cur; dirty = true; }
  }
  if (!dirty) return RLBM_OK;
  cudaError_t e = cudaMemcpyAsync(b->inst_dev, b->inst_host, sizeof(BatchInst) * b->h.size(), cudaMemcpyHostToDevice,
                                  b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return batch_fail(b, RLBM_ERR_CUDA, cudaGetErrorString(e));
  return RLBM_OK;
}

void drop_graphs(rlbm_batch* b) {
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  b->graphs.clear();
}

}  // namespace

extern "C" {

int rlbm_batch_create(const rlbm_params* params, int count, rlbm_batch** out) {
  if (!params || count <= 0 || !out) return RLBM_ERR_INVALID_ARG;
  *out = nullptr;
  std::unique_ptr<rlbm_batch> b(new rlbm_batch());
  b->stream = (cudaStream_t)params[0].stream;
  int rc = RLBM_OK;
  cudaError_t e;
  auto cleanup = [&]() {
    for (auto* h : b->h) rlbm_destroy(h);
    b->h.clear();
  };
  std::vector<const rlbm_handle*> kind_owner(kNumKinds, nullptr);
  for (int i = 0; i < count; ++i) {
    if (params[i].stream != params[0].stream) {
      cleanup();
      return RLBM_ERR_INVALID_ARG;
    }
    rlbm_handle* h = nullptr;
    rc = rlbm_create(&params[i], &h);
    if (rc != RLBM_OK) {
      cleanup();
      return rc;
    }
    b->h.push_back(h);
    int kind;
    if (kind_of(h, &kind) != 0) {
      cleanup();
      return RLBM_ERR_UNSUPPORTED;   // batched kernel: FP32 storage, order 2, built-in stencils
    }
    if (kind_owner[kind] && !same_stencil(kind_owner[kind], h)) {
      cleanup();
      return RLBM_ERR_UNSUPPORTED;   // one stencil table per kind
    }
    kind_owner[kind] = h;
    b->kind.push_back(kind);
  }
  b->tile_begin.assign(count, 0);
  // constant tables (pinned host source for the graph's memcpy node)
  e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMallocHost(&b->tab_host, sizeof(Tables<float>) * kNumKinds);
  if (e == cudaSuccess) e = cudaMallocHost(&b->inst_host, sizeof(BatchInst) * count);
  if (e == cudaSuccess) e = cudaMalloc(&b->inst_dev, sizeof(BatchInst) * count);
  if (e == cudaSuccess) e = cudaMalloc(&b->bar, sizeof(BarrierState));
  if (e == cudaSuccess) e = cudaMalloc(&b->timeouts, sizeof(unsigned long long));
  for (int i = 0; i < count && e == cudaSuccess; ++i) {
    cudaStream_t cs = nullptr;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) b->chain_streams.push_back(cs);
  }
  for (int i = 0; i <= count && e == cudaSuccess; ++i) {
    cudaEvent_t ev = nullptr;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) b->chain_events.push_back(ev);
  }
  if (e != cudaSuccess) {
    for (cudaStream_t cs : b->chain_streams) cudaStreamDestroy(cs);
    for (cudaEvent_t ev : b->chain_events) cudaEventDestroy(ev);
    b->chain_streams.clear();
    b->chain_events.clear();
    cleanup();
    return RLBM_ERR_OOM;
  }
  std::memset(b->tab_host, 0, sizeof(Tables<float>) * kNumKinds);
  for (int k = 0; k < kNumKinds; ++k)
    if (kind_owner[k]) b->tab_host[k] = *kind_owner[k]->tf;
  for (int i = 0; i < count; ++i) {
    rlbm_handle* h = b->h[i];
    BatchInst& I = b->inst_host[i];
    std::memset(&I, 0, sizeof(I));
    I.s = h->sc;
    I.buf[0] = (float*)h->buf[0];
    I.buf[1] = (float*)h->buf[1];
    I.tau_field = (const float*)h->tau_field;
    I.status = h->status;
    I.kind = b->kind[i];
    I.tiles_x = (h->p.nx + 31) / 32;     // tiles are 32 wide for both shapes
    I.cur = h->cur;
  }
  // the tile -> instance map starts with the 32 x 8 shape; rlbm_batch_config
  // rebuilds it for the 32 x 4 shape
  b->tile_shape = 0;
  std::vector<int> tile_inst = build_tile_map(b.get(), 8);
  const int tiles = b->total_tiles;
  // room for the 32 x 4 map (twice the tiles at most)
  e = cudaMalloc(&b->tile_inst_dev, sizeof(int) * (size_t)tiles * 2 + 64);
  if (e != cudaSuccess) {
    cleanup();
    return RLBM_ERR_OOM;
  }
  cudaMemcpy(b->tile_inst_dev, tile_inst.data(), sizeof(int) * tiles, cudaMemcpyHostToDevice);
  cudaMemcpy(b->inst_dev, b->inst_host, sizeof(BatchInst) * count, cudaMemcpyHostToDevice);
  cudaMemset(b->bar, 0, sizeof(BarrierState));
  cudaMemset(b->timeouts, 0, sizeof(unsigned long long));
  // co-resident grid limits for the cooperative launch
  int dev = 0, sms = 0, nb8 = 1 << 30, nb4 = 1 << 30;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  for (int k = 0; k < kNumKinds; ++k) {
    if (!kind_owner[k]) continue;
    nb8 = std::min(nb8, blocks_per_sm<32, 8>(k));
    nb4 = std::min(nb4, blocks_per_sm<32, 4>(k));
  }
  b->grid_max[0] = nb8 * sms;
  b->grid_max[1] = nb4 * sms;
  b->grid = b->grid_max[0];
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess || b->grid <= 0) {
    cleanup();
    return RLBM_ERR_CUDA;
  }
  *out = b.release();
  return RLBM_OK;
}

void rlbm_batch_destroy(rlbm_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  drop_graphs(b);
  for (auto* h : b->h) rlbm_destroy(h);
  cudaFreeHost(b->tab_host);
  cudaFreeHost(b->inst_host);
  cudaFree(b->inst_dev);
  cudaFree(b->tile_inst_dev);
  cudaFree(b->bar);
  cudaFree(b->timeouts);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  for (cudaStream_t cs : b->chain_streams) cudaStreamDestroy(cs);
  for (cudaEvent_t ev : b->chain_events) cudaEventDestroy(ev);
  delete b;
}

int rlbm_batch_size(const rlbm_batch* b) { return b ? (int)b->h.size() : -1; }

rlbm_handle* rlbm_batch_handle(rlbm_batch* b, int i) {
  if (!b || i < 0 || i >= (int)b->h.size()) return nullptr;
  return b->h[i];
}

int rlbm_batch_config(rlbm_batch* b, int tile_shape, int grid) {
  if (!b || tile_shape < 0 || tile_shape > kChains) return RLBM_ERR_INVALID_ARG;
  if (tile_shape == kChains) {          // the grid does not apply
    b->tile_shape = kChains;
    drop_graphs(b);
    return RLBM_OK;
  }
  const int gmax = b->grid_max[tile_shape];
  if (grid <= 0 || grid > gmax) return batch_fail(b, RLBM_ERR_INVALID_ARG, "grid exceeds co-resident blocks");
  if (tile_shape != b->tile_shape) {
    // rebuild the tile -> instance map and tile counts for the new shape
    std::vector<int> tile_inst = build_tile_map(b, tile_shape == 0 ? 8 : 4);
    const int tiles = b->total_tiles;
    cudaError_t e = cudaMemcpyAsync(b->tile_inst_dev, tile_inst.data(), sizeof(int) * tiles, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->inst_dev, b->inst_host, sizeof(BatchInst) * b->h.size(), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return batch_fail(b, RLBM_ERR_CUDA, cudaGetErrorString(e));
  }
  b->tile_shape = tile_shape;
  b->grid = grid;
  drop_graphs(b);
  return RLBM_OK;
}

int rlbm_batch_step(rlbm_batch* b, int nsteps) {
  if (!b || nsteps < 0) return RLBM_ERR_INVALID_ARG;
  if (nsteps == 0) return RLBM_OK;
  int rc = sync_descriptors(b);
  if (rc != RLBM_OK) return rc;
  std::string parity;
  if (b->tile_shape == kChains)
    for (const rlbm_handle* h : b->h) parity.push_back(h->cur ? '1' : '0');
  const std::pair<long long, std::string> key((long long)nsteps * 4 + b->tile_shape, parity);
  cudaGraphExec_t exec = nullptr;
  auto it = b->graphs.find(key);
  if (it != b->graphs.end()) {
    exec = it->second;
  } else {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return batch_fail(b, RLBM_ERR_CUDA, std::string("begin capture: ") + cudaGetErrorString(e));
    cudaError_t e2 = enqueue(b, nsteps, b->cap_stream);
    e = cudaStreamEndCapture(b->cap_stream, &g);
    if (e2 != cudaSuccess || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return batch_fail(b, RLBM_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e2 != cudaSuccess ? e2 : e));
    }
    e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return batch_fail(b, RLBM_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e));
    b->graphs[key] = exec;
  }
  cudaError_t e = cudaGraphLaunch(exec, b->stream);
  if (e != cudaSuccess) return batch_fail(b, RLBM_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
  for (size_t i = 0; i < b->h.size(); ++i) {
    rlbm_handle* h = b->h[i];
    h->cur ^= (nsteps & 1);
    h->t += nsteps;
    h->have_prev = true;
    b->inst_host[i].cur = h->cur;
  }
  return RLBM_OK;
}

int rlbm_batch_sync_status(rlbm_batch* b, long long* nonphysical) {
  if (!b) return RLBM_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return batch_fail(b, RLBM_ERR_CUDA, cudaGetErrorString(e));
  unsigned long long to = 0;
  e = cudaMemcpy(&to, b->timeouts, sizeof(to), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return batch_fail(b, RLBM_ERR_CUDA, cudaGetErrorString(e));
  long long total = 0;
  int worst = RLBM_OK;
  for (auto* h : b->h) {
    long long c = 0;
    int rc = rlbm_sync_status(h, &c);
    total += c;
    if (rc != RLBM_OK && worst == RLBM_OK) worst = rc;
  }
  if (nonphysical) *nonphysical = total;
  if (to) {
    cudaMemset(b->timeouts, 0, sizeof(unsigned long long));
    cudaMemset(b->bar, 0, sizeof(BarrierState));
    return batch_fail(b, RLBM_ERR_TIMEOUT, "grid barrier wait timed out");
  }
  return worst;
}

int rlbm_batch_set_spin_limit(rlbm_batch* b, long long limit) {
  if (!b || limit <= 0) return RLBM_ERR_INVALID_ARG;
  b->spin_limit = limit;
  drop_graphs(b);
  return RLBM_OK;
}

int rlbm_batch_info(const rlbm_batch* b, int* tile_shape, int* grid, int* grid_max, long long* total_tiles) {
  if (!b) return RLBM_ERR_INVALID_ARG;
  if (tile_shape) *tile_shape = b->tile_shape;
  if (grid) *grid = b->tile_shape == kChains ? 0 : b->grid;
  if (grid_max) { grid_max[0] = b->grid_max[0]; grid_max[1] = b->grid_max[1]; }
  if (total_tiles) *total_tiles = b->total_tiles;
  return RLBM_OK;
}

int rlbm_batch_tune(rlbm_batch* b, int trial_steps, int* tile_shape, int* grid, float* ms_per_step) {
  if (!b || trial_steps <= 0) return RLBM_ERR_INVALID_ARG;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return batch_fail(b, RLBM_ERR_CUDA, "event creation");
  float best = 1e30f;
  int best_shape = b->tile_shape, best_grid = b->grid;
  int rc = RLBM_OK;
  for (int shape = 0; shape < 2 && rc == RLBM_OK; ++shape) {
    const int gmax = b->grid_max[shape];
    const int cands[5] = {gmax, (gmax * 3) / 4, gmax / 2, gmax / 3, gmax / 4};
    for (int c = 0; c < 5 && rc == RLBM_OK; ++c) {
      if (cands[c] <= 0) continue;
      rc = rlbm_batch_config(b, shape, cands[c]);
      if (rc == RLBM_OK) rc = rlbm_batch_step(b, trial_steps);   // capture + warm-up
      if (rc != RLBM_OK) break;
      cudaEventRecord(e0, b->stream);
      rc = rlbm_batch_step(b, trial_steps);
      cudaEventRecord(e1, b->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) rc = batch_fail(b, RLBM_ERR_CUDA, "tuning run failed");
      if (rc != RLBM_OK) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) { best = ms; best_shape = shape; best_grid = cands[c]; }
    }
  }
  // the per-instance chains (no grid): two untimed runs capture the graphs of
  // both buffer parities, the third is timed
  if (rc == RLBM_OK) rc = rlbm_batch_config(b, kChains, 0);
  for (int rep = 0; rep < 3 && rc == RLBM_OK; ++rep) {
    if (rep < 2) {
      rc = rlbm_batch_step(b, trial_steps);
      continue;
    }
    cudaEventRecord(e0, b->stream);
    rc = rlbm_batch_step(b, trial_steps);
    cudaEventRecord(e1, b->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) rc = batch_fail(b, RLBM_ERR_CUDA, "tuning run failed");
    if (rc != RLBM_OK) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) { best = ms; best_shape = kChains; best_grid = 0; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != RLBM_OK) return rc;
  rc = rlbm_batch_config(b, best_shape, best_shape == kChains ? 0 : best_grid);
  if (tile_shape) *tile_shape = best_shape;
  if (grid) *grid = best_grid;
  if (ms_per_step) *ms_per_step = best / trial_steps;
  return rc;
}

const char* rlbm_batch_last_error(const rlbm_batch* b) { return b ? b->err.c_str() : "null batch"; }

}  // extern "C"
