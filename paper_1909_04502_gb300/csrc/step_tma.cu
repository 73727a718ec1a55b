// Fused RLBM step with TMA-staged streaming (FP32 storage, massless order-2
// stencil, Q = 28, on-lattice or bilinear pull; Sec. 6.2 steps 1-8).
//
// A persistent CTA of 32 x TY threads walks the grid's 32 x TY tiles with a
// stride of gridDim.x.  For each tile, one thread issues 28 tensor copies
// (cp.async.bulk.tensor, one per population: the rectangle of the population's
// plane that the tile pulls from) into one of two shared-memory stages and
// arms the stage's mbarrier with the byte count.  The copies for tile j + 2
// are issued as soon as every thread has read tile j out of its stage, so
// the HBM reads of later tiles overlap the collision arithmetic of the
// current ones instead of alternating with it.  The pull then reads shared
// memory: on-lattice one element per population, bilinear the four taps.
//
// Box geometry: the copy of population i for a tile at column x0 starts at
// column x0 + px + dx_i rounded down to a multiple of 4 elements (a tensor
// copy must start on a 16-byte boundary); x0 and px are multiples of 8
// elements, so the remainder r_i = dx_i & 3 is the same for every tile and
// the thread of column c reads box column c + r_i (+1 for the bilinear tap).
// Boxes are 36 columns wide (r_i + 32 + 1 <= 36) and TY (+1 bilinear) rows
// high.  Box reads past the end of a plane fill zeros and are never used.
//
// Every wait on an mbarrier is bounded (about one second of clock cycles);
// a wait that runs out makes the CTA record a timeout in status[1], wait
// (bounded again) for its own copies still in flight, and leave.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/rlbm.h"
#include "handle.h"
#include "step_impl.cuh"
#include "step_tma.h"

namespace rlbm {

namespace {

constexpr int kBoxW = 36;
constexpr long long kWaitCycles = 2LL << 30;   // ~1 s at the GB300 SM clock

template <int MODE, int TY>
struct TmaShape {
  static constexpr int kBoxH = TY + (MODE == kBilinear ? 1 : 0);
  static constexpr int kSlab = ((kBoxH * kBoxW * 4 + 127) / 128) * 128;   // bytes per population, 128-B aligned
  static constexpr int kStage = 28 * kSlab;
  static constexpr int kSmem = 2 * kStage + 64;                            // + two mbarriers
  static constexpr unsigned kTx = 28u * kBoxH * kBoxW * 4u;                // bytes the 28 copies deliver
};

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0u;
}

// Bounded wait for the completion of phase `parity` of an mbarrier.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > kWaitCycles) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, int x, int y, int z,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"((unsigned long long)tm), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

template <int MODE, int TY>
__device__ __forceinline__ void issue_tile(const Tables<float>& tb, const Scalars& s, const CUtensorMap* tm,
                                           unsigned char* stage, unsigned long long* bar, int tile, int tiles_x) {
  using Sh = TmaShape<MODE, TY>;
  const int ty0 = tile / tiles_x;
  const int x0 = (tile - ty0 * tiles_x) * 32 + s.px;
  const int y0 = ty0 * TY + s.hy;
  mbar_expect_tx(bar, Sh::kTx);
#pragma unroll
  for (int i = 0; i < 28; ++i) {
    const int xs = x0 + (int)tb.dx[i];     // >= 0: px >= hx >= -dx_i
    tma_load_3d(stage + i * Sh::kSlab, tm, xs & ~3, y0 + (int)tb.dy[i], i, bar);
  }
}

template <int MODE, int TY>
__device__ __forceinline__ void gather_smem(const Tables<float>& tb, const unsigned char* stage, int cx, int cy,
                                            float (&g)[28]) {
  using Sh = TmaShape<MODE, TY>;
#pragma unroll
  for (int i = 0; i < 28; ++i) {
    const float* sl = reinterpret_cast<const float*>(stage + i * Sh::kSlab) + cy * kBoxW + cx + ((int)tb.dx[i] & 3);
    if constexpr (MODE == kOnLattice) {
      g[i] = sl[0];
    } else {
      float v = tb.bw[i][0] * sl[0];
      v = fmaf(tb.bw[i][1], sl[1], v);
      v = fmaf(tb.bw[i][2], sl[kBoxW], v);
      v = fmaf(tb.bw[i][3], sl[kBoxW + 1], v);
      g[i] = v;
    }
  }
}

template <int MODE, int TY>
constexpr int tma_min_blocks() {
  return (228 * 1024) / (TmaShape<MODE, TY>::kSmem + 1024) < 1 ? 1 : (228 * 1024) / (TmaShape<MODE, TY>::kSmem + 1024);
}

template <int MODE, int TY>
__global__ void __launch_bounds__(32 * TY, tma_min_blocks<MODE, TY>())
    k_step_tma(const __grid_constant__ Tables<float> tb, const __grid_constant__ StepArgs<float> a,
               const __grid_constant__ CUtensorMap tm) {
  using Sh = TmaShape<MODE, TY>;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem + 2 * Sh::kStage);
  const Scalars& s = a.s;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  const int tiles_x = (s.nx + 31) / 32;
  const int ntiles = tiles_x * ((s.ny + TY - 1) / TY);
  const int G = (int)gridDim.x;
  if (tid == 0) {
    asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&tm) : "memory");
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {
    for (int j = 0; j < 2; ++j) {
      const int t = (int)blockIdx.x + j * G;
      if (t < ntiles) issue_tile<MODE, TY>(tb, s, &tm, smem + j * Sh::kStage, &bar[j], t, tiles_x);
    }
  }
  int j = 0;
  for (int t = (int)blockIdx.x; t < ntiles; t += G, ++j) {
    const int st = j & 1;
    const unsigned par = (unsigned)(j >> 1) & 1u;
    const bool ok = mbar_wait_bounded(&bar[st], par);
    if (__syncthreads_or(!ok)) {
      // give up: record it, let this CTA's copies in flight land, leave
      if (tid == 0) {
        atomicAdd(a.status + 1, 1ULL);
        mbar_wait_bounded(&bar[st], par);
        if (t + G < ntiles) mbar_wait_bounded(&bar[st ^ 1], (unsigned)((j + 1) >> 1) & 1u);
      }
      __syncthreads();
      return;
    }
    float g[28];
    gather_smem<MODE, TY>(tb, smem + st * Sh::kStage, threadIdx.x, threadIdx.y, g);
    __syncthreads();   // every thread has read stage st
    if (tid == 0 && t + 2 * G < ntiles)
      issue_tile<MODE, TY>(tb, s, &tm, smem + st * Sh::kStage, &bar[st], t + 2 * G, tiles_x);
    const int ty0 = t / tiles_x;
    const int x = (t - ty0 * tiles_x) * 32 + (int)threadIdx.x;
    const int y = ty0 * TY + (int)threadIdx.y;
    if (x < s.nx && y < s.ny) collide_store<float, 28, true, 9, true>(tb, s, g, a.fout, a.tau_field, a.status, x, y);
  }
}

template <int MODE, int TY>
cudaError_t launch_variant(const Tables<float>& tb, const StepArgs<float>& a, const CUtensorMap& tm,
                           cudaStream_t st) {
  using Sh = TmaShape<MODE, TY>;
  static int blocks_per_sm = -1;
  static int sms = 0;
  static std::once_flag once;
  static cudaError_t init_err = cudaSuccess;
  std::call_once(once, [] {
    init_err = cudaFuncSetAttribute(k_step_tma<MODE, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, Sh::kSmem);
    int dev = 0;
    if (init_err == cudaSuccess) init_err = cudaGetDevice(&dev);
    if (init_err == cudaSuccess) init_err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (init_err == cudaSuccess)
      init_err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_step_tma<MODE, TY>, 32 * TY,
                                                              Sh::kSmem);
  });
  if (init_err != cudaSuccess) return init_err;
  if (blocks_per_sm <= 0) return cudaErrorInvalidConfiguration;
  const long long ntiles = (long long)((a.s.nx + 31) / 32) * ((a.s.ny + TY - 1) / TY);
  const int grid = (int)std::min<long long>(ntiles, (long long)blocks_per_sm * sms);
  k_step_tma<MODE, TY><<<grid, dim3(32, TY), Sh::kSmem, st>>>(tb, a, tm);
  return cudaGetLastError();
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn(std::string* err) {
  static EncodeFn fn = nullptr;
  static std::once_flag once;
  static std::string why;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p)
      why = "cuTensorMapEncodeTiled is not available from the driver";
    else
      fn = reinterpret_cast<EncodeFn>(p);
  });
  if (!fn && err) *err = why;
  return fn;
}

}  // namespace

// FP32 storage, the massless Q = 28 order-2 stencil in orbit order (the
// kernel uses the orbit-symmetric collision, like the direct kernel for this
// stencil), and a padded layout at
// least one box wide and high (smaller grids use the direct-load kernel).
bool tma_supported(const rlbm_handle* h) {
  const Scalars& s = h->sc;
  return h->elem == 4 && h->q.Q == 28 && s.sym && h->K == 9 && (s.px % 8) == 0 && (s.pitch % 8) == 0 &&
         (s.plane % 8) == 0 && s.pitch >= kBoxW && s.ny + 2 * s.hy >= 9;
}

int tma_box_rows(int mode, int ty) { return ty + (mode == kBilinear ? 1 : 0); }

// Tensor map of one population buffer: dims (pitch, ny + 2 hy, Q) in
// elements, row stride pitch * 4 B, plane stride plane * 4 B, box
// (36, box_rows, 1), no swizzle, zero fill outside.
bool tma_encode(const rlbm_handle* h, void* buf, int box_rows, CUtensorMap* out, std::string* err) {
  EncodeFn fn = encode_fn(err);
  if (!fn) return false;
  const Scalars& s = h->sc;
  const cuuint64_t dims[3] = {(cuuint64_t)s.pitch, (cuuint64_t)(s.ny + 2 * s.hy), (cuuint64_t)s.Q};
  const cuuint64_t strides[2] = {(cuuint64_t)s.pitch * 4u, (cuuint64_t)s.plane * 4u};
  const cuuint32_t box[3] = {(cuuint32_t)kBoxW, (cuuint32_t)box_rows, 1u};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  CUresult r = fn(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, buf, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    if (err) *err = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
    return false;
  }
  return true;
}

cudaError_t launch_step_tma(const Tables<float>& tb, const StepArgs<float>& a, int mode, int ty,
                            const CUtensorMap& tm, cudaStream_t st) {
  if (mode == kBilinear)
    return ty == 8 ? launch_variant<kBilinear, 8>(tb, a, tm, st) : launch_variant<kBilinear, 4>(tb, a, tm, st);
  return ty == 8 ? launch_variant<kOnLattice, 8>(tb, a, tm, st) : launch_variant<kOnLattice, 4>(tb, a, tm, st);
}

}  // namespace rlbm
