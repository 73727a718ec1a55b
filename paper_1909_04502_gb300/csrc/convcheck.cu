// rlbm_convert_f32_f64: the FP32 <-> FP64 conversions the FP32-storage
// kernels run on the integer pipe (fpconv.cuh), applied element-wise to
// device arrays, so that they can be compared with the hardware conversions.
#include <cuda_runtime.h>

#include "../../include/rlbm.h"
#include "fpconv.cuh"

namespace {

__global__ void k_convert(const float* in_f, double* out_d, int nf, const double* in_d, float* out_f, int nd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nf) out_d[i] = rlbm::f2d(in_f[i]);
  if (i < nd) out_f[i] = rlbm::d2f(in_d[i]);
}

}  // namespace

extern "C" int rlbm_convert_f32_f64(const float* in_f, double* out_d, int nf, const double* in_d, float* out_f,
                                    int nd, void* stream) {
  if (nf < 0 || nd < 0 || (nf > 0 && (!in_f || !out_d)) || (nd > 0 && (!in_d || !out_f)))
    return RLBM_ERR_INVALID_ARG;
  const int n = nf > nd ? nf : nd;
  if (n == 0) return RLBM_OK;
  k_convert<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(in_f, out_d, nf, in_d, out_f, nd);
  return cudaGetLastError() == cudaSuccess ? RLBM_OK : RLBM_ERR_CUDA;
}
