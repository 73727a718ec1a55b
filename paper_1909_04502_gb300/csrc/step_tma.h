// TMA-staged step kernel (step_tma.cu): support test, tensor-map encoding
// and launcher.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <string>

#include "kernels.cuh"

struct rlbm_handle;

namespace rlbm {

// Tensor maps of the two population buffers for the two tile heights
// (index 0: 32 x 8 tiles, 1: 32 x 4 tiles).
struct TmaMaps {
  CUtensorMap m[2][2];
};

bool tma_supported(const rlbm_handle* h);
int tma_box_rows(int mode, int ty);
bool tma_encode(const rlbm_handle* h, void* buf, int box_rows, CUtensorMap* out, std::string* err);
cudaError_t launch_step_tma(const Tables<float>& tb, const StepArgs<float>& a, int mode, int ty,
                            const CUtensorMap& tm, cudaStream_t st);

}  // namespace rlbm
