// Host-callable launchers of the fused RLBM kernels (defined in step_o2.cu,
// step_o3.cu, step_o3m.cu).
#pragma once
#include "kernels.cuh"

namespace rlbm {

template <typename S>
cudaError_t launch_step_k9(const Tables<S>& tb, const StepArgs<S>& a, int mode, cudaStream_t st);
template <typename S>
cudaError_t launch_step_k16(const Tables<S>& tb, const StepArgs<S>& a, int mode, cudaStream_t st);
template <typename S>
cudaError_t launch_step_k16_massive_sym(const Tables<S>& tb, const StepArgs<S>& a, int mode, cudaStream_t st);
template <typename S>
cudaError_t launch_fields(const Tables<S>& tb, const MomentArgs<S>& a, int mode, cudaStream_t st);
template <typename S>
cudaError_t launch_init(const Tables<S>& tb, const InitArgs<S>& a, cudaStream_t st);

template <typename S>
inline cudaError_t launch_step(const Tables<S>& tb, const StepArgs<S>& a, int mode, cudaStream_t st) {
  return a.s.K == 9 ? launch_step_k9<S>(tb, a, mode, st) : launch_step_k16<S>(tb, a, mode, st);
}

}  // namespace rlbm
