// Orbit-symmetric order-3 (K = 16) instantiations of the fused step kernel
// for the built-in massive stencils (App. H columns A-D) and the paper's
// 45-vector performance-table stencil (Sec. 6.3), in a translation
// unit of their own so that they compile in parallel with step_o3.cu.
#include "dispatch.h"
#include "step_impl.cuh"

namespace rlbm {

template <typename S>
cudaError_t launch_step_k16_massive_sym(const Tables<S>& tb, const StepArgs<S>& a, int mode, cudaStream_t st) {
  switch (a.s.Q) {
    case 45: return launch_step_q<S, 45, true, 16, true>(tb, a, mode, st);
    case 49: return launch_step_q<S, 49, true, 16, true>(tb, a, mode, st);
    case 53: return launch_step_q<S, 53, true, 16, true>(tb, a, mode, st);
    case 57: return launch_step_q<S, 57, true, 16, true>(tb, a, mode, st);
    case 65: return launch_step_q<S, 65, true, 16, true>(tb, a, mode, st);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_step_k16_massive_sym<float>(const Tables<float>&, const StepArgs<float>&, int,
                                                         cudaStream_t);
template cudaError_t launch_step_k16_massive_sym<double>(const Tables<double>&, const StepArgs<double>&, int,
                                                          cudaStream_t);

}  // namespace rlbm
