// Order-3 (K = 16) instantiations of the fused step kernel.
#include "dispatch.h"
#include "step_impl.cuh"

namespace rlbm {

template <typename S>
cudaError_t launch_step_k16(const Tables<S>& tb, const StepArgs<S>& a, int mode, cudaStream_t st) {
  if (a.s.Q == 44 && a.s.sym) return launch_step_q<S, 44, true, 16, true>(tb, a, mode, st);   // massless order 3
  if (a.s.sym) return launch_step_k16_massive_sym<S>(tb, a, mode, st);                        // step_o3m.cu
  const int Q = a.s.Q;
  if (Q <= 48) return launch_step_q<S, 48, false, 16>(tb, a, mode, st);
  if (Q <= 56) return launch_step_q<S, 56, false, 16>(tb, a, mode, st);
  if (Q <= 64) return launch_step_q<S, 64, false, 16>(tb, a, mode, st);
  if (Q <= 72) return launch_step_q<S, 72, false, 16>(tb, a, mode, st);
  return cudaErrorInvalidValue;
}

template cudaError_t launch_step_k16<float>(const Tables<float>&, const StepArgs<float>&, int, cudaStream_t);
template cudaError_t launch_step_k16<double>(const Tables<double>&, const StepArgs<double>&, int, cudaStream_t);

}  // namespace rlbm
