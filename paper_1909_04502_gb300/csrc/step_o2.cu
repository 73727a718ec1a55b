// Order-2 (K = 9) instantiations of the fused kernels, and the field kernels
// for every population bucket.
#include "dispatch.h"
#include "step_impl.cuh"

namespace rlbm {

template <typename S>
cudaError_t launch_step_k9(const Tables<S>& tb, const StepArgs<S>& a, int mode, cudaStream_t st) {
  // exact orbit-symmetric instantiations for the built-in stencils (massless
  // Q = 28; massive m~ = 10, 5, 1: Q = 25, 29, 33), bounded buckets otherwise
  if (a.s.Q == 28 && a.s.sym) {
    if constexpr (sizeof(S) == 4)
      if (a.macro) return launch_step_q<S, 28, true, 9, true, true>(tb, a, mode, st);
    return launch_step_q<S, 28, true, 9, true>(tb, a, mode, st);
  }
  if (a.macro) return cudaErrorInvalidValue;   // macroscopic output: built-in massless FP32 stencil only
  if (a.s.sym_fw) {                             // the same with the force term or equilibrium walls
    switch (a.s.Q) {
      case 28: return launch_step_q<S, 28, true, 9, true, false, true>(tb, a, mode, st);
      case 25: return launch_step_q<S, 25, true, 9, true, false, true>(tb, a, mode, st);
      case 29: return launch_step_q<S, 29, true, 9, true, false, true>(tb, a, mode, st);
      case 33: return launch_step_q<S, 33, true, 9, true, false, true>(tb, a, mode, st);
      default: break;
    }
  }
  if (a.s.sym) {
    switch (a.s.Q) {
      case 25: return launch_step_q<S, 25, true, 9, true>(tb, a, mode, st);
      case 29: return launch_step_q<S, 29, true, 9, true>(tb, a, mode, st);
      case 33: return launch_step_q<S, 33, true, 9, true>(tb, a, mode, st);
      default: break;
    }
  }
  const int Q = a.s.Q;
  if (Q <= 32) return launch_step_q<S, 32, false, 9>(tb, a, mode, st);
  if (Q <= 40) return launch_step_q<S, 40, false, 9>(tb, a, mode, st);
  if (Q <= 48) return launch_step_q<S, 48, false, 9>(tb, a, mode, st);
  return cudaErrorInvalidValue;
}

template <typename S>
cudaError_t launch_fields(const Tables<S>& tb, const MomentArgs<S>& a, int mode, cudaStream_t st) {
  const int Q = a.s.Q;
  if (Q <= 32) return launch_fields_q<S, 32, false>(tb, a, mode, st);
  if (Q <= 48) return launch_fields_q<S, 48, false>(tb, a, mode, st);
  if (Q <= 72) return launch_fields_q<S, 72, false>(tb, a, mode, st);
  return cudaErrorInvalidValue;
}

template <typename S>
cudaError_t launch_init(const Tables<S>& tb, const InitArgs<S>& a, cudaStream_t st) {
  if (a.s.K == 9) return launch_init_k<S, 9>(tb, a, st);
  if (a.s.K == 16) return launch_init_k<S, 16>(tb, a, st);
  return cudaErrorInvalidValue;
}

template cudaError_t launch_step_k9<float>(const Tables<float>&, const StepArgs<float>&, int, cudaStream_t);
template cudaError_t launch_step_k9<double>(const Tables<double>&, const StepArgs<double>&, int, cudaStream_t);
template cudaError_t launch_fields<float>(const Tables<float>&, const MomentArgs<float>&, int, cudaStream_t);
template cudaError_t launch_fields<double>(const Tables<double>&, const MomentArgs<double>&, int, cudaStream_t);
template cudaError_t launch_init<float>(const Tables<float>&, const InitArgs<float>&, cudaStream_t);
template cudaError_t launch_init<double>(const Tables<double>&, const InitArgs<double>&, cudaStream_t);

}  // namespace rlbm
