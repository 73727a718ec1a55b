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

// Extended-precision equilibrium of the order-3 massive FP32 step
// (step_xeq.cu): the low parts of the equilibrium matrix, H - (float)H, and
// m, n_ref, T_ref as (hi, lo) pairs.  Passed by value as a kernel parameter.
struct XeqTables {
  float Hl[kMaxQ][kMaxK];
  float m[2], n_ref[2], T_ref[2];
};
// Population counts with an orbit-symmetric order-3 kernel (the built-in
// App. H columns A-D and the 45-vector stencil of Sec. 6.3).
bool xeq_supported_q(int Q);
cudaError_t launch_step_xeq(const Tables<float>& tb, const XeqTables& xq, const StepArgs<float>& a, int mode,
                            cudaStream_t st);
cudaError_t launch_init_xeq(const Tables<float>& tb, const XeqTables& xq, const InitArgs<float>& a,
                            cudaStream_t st);

template <typename S>
inline cudaError_t launch_step(const Tables<S>& tb, const StepArgs<S>& a, int mode, cudaStream_t st) {
  return a.s.K == 9 ? launch_step_k9<S>(tb, a, mode, st) : launch_step_k16<S>(tb, a, mode, st);
}

}  // namespace rlbm
