// Internal state behind an rlbm_handle (include/rlbm.h).
#pragma once
#include <cuda_runtime.h>

#include <memory>
#include <string>
#include <vector>

#include "../../include/rlbm.h"
#include "dispatch.h"
#include "kernels.cuh"
#include "setup.h"
#include "step_tma.h"

struct rlbm_handle {
  rlbm_params p;                 // copy of the creation parameters (pointers cleared)
  rlbm::Quadrature q;            // discrete momenta and weights
  int K = 0;                     // moment-vector length
  std::vector<double> H;         // Q x K equilibrium matrix
  std::vector<double> fref;      // reference populations (shift of FP32 storage)
  rlbm::Scalars sc;              // kernel scalars
  std::unique_ptr<rlbm::Tables<float>> tf;    // kernel tables, FP32 storage
  std::unique_ptr<rlbm::Tables<double>> td;   // kernel tables, FP64
  std::unique_ptr<rlbm::XeqTables> txq;       // FP32 storage at order 3, m~ >= 6: extended-precision
                                              // equilibrium tables (step_xeq.cu), else null
  size_t elem = 4;               // bytes per stored population
  void* buf[2] = {nullptr, nullptr};   // ping-pong population buffers
  int cur = 0;                   // buf[cur] holds f*(t)
  bool have_prev = false;        // buf[cur ^ 1] holds f*(t-1)
  double* fields = nullptr;      // [14][plane] field output / staging
  void* tau_field = nullptr;     // per-cell tau, storage precision
  unsigned long long* status = nullptr;   // [0] non-physical count, [1] timeouts
  double* fref_dev = nullptr;    // fref on the device
  double* staging = nullptr;     // Q x ncell FP64 staging (lazy)
  cudaStream_t stream = nullptr;
  std::unique_ptr<rlbm::TmaMaps> tma;   // tensor maps of buf[0], buf[1] (TMA-staged kernel), or null
  int step_kernel = 0;           // RLBM_KERNEL_* requested by the caller (0: automatic)
  long long t = 0;
  std::string err = "no error";
};
