// Kernel-side tables and arguments of the (3+1)-d massless step (step3.cu).
#pragma once
#include <cuda_runtime.h>

#include "setup.h"

namespace rlbm {

constexpr int kRuns3 = 12;   // sign-orbit runs of the order-2 table

struct Tables3 {
  double c[kMaxQ3][4];    // p0, px, py, pz of population i
  double v[kMaxQ3][3];    // microscopic velocity p / p0
  double H[kMaxQ3][14];   // equilibrium matrix: f^eq_i = sum_k H_ik M_k
  double fref[kMaxQ3];    // FP32 storage: f_ref,i = f^eq_i(n_ref, rest, T_ref) (stored g = f - f_ref)
  float vf[kMaxQ3][3];    // FP32 copies of v and H
  float Hf[kMaxQ3][14];
  int off[kMaxQ3];        // pull source of population i relative to the cell: i * plane - n_i . strides
  // sign-orbit form (order 2: 9 runs of 8, then the axis pairs along x, y, z):
  // the moment monomials p0, px, py, pz, p0p0, p0px, p0py, p0pz, pxpx, pxpy,
  // pxpz, pypy, pypz, pzpz of each run's first member (all components >= 0),
  // in FP64 and rounded to FP32
  double mono[kRuns3][14];
  float monof[kRuns3][14];
};

struct Scalars3 {
  int Q, nx, ny, nz;
  int h, px, pitch;       // halo width, x offset of the interior, row pitch (elements)
  long long slab, plane;  // elements per z-slab and per population plane
  double tau;
  double n_ref, T_ref;    // FP32 storage reference state (0, 0 for FP64 storage)
  float f_n_ref, f_T_ref, f_inv_tau;   // FP32 copies of n_ref, T_ref and 1 / tau
};

// S: storage type (double: f; float: g = f - f_ref)
template <typename S>
struct Step3Args {
  const S* fin;
  S* fout;
  unsigned long long* status;
  Scalars3 s;
};

template <typename S>
struct Init3Args {
  S* f;
  const double *n, *ux, *uy, *uz, *T;   // device fields, row-major [z][y][x]
  Scalars3 s;
};

template <typename S>
struct Fields3Args {
  const S* fin;           // f*(t-1), pulled (pull = 1), or f*(0) read in place (pull = 0)
  int pull;
  double* out;            // [6][nz][ny][nx]: n, ux, uy, uz, T, eps
  Scalars3 s;
};

// Order 3 (Q = 288, K = 30): the step takes its tables as Tables3s3; init
// and fields read device arrays.
template <typename S>
struct Step3qArgs {
  const S* fin;
  S* fout;
  unsigned long long* status;
  Scalars3 s;
};

template <typename S>
struct Init3qArgs {
  S* f;
  const double *n, *ux, *uy, *uz, *T;
  Scalars3 s;
  const double* H;      // Q x 30
  const double* fref;   // Q
};

template <typename S>
struct Fields3qArgs {
  const S* fin;
  int pull;
  double* out;
  Scalars3 s;
  const double* c;      // Q x 4
  const int* off;       // Q pull shifts, as in Step3qArgs
  const double* fref;   // Q
};

template <typename S>
cudaError_t launch_init3q(const Init3qArgs<S>& a, cudaStream_t st);
template <typename S>
cudaError_t launch_fields3q(const Fields3qArgs<S>& a, cudaStream_t st);

// order 2, FP32 storage, in sign-orbit form (k_step3fs, Tables3::monof filled)
cudaError_t launch_step3f_sym(const Tables3& tb, const Step3Args<float>& a, cudaStream_t st);
// The order-3 table in sign-orbit form: 33 runs of 8 and 6 runs of 4 (the
// (5, 4, 0) patterns, non-zero components x y, x z, x y, x z, y z, y z), each
// run's first member's equilibrium row, moment monomials (as Tables3::mono)
// and velocity p / p0, the runs' first populations and the pull shifts.
constexpr int kRuns8o3 = 33, kRuns4o3 = 6;
template <typename S>
struct Tables3s3 {
  S H8[kRuns8o3][30], mono8[kRuns8o3][14], v8[kRuns8o3][3];
  S H4[kRuns4o3][30], mono4[kRuns4o3][14], v4[kRuns4o3][3];
  int start8[kRuns8o3], start4[kRuns4o3];
  int off[288];           // pull shifts -n_i . strides (i * plane added in 64 bits)
  int off8[kRuns8o3][8], off4[kRuns4o3][4];   // the same shifts by run and member
};
// order 3 in sign-orbit form: FP64 (k_step3qs) and FP32 storage (k_step3qsf)
template <typename S>
cudaError_t launch_step3q_sym(const Tables3s3<S>& tb, const Step3qArgs<S>& a, cudaStream_t st);
cudaError_t launch_step3q_symf(const Tables3s3<float>& tb, const Step3qArgs<float>& a, cudaStream_t st);

// FP64 step of the order-2 table in sign-orbit form (Tables3::mono filled)
template <typename S>
cudaError_t launch_step3_sym(const Tables3& tb, const Step3Args<S>& a, cudaStream_t st);
template <typename S>
cudaError_t launch_init3(const Tables3& tb, const Init3Args<S>& a, cudaStream_t st);
template <typename S>
cudaError_t launch_fields3(const Tables3& tb, const Fields3Args<S>& a, cudaStream_t st);

}  // namespace rlbm
