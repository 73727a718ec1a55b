// Device side of the fused RLBM step (Sec. 6.2 of arXiv:1909.04502).
//
// Layout in HBM: structure of arrays, population plane i at offset
// i * plane, cell (x, y) at y * nx + x inside a plane; plane is nx*ny rounded
// up to a multiple of 32 elements.  FP32-storage handles store
// g_i = f_i - f_ref,i where f_ref is the equilibrium of the reference state
// (n_ref, U = (1,0,0), T_ref); streaming and collision are affine, so the
// shift is exact and keeps FP32 rounding proportional to |f - f_ref|.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "setup.h"

namespace rlbm {

enum { kOnLattice = 0, kBilinear = 1 };

// Per-handle constants, passed by value as a __grid_constant__ kernel
// parameter (constant bank: every warp reads the same population's entry).
template <typename R>
struct Tables {
  R c[kMaxQ][9];        // p0, px, py, p0p0, p0px, p0py, pxpx, pxpy, pypy
  R vx[kMaxQ], vy[kMaxQ];  // microscopic velocity v_i = p_i / p_i^0
  R H[kMaxQ][kMaxK];    // equilibrium matrix: f^eq_i - f_ref,i = sum_k H_ik dM_k
  R bw[kMaxQ][4];       // bilinear weights of taps (0,0), (1,0), (0,1), (1,1)
  int sxp[kMaxQ], syp[kMaxQ];   // on-lattice source offset -n_i reduced mod (nx, ny)
  int sxr[kMaxQ];               // raw -n_ix (free-flow clamp)
  int oxp[kMaxQ], oyp[kMaxQ];   // bilinear base tap offset o_i reduced mod (nx, ny)
  int oxr[kMaxQ];               // raw o_ix
};

struct Scalars {
  int Q, K, order;
  int nx, ny, ncell;
  long long plane;
  int boundary;          // 0 periodic, 1 free-flow in x
  int tau_mode;          // 0 const, 1 field, 2 eta/s
  double tau;            // const tau
  double tau_coef;       // (eta/s)(d+2) kappa  (tau = tau_coef / T)
  double m;              // rest mass m~
  double n_ref, T_ref;   // reference state (n_ref = 0: no shift)
  double N0_ref;         // n_ref
  double T00_ref;        // eps_ref = n_ref (m^2 + 2 m T_ref + 2 T_ref^2)/(m + T_ref)
  double Tii_ref;        // P_ref = n_ref T_ref
  double r2_ref;         // T_ref r2(T_ref) with r2(T) = (m^2 + 3mT + 3T^2)/(m+T)
  float kappa_guess;     // P/eps of the reference EOS, for the FP32 first guess
};

template <typename S>
struct StepArgs {
  Scalars s;
  const S* fin;          // f*(t) (or g*)
  S* fout;               // f*(t+1)
  const S* tau_field;    // per-cell tau (tau_mode 1)
  unsigned long long* status;   // count of non-physical cell updates
};

template <typename S>
struct MomentArgs {
  Scalars s;
  const S* fin;
  int gather;            // 1: stream first (fields of S f*), 0: fields of fin itself
  double* out;           // [14][plane]: n ux uy T eps N0 Nx Ny T00 T0x T0y Txx Txy Tyy
  int want_moments;      // write planes 5..13
  unsigned long long* status;
};

template <typename S>
struct InitArgs {
  Scalars s;
  const double* n;
  const double* ux;
  const double* uy;
  const double* T;
  S* fout;
  unsigned long long* status;
};

// Macroscopic state of one cell in FP64 (Sec. 6.2 steps 2-4).
struct Macro {
  double eps, U0, Ux, Uy, n, T;
  bool ok;
};

}  // namespace rlbm
