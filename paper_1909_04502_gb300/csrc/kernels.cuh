// Device side of the fused RLBM step (Sec. 6.2 of arXiv:1909.04502).
//
// Layout in HBM: structure of arrays.  Population plane i starts at element
// i * plane.  Inside a plane, rows have a stride of `pitch` elements and the
// interior cell (x, y) sits at (y + hy) * pitch + (x + px); around the
// interior a halo of hx cells (left and right) and hy rows (top and bottom)
// holds copies of cells: periodic images, or the boundary cell for free-flow
// ends.  The step kernel writes each result into the interior and into every
// halo position that shows the same cell, so the next step's pull reads need
// no wrap-around arithmetic.  px (>= hx) aligns row starts to 32 bytes.
//
// FP32-storage handles store g_i = f_i - f_ref,i where f_ref is the
// equilibrium of the reference state (n_ref, U = (1,0,0), T_ref); streaming
// and collision are affine, so the shift is exact and keeps FP32 rounding
// proportional to |f - f_ref|.
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
  R c[kMaxQ][9];           // p0, px, py, p0p0, p0px, p0py, pxpx, pxpy, pypy
  R vx[kMaxQ], vy[kMaxQ];  // microscopic velocity v_i = p_i / p_i^0
  R H[kMaxQ][kMaxK];       // equilibrium matrix: f^eq_i - f_ref,i = sum_k H_ik dM_k
  R bw[kMaxQ][4];          // bilinear weights of taps (0,0), (1,0), (0,1), (1,1)
  int off[kMaxQ];          // pull source offset in elements: on-lattice -n_iy*pitch - n_ix;
                           // bilinear o_iy*pitch + o_ix (tap (0,0))
  short dx[kMaxQ], dy[kMaxQ];   // the same offset before the pitch is applied: off = dy*pitch + dx
  int roff[kMaxQ];         // transposed streaming (adjoint pull) relative to the cell, plane
                           // included: pl[i] + n_iy*pitch + n_ix on-lattice; bilinear
                           // pl[i] + (-o_iy-1)*pitch + (-o_ix-1), tap weights bw[i][3-k]
  int pl[kMaxQ];           // i * plane: start of population plane i
  int offp[kMaxQ];         // pl[i] + off[i]: pull source of population i relative to the cell
  int offr[kMaxQ];         // offp[i] + pitch: the bilinear taps' second row
  R fref[kMaxQ];           // reference populations f_ref,i (0 without the storage shift)
};

struct Scalars {
  int Q, K, order;
  int nx, ny, ncell;
  int pitch, hx, hy, px;   // padded layout (see file comment)
  long long plane;
  int boundary;            // 0 periodic, 1 free-flow in x
  int tau_mode;            // 0 const, 1 field, 2 eta/s
  double tau;              // const tau
  double tau_coef;         // (eta/s)(d+2) kappa  (tau = tau_coef / T)
  double m;                // rest mass m~
  double n_ref, T_ref;     // reference state (n_ref = 0: no shift)
  double N0_ref;           // n_ref
  double T00_ref;          // eps_ref = n_ref (m^2 + 2 m T_ref + 2 T_ref^2)/(m + T_ref)
  double Tii_ref;          // P_ref = n_ref T_ref
  double PE_ref;           // P_ref + eps_ref
  double n_ref2;           // n_ref^2
  float kappa_guess;       // P/eps of the reference EOS, for the FP32 first guess
  int massless;            // m == 0
  int sym;                 // orbit-ordered stencil with exactly symmetric H (and no force, no walls)
  int force;               // gravity-like force present (m > 0 and g != 0)
  double gx, gy;           // its acceleration
  float f_gx, f_gy;
  double wall_T[2];        // equilibrium walls: prescribed temperature of the first / last column (0: own T)
  float f_wall_T[2];
  int iplane;              // plane as int (Q * plane < 2^31 is checked at creation)
  // FP32 copies of the scalars used by the FP32-storage kernels
  float f_tau, f_tau_coef, f_m, f_n_ref, f_T_ref, f_T00_ref, f_Tii_ref;
  float f_PE_hi, f_PE_lo;  // P_ref + eps_ref as a float-float pair (hi + lo)
  int sym_fw;              // orbit-ordered stencil with exactly symmetric H, with a force or walls
};

// Parity of the px and py exponents of basis monomial k of setup.h
// (1 | p0 px py | p0px p0py pxpx pxpy pypy | p0pxpx p0pxpy p0pypy pxpxpx
// pxpxpy pxpypy pypypy), and the monomial with the two exponents exchanged.
__host__ __device__ constexpr int mono_ax(int k) {
  return (k == 2 || k == 4 || k == 7 || k == 10 || k == 12 || k == 14) ? 1 : 0;
}
__host__ __device__ constexpr int mono_ay(int k) {
  return (k == 3 || k == 5 || k == 7 || k == 10 || k == 13 || k == 15) ? 1 : 0;
}
__host__ __device__ constexpr int mono_swap(int k) {
  return k == 2 ? 3 : k == 3 ? 2 : k == 4 ? 5 : k == 5 ? 4 : k == 6 ? 8 : k == 8 ? 6 : k == 9 ? 11 : k == 11 ? 9
       : k == 12 ? 15 : k == 15 ? 12 : k == 13 ? 14 : k == 14 ? 13 : k;
}

// Storage index of interior cell (x, y).
__host__ __device__ __forceinline__ long long sidx(const Scalars& s, int x, int y) {
  return (long long)(y + s.hy) * s.pitch + (x + s.px);
}

// Macroscopic state of f(t+1)'s cells as the FP32-storage step leaves it:
// planes n, T, U^0, U^x, U^y, n - n_ref, T - T_ref, eps ([kMacroPlanes][ncell]).
constexpr int kMacroPlanes = 8;

template <typename S>
struct StepArgs {
  Scalars s;
  const S* fin;          // f*(t) (or g*)
  S* fout;               // f*(t+1)
  const S* tau_field;    // per-cell tau, row-major [ny][nx] (tau_mode 1)
  unsigned long long* status;   // count of non-physical cell updates
  float* macro = nullptr;       // optional macroscopic-state output (FP32 storage)
};

template <typename S>
struct MomentArgs {
  Scalars s;
  const S* fin;
  int gather;            // 1: stream first (fields of S f*), 0: fields of fin itself
  double* out;           // [14][ncell] (row-major cells): n ux uy T eps N0 Nx Ny T00 T0x T0y Txx Txy Tyy
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

// Macroscopic state of one cell (Sec. 6.2 steps 2-4).  FP64 mode fills the
// double members; the FP32-storage path also fills the float members used by
// the FP32 equilibrium (dn = n - n_ref and dT = T - T_ref carry FP64 accuracy).
struct Macro {
  double eps, U0, Ux, Uy, n, T;
  float fU0, fUx, fUy, fn, fT, fdn, fdT, feps;
  bool ok;
};

}  // namespace rlbm
