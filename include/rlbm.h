/*
 * rlbm.h -- C ABI of the GB300-native relativistic lattice Boltzmann (RLBM) step.
 *
 * The method is the one of Gabbana, Simeoni, Succi, Tripiccione,
 * "Relativistic Lattice Boltzmann Methods: Theory and Applications"
 * (arXiv:1909.04502).  One time step is the fused per-cell update of
 * Sec. 6.2: stream (Eq. discrete-rbe), moments N^a and T^ab (step 1),
 * Landau-frame eigen-solve (step 2, Sec. 4), n = U.N (step 3), T from the
 * EOS (step 4, Eq. eos-ddim), polynomial equilibrium (step 5,
 * Eq. mj-discrete-feq), local tau (step 7) and Anderson-Witting relaxation
 * (step 8).
 *
 * Units: lattice units c = k_B = T0 = 1, Delta t = 1 (Sec. 5.3, Sec. 6.1).
 * Metric eta = diag(1, -1, -1).  Fields are FP64, row-major [y][x]
 * (index y*nx + x).  Velocities are 3-velocities u = U^i/U^0 (fraction of c).
 *
 * State convention.  The library holds the post-collision populations
 * f*(t).  rlbm_step advances t -> t+1: f(t+1) = S f*(t) (streaming),
 * f*(t+1) = C(f(t+1)) (collision).  rlbm_init sets f(0) = f*(0) =
 * f^eq(n, u, T) (Sec. 6.2, first paragraph: collision of an equilibrium is
 * the identity).  rlbm_moments reports the Landau-frame fields of the
 * streamed f(t), i.e. those computed in steps 1-4 at time t.
 *
 * Errors.  Every int-returning call returns RLBM_OK (0) or a negative
 * RLBM_ERR_* code; rlbm_last_error() gives a message.  Calls are asynchronous
 * on the handle's CUDA stream unless stated otherwise; device-side faults of
 * the physics (a cell without a timelike Landau eigenvector, n <= 0,
 * T <= 0, non-finite values) are recorded in a device status word and
 * reported by rlbm_sync_status().
 *
 * Ownership.  Host arrays passed in are caller-owned and read or written
 * before the call returns (the call synchronises the stream when it copies
 * from or to host memory).  Device pointers passed in are borrowed for the
 * duration of the call.  The handle owns every buffer it allocates;
 * ownership never transfers.
 */
#ifndef RLBM_H
#define RLBM_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
  RLBM_OK = 0,
  RLBM_ERR_INVALID_ARG = -1,   /* bad parameter or size                        */
  RLBM_ERR_UNSUPPORTED = -2,   /* valid but not implemented                    */
  RLBM_ERR_CUDA = -3,          /* a CUDA runtime call failed                   */
  RLBM_ERR_NONPHYSICAL = -4,   /* a cell had no physical Landau frame          */
  RLBM_ERR_TIMEOUT = -5,       /* a bounded device-side wait gave up           */
  RLBM_ERR_OOM = -6,           /* device allocation failed                     */
  RLBM_ERR_QUADRATURE = -7     /* no non-negative quadrature found             */
};

/* Quadratures (App. H; Sec. 5.3). */
enum {
  RLBM_QUAD_MASSLESS = 0,      /* m~ = 0: App. H (2+1)-d table of the requested order
                                  (order 2: Q = 28, order 3: Q = 44)             */
  RLBM_QUAD_MASSIVE = 1,       /* m~ > 0: Eq. discrete-momentum-vectors on an FS stencil,
                                  weights from Eq. mj-orthogonal-conditions,
                                  v0 by the line search of Sec. 5.3              */
  RLBM_QUAD_CUSTOM = 2         /* caller table: custom_table / custom_Q           */
};

/* Boundaries in x (y is always periodic): periodic; free-flow ends (pulls
 * from beyond an end read the end cell); equilibrium walls at the first and
 * last column (pulls as free-flow; after each collision the wall cells hold
 * the equilibrium at zero flow speed with their own n and T -- the no-slip
 * walls of the paper's Poiseuille validation, Sec. 8.1). */
enum { RLBM_BC_PERIODIC = 0, RLBM_BC_FREEFLOW_X = 1, RLBM_BC_EQWALL_X = 2 };
enum { RLBM_FP64 = 0, RLBM_FP32_STORE = 1 };   /* storage/collision precision    */
enum { RLBM_ONLATTICE = 0, RLBM_BILINEAR = 1 };
/* Step kernels (rlbm_set_step_kernel).  Both compute the same update (Sec.
 * 6.2); they differ in how the pull reads f*: DIRECT loads every tap from
 * global memory, one cell per thread; TMA_32X8 / TMA_32X4 are persistent
 * kernels that stage each tile's source rectangles of all populations in
 * shared memory with tensor copies, two tiles ahead of the arithmetic. */
enum { RLBM_KERNEL_AUTO = 0, RLBM_KERNEL_DIRECT = 1, RLBM_KERNEL_TMA_32X8 = 2, RLBM_KERNEL_TMA_32X4 = 3 };
enum { RLBM_TAU_CONST = 0, RLBM_TAU_FIELD = 1, RLBM_TAU_ETA_OVER_S = 2 };

typedef struct rlbm_params {
  int d;              /* spatial dimensions: 2, or 1 for a one-dimensional problem run
                         on the d = 2 stencil over an nx x 1 grid (ny must be 1; the
                         gas stays two-dimensional: EOS and eta/s -> tau of d = 2).
                         The native (1+1)-d gas is rlbm1_*, d = 3 is rlbm3_*     */
  double m;           /* rest mass m~ = m c^2/(k_B T0); zeta = m~/T~ (Sec. 5.2)      */
  int order;          /* expansion order N of Eq. mj-discrete-feq: 2 or 3           */
  int quadrature;     /* RLBM_QUAD_*                                                 */
  const int* groups;  /* RLBM_QUAD_MASSIVE: n_groups generator vectors (x, y) of the
                         FS stencil (Sec. 5.3); NULL selects the built-in choice   */
  int n_groups;
  double v0;          /* RLBM_QUAD_MASSIVE: v0 of Eq. discrete-momentum-vectors;
                         0 = search for a non-negative solution                    */
  const double* custom_table; /* RLBM_QUAD_CUSTOM: custom_Q rows (nx, ny, p0, px, py, w) */
  int custom_Q;
  int tau_mode;       /* RLBM_TAU_*                                                  */
  double tau;         /* RLBM_TAU_CONST: relaxation time in units of Delta t        */
  double eta_over_s;  /* RLBM_TAU_ETA_OVER_S: tau = (eta/s)(d+2) kappa / T (step 7)  */
  double kappa;       /*   kappa = hbar/(k_B T0 dt)                                  */
  int boundary;       /* RLBM_BC_*                                                   */
  int nx, ny;         /* grid size in cells                                          */
  int precision;      /* RLBM_FP64 | RLBM_FP32_STORE: FP32 populations g = f - f_ref
                         with an FP32 Landau solve whose eigenvalue gets one Newton
                         correction from a float-float (about 48-bit) residual; at
                         order 3 with m~ >= 6 on an orbit-symmetric stencil (App. H
                         columns A-D, the Sec. 6.3 stencil) the equilibrium moments
                         are float-float and H dM a compensated sum as well, since
                         FP32 moments lose the 1e-5 bar there                      */
  int stream_mode;    /* RLBM_ONLATTICE | RLBM_BILINEAR                              */
  double lambda;      /* RLBM_BILINEAR: displacement per step = lambda * v_i cells
                         (lambda = 1/dx in units of c dt; the on-lattice value is
                         ||n_i|| for m~ = 0 and 1/v0 for m~ > 0)                     */
  double n_ref, T_ref;/* reference state of the shifted FP32 storage (default 1, 1) */
  void* stream;       /* cudaStream_t all work is issued on (NULL = legacy default) */
  double gx, gy;      /* gravity-like acceleration g (lattice units): Minkowski force
                         K = (g.p, p^0 g) added by forcing scheme B (Sec. 4.4),
                         F_i = (m/T) f^eq_i (U^0 g.v_i - g.U) per step; acts on
                         massive particles only (m~ > 0); default 0             */
  double wall_T[2];   /* RLBM_BC_EQWALL_X: temperature of the first / last column's
                         equilibrium (the heated plates of the paper's thermal-
                         conductivity runs, Sec. 7.2); 0 = the cell's own T       */
} rlbm_params;

typedef struct rlbm_handle rlbm_handle;

/* Fill *p with defaults: d = 2, m = 0, order 2, massless quadrature, tau 1,
 * periodic, FP32 storage, on-lattice, n_ref = T_ref = 1. */
void rlbm_default_params(rlbm_params* p);

/* Build the stencil, quadrature and equilibrium tables (Sec. 5.2-5.3, App. F-H)
 * on the host in FP64 and allocate two population buffers, a tau buffer and a
 * status word on the current device.  Synchronous. */
int rlbm_create(const rlbm_params* p, rlbm_handle** out);

/* Host-only planning: build the quadrature and equilibrium tables for *p
 * exactly as rlbm_create does, without touching a GPU.  Outputs (all
 * nullable except Q and K): nvec 2*Q ints, p 3*Q, w Q, H Q*K (row-major,
 * f^eq_i = sum_k H_ik M_k with M the Maxwell-Juttner moments of the basis
 * p0^e px^a py^b, e in {0,1}, e + a + b <= N, in the order 1 | p0 px py |
 * p0px p0py pxpx pxpy pypy | p0pxpx p0pxpy p0pypy pxpxpx pxpxpy pxpypy
 * pypypy; at N = 3 the members with p0 are shifted, (p0 - m) px^a py^b), v0
 * the massive parameter.  Arrays must hold 72 rows (72*16 for H). */
int rlbm_plan(const rlbm_params* p, int* Q, int* K, int* nvec, double* pmom, double* w,
              double* H, double* v0);

/* Release everything the handle owns.  Synchronises its stream first. */
void rlbm_destroy(rlbm_handle* h);

/* Set f(0) = f*(0) = f^eq(n, u, T) (Sec. 6.2).  n, ux, uy, T: nx*ny FP64 each,
 * host (on_device = 0) or device (on_device = 1) pointers.  Resets t to 0. */
int rlbm_init(rlbm_handle* h, const double* n, const double* ux, const double* uy,
              const double* T, int on_device);

/* Set the per-cell relaxation time (tau_mode RLBM_TAU_FIELD), nx*ny FP64. */
int rlbm_set_tau_field(rlbm_handle* h, const double* tau, int on_device);

/* Advance nsteps time steps (asynchronous on the handle's stream). */
int rlbm_step(rlbm_handle* h, int nsteps);

/* Choose the step kernel (RLBM_KERNEL_*); the TMA-staged kernels need FP32
 * storage, the massless Q = 28 order-2 stencil and padded rows of at least
 * 36 elements (RLBM_ERR_UNSUPPORTED otherwise).  AUTO (the default) is
 * DIRECT, the faster kernel at every grid size measured on GB300.  The kernels evaluate the same
 * expressions in the same order, so their results are bitwise identical.
 * No counterpart in the paper. */
int rlbm_set_step_kernel(rlbm_handle* h, int kernel);
/* The kernel rlbm_step launches for this handle (RLBM_KERNEL_DIRECT,
 * _TMA_32X8 or _TMA_32X4), or RLBM_ERR_INVALID_ARG. */
int rlbm_step_kernel(const rlbm_handle* h);

/* Landau-frame fields of f(t) (steps 1-4 of Sec. 6.2).  Every output is
 * nullable; n, ux, uy, T, eps: nx*ny FP64; Nab: 3*nx*ny (N^0, N^x, N^y
 * planes); Tab: 6*nx*ny (T^00, T^0x, T^0y, T^xx, T^xy, T^yy planes).
 * With on_device = 0 the call copies to host and synchronises. */
int rlbm_moments(rlbm_handle* h, double* n, double* ux, double* uy, double* T,
                 double* eps, double* Nab, double* Tab, int on_device);

/* Post-collision populations f*(t) as FP64 [Q][ny][nx] (unshifted), and
 * their replacement (checkpoint / restart).  set_populations keeps t. */
int rlbm_get_populations(rlbm_handle* h, double* f, int on_device);
int rlbm_set_populations(rlbm_handle* h, const double* f, int on_device);

/* Stencil actually used: Q, integer vectors n_i (2Q, x then y per row),
 * momenta p_i^mu (3Q), weights w_i (Q).  Every pointer but Q is nullable. */
int rlbm_stencil(const rlbm_handle* h, int* Q, int* nvec, double* p, double* w);

/* Number of completed time steps. */
long long rlbm_time(const rlbm_handle* h);

/* Synchronise the stream and report device-side status: RLBM_OK,
 * RLBM_ERR_NONPHYSICAL (*count, nullable, gets the number of flagged cell
 * updates since the last call) or RLBM_ERR_CUDA.  Clears the status. */
int rlbm_sync_status(rlbm_handle* h, long long* count);

/* Change the stream subsequent calls are issued on. */
int rlbm_set_stream(rlbm_handle* h, void* stream);

/* Device pointers of the current f*(t) buffer and of the previous one
 * (borrowed; valid until the next rlbm_step / rlbm_destroy), element size
 * (4 or 8 bytes), population-plane stride in elements, and the padded
 * layout {pitch, hx, hy, px} (nullable, 4 ints).  Plane i starts at element
 * i * plane; interior cell (x, y) is at (y + hy) * pitch + (x + px); the hx
 * columns left and right and the hy rows above and below hold copies of
 * cells (periodic images, or the first / last column for free-flow ends) so
 * that streaming reads need no wrap-around.  FP32-storage handles hold
 * g = f - f_ref (f_ref,i = f^eq_i(n_ref, 0, T_ref)); FP64 handles hold f. */
int rlbm_buffers(rlbm_handle* h, void** cur, void** prev, int* elem_size, long long* plane,
                 int* layout);

/* Allocation-free variant of the fused step, for callers that cannot
 * allocate device memory: code that runs inside another runtime which owns
 * the device memory (a plugin whose buffers come from the host application's
 * pool), code that must not allocate while it records or replays work, or
 * code that cannot afford the device-wide synchronisation of cudaMalloc /
 * cudaFree.  The paper has no counterpart (it describes no API).
 *
 * f_a holds f*(t) on entry, halo included, in the storage layout of a
 * handle created with the same parameters (rlbm_buffers describes it; a
 * copy of such a handle's buffer is a valid start).  f_b is a second buffer
 * of the same size.  FP32 storage holds f - f_ref (pass n_ref = 0 to store
 * f).  The call runs nsteps steps,
 * alternating f_a -> f_b -> f_a ...: the result is in f_b when nsteps is
 * odd and in f_a when it is even.  tau_field (device, storage precision,
 * nx*ny) is read when p->tau_mode is RLBM_TAU_FIELD.  Work is issued on
 * p->stream.  If counts is non-NULL it receives, per step, the number of
 * non-physical cell updates; the call then synchronises the stream and
 * returns RLBM_ERR_NONPHYSICAL if any count is non-zero.
 *
 * Memory.  The call allocates no device memory: its only scratch is a
 * file-scope device array of 1024 eight-byte counters (one per step), which
 * every GPU that loads the library holds until the process exits.  nsteps
 * above 1024 is rejected with RLBM_ERR_INVALID_ARG.  The first call on a
 * device looks the array up (cudaGetSymbolAddress) for that device; make it
 * before any stream capture.  All calls share the array and each clears its
 * counters first, so calls that overlap on the GPU race on it.  The host
 * side caches the tables of each parameter set in host memory.  Errors are
 * reported through rlbm_last_error(NULL). */
int rlbm_step_noalloc(const rlbm_params* p, void* f_a, void* f_b, const void* tau_field, int nsteps,
                      long long* counts);

/* ------------------------------------------------------------------------
 * Batched simulations: many independent grids (different sizes, tau and
 * stencils; FP32 storage, order 2, built-in stencils, constant or eta/s tau)
 * advanced together from one captured CUDA graph per call, under one of two
 * schedules: persistent cooperative kernels, one per stencil kind present
 * (the kinds run one after another, each over all its instances' tiles, with
 * a grid-wide barrier between steps), or independent chains of each
 * instance's single-grid step kernels (each instance waits only on its own
 * previous step; the chains run concurrently).  Not in the paper: it serves the paper's
 * calibration of tau against transport coefficients (Sec. 7), which runs many
 * independent simulations.  Each instance stays an ordinary handle
 * (rlbm_batch_handle) for init / moments / populations; the batched step is
 * bitwise identical to rlbm_step on every instance.
 * ------------------------------------------------------------------------ */
typedef struct rlbm_batch rlbm_batch;

/* Create count handles from params[0..count) (all on params[0].stream) and
 * the batch machinery.  RLBM_ERR_UNSUPPORTED for configurations outside the
 * batched kernel (FP64, order 3, tau fields, stencils other than the massless
 * Q = 28 (on-lattice or bilinear) and the built-in massive Q = 25, 29, 33,
 * each in orbit order with an exactly symmetric equilibrium matrix;
 * two instances of one stencil size must share the same stencil). */
int rlbm_batch_create(const rlbm_params* params, int count, rlbm_batch** out);
void rlbm_batch_destroy(rlbm_batch* b);
int rlbm_batch_size(const rlbm_batch* b);
/* The i-th instance (borrowed; owned by the batch). */
rlbm_handle* rlbm_batch_handle(rlbm_batch* b, int i);
/* Advance every instance by nsteps (one graph launch; asynchronous). */
int rlbm_batch_step(rlbm_batch* b, int nsteps);
/* Schedule: tile_shape 0 or 1 runs the persistent kernels with 32 x 8 or
 * 32 x 4 cells per block and grid = persistent blocks (at most the
 * co-resident limit; a kind with fewer tiles runs with one block per tile);
 * tile_shape 2 runs the per-instance chains (grid ignored). */
int rlbm_batch_config(rlbm_batch* b, int tile_shape, int grid);
/* Autotuner: times trial_steps steps for each tile shape and five grid
 * sizes (1, 3/4, 1/2, 1/3 and 1/4 of the co-resident limit) and for the
 * per-instance chains (tile_shape 2, grid 0), and keeps the fastest.  It
 * advances every instance by 23 * trial_steps steps; call it before
 * rlbm_init of the instances.
 * Outputs are nullable. */
int rlbm_batch_tune(rlbm_batch* b, int trial_steps, int* tile_shape, int* grid, float* ms_per_step);
/* Current configuration (grid 0 for the per-instance chains), co-resident
 * limits {32x8, 32x4} (the smallest over the kinds present) and tile count. */
int rlbm_batch_info(const rlbm_batch* b, int* tile_shape, int* grid, int* grid_max, long long* total_tiles);
/* Iteration limit of the bounded grid-barrier wait (default 2^24 polls of
 * about 64 ns).  A wait that runs out sets the batch error flag; every block
 * leaves the kernel and rlbm_batch_sync_status returns RLBM_ERR_TIMEOUT. */
int rlbm_batch_set_spin_limit(rlbm_batch* b, long long limit);
/* Synchronise; report timeouts (RLBM_ERR_TIMEOUT, then clears them) or the
 * first instance error; *nonphysical (nullable) gets the summed count. */
int rlbm_batch_sync_status(rlbm_batch* b, long long* nonphysical);
const char* rlbm_batch_last_error(const rlbm_batch* b);

/* ------------------------------------------------------------------------
 * Adjoint (reverse-mode gradient) of a run of the fused step.  Not in the
 * paper: it serves the calibration of kinetic parameters against transport
 * coefficients (Sec. 7) by gradients.  Loss on the run's final fields:
 *   L = 1/2 sum_x |u(x, T) - u_target(x)|^2,  u = U^i/U^0 of f(T)
 * (the fields rlbm_moments reports after T steps).  Gradients with respect
 * to the per-cell relaxation time tau(x) (constant in time) and the initial
 * velocity u0(x).  The backward pass recomputes the forward states segment
 * by segment from checkpoints taken every checkpoint_every steps.
 * Periodic boundaries, order 2, constant or per-cell tau, no external force;
 * both precisions.
 * ------------------------------------------------------------------------ */
typedef struct rlbm_adjoint rlbm_adjoint;

/* Allocate checkpoints (ceil(nsteps / checkpoint_every) population buffers),
 * two segments of checkpoint_every + 1 buffers (the backward pass recomputes
 * one segment on a second, lowest-priority stream while it runs the adjoint
 * steps of the other), two adjoint buffers and per-cell accumulators for a
 * run of nsteps steps of handle h (borrowed). */
int rlbm_adjoint_create(rlbm_handle* h, int nsteps, int checkpoint_every, rlbm_adjoint** out);
void rlbm_adjoint_destroy(rlbm_adjoint* A);
/* Forward pass: rlbm_init(n, u, T) then nsteps steps, saving checkpoints.
 * Leaves the handle at t = nsteps. */
int rlbm_adjoint_forward(rlbm_adjoint* A, const double* n, const double* ux, const double* uy, const double* T,
                         int on_device);
/* Backward pass for the targets (nx*ny each): loss (1 value), dL/dtau,
 * dL/dux0, dL/duy0 (nx*ny each; all outputs nullable), on the host
 * (out_on_device = 0) or the device.  Synchronous. */
int rlbm_adjoint_backward(rlbm_adjoint* A, const double* ux_target, const double* uy_target, int on_device,
                          double* loss, double* grad_tau, double* grad_ux0, double* grad_uy0, int out_on_device);
const char* rlbm_adjoint_last_error(const rlbm_adjoint* A);

/* One adjoint step, the building block of rlbm_adjoint_backward: the
 * vector-Jacobian product of one collide-and-stream step (Eq. discrete-rbe,
 * Sec. 6.2) with f(t) = S x(t-1) and f(t+1) = S C(f(t)):
 *   a_out = dL/df(t) = C'(f(t))^T S^T a_next,   a_next = dL/df(t+1),
 * and grad_tau[cell] += dL/dtau(cell) of this step.  x_prev = x(t-1), the
 * post-collision populations the forward step started from; x_prev, a_next
 * and a_out are device buffers in the handle's padded layout and storage
 * type (rlbm_buffers), halo images included; a_out gets its halo images
 * written.  grad_tau: device FP64 [ny][nx], accumulated.  All pointers are
 * borrowed; asynchronous on the handle's stream.  Periodic boundaries,
 * order 2, constant or per-cell tau, no external force (RLBM_ERR_UNSUPPORTED
 * otherwise).
 * No counterpart in the paper. */
int rlbm_adjoint_step(rlbm_handle* h, const void* x_prev, const void* a_next, void* a_out, double* grad_tau);

/* The FP32 <-> FP64 conversions of the FP32-storage kernels, element by
 * element on device arrays (asynchronous on `stream`): out_d[i] = in_f[i]
 * converted exactly to FP64 (i < nf), out_f[i] = in_d[i] rounded to FP32
 * (i < nd).  The kernels do these on the integer pipe from the IEEE-754 bit
 * layouts (a hardware conversion costs about an FP64 multiply on this part);
 * they differ from the hardware's in three documented ways: FP64 -> FP32
 * rounds a value exactly halfway between two floats away from zero (the
 * hardware rounds it to even), results below the smallest normal float
 * become signed zero, and FP32 denormal inputs convert to signed zero.
 * Infinities and NaNs keep their class.  No counterpart in the paper: a
 * check of the library's own arithmetic. */
int rlbm_convert_f32_f64(const float* in_f, double* out_d, int nf, const double* in_d, float* out_f, int nd,
                         void* stream);

/* Message of the last error on this handle (or of the last failed
 * rlbm_create when h is NULL).  Never NULL. */
const char* rlbm_last_error(const rlbm_handle* h);

/* Static description of an error code. */
const char* rlbm_strerror(int code);

/* ------------------------------------------------------------------------
 * (3+1) dimensions: massless particles, expansion orders 2 and 3 (Sec. 5-6
 * with d = 3).  Stencils and weights: App. H, "(3+1) dimensions".  Order 2
 * is read with the group (+-2, +-2, +-1) (the printed (+-2, +-1, +-1) does
 * not have the common length 3 of a massless stencil) and the weights shell
 * by shell (per shell the (2, 2, 1) group, then (3, 0, 0)): Q = 78.  Order 3
 * (v0 = 1/sqrt(41)) reads as printed, weights shell by shell: Q = 288.
 * On-lattice streaming, periodic in x, y and z, constant tau.
 * EOS eps = 3 n T.  Fields are row-major [z][y][x] arrays of nx*ny*nz doubles.
 * ------------------------------------------------------------------------ */
typedef struct rlbm3_handle rlbm3_handle;

/* Host-only: Q, K and the tables rlbm3_create builds for expansion order
 * `order` (2 or 3) -- stencil vectors nvec (3*Q ints), momenta p (4*Q),
 * weights w (Q), equilibrium matrix H (Q*K, row-major, f^eq_i = sum_k H_ik
 * M_k with M the MJ moments of the basis 1 | p0 px py pz | p0px p0py p0pz
 * pxpx pxpy pxpz pypy pypz pzpz, K = 14, and at order 3 further p0 (xx xy xz
 * yy yz zz) | xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz, K = 30); arrays
 * nullable, room for 80 rows (order 2) or 288 rows (order 3).
 * RLBM_ERR_INVALID_ARG for another order. */
int rlbm3_plan(int order, int* Q, int* K, int* nvec, double* p, double* w, double* H);

/* Tables on the host (double-double), two population buffers on the current
 * device; stream: cudaStream_t all work is issued on.  order: 2 (App. H
 * order-2 stencil, Q = 78, halo 3) or 3 (App. H order-3 stencil, v0 =
 * 1/sqrt(41), Q = 288, halo 6).  precision: RLBM_FP64 (f stored and collided
 * in FP64) or RLBM_FP32_STORE (g = f - f_ref stored and collided in FP32,
 * f_ref the equilibrium at n = T = 1 at rest; the Landau root is found in
 * FP32 and corrected by one Newton step whose residual, eigenvector, norm
 * nu^2, w = v.N and the numerator of n - 1 are evaluated in FP64; n, n - 1,
 * T - 1 and U are then FP32 quotients of those FP64 values).  Each side
 * at least the halo width (3, or 6 at order 3) and nx*ny*nz <= 2^28.
 * The steps evaluate the table in sign-orbit form (runs of sign variants
 * whose equilibrium rows differ only by the basis members' signs);
 * RLBM_ERR_QUADRATURE if that identity does not hold exactly (the built-in
 * tables satisfy it).  Synchronous. */
int rlbm3_create(int nx, int ny, int nz, double tau, int order, int precision, void* stream,
                 rlbm3_handle** out);
void rlbm3_destroy(rlbm3_handle* h);

/* Q, stencil vectors nvec (3*Q ints, nullable), momenta p (4*Q: p0, px, py,
 * pz; nullable), weights w (Q, nullable) in the library's population order. */
int rlbm3_stencil(const rlbm3_handle* h, int* Q, int* nvec, double* p, double* w);

/* f*(0) = f^eq(n, U(u), T) from host (on_device = 0: copied, then synchronous)
 * or device arrays (on_device = 1: borrowed, asynchronous). */
int rlbm3_init(rlbm3_handle* h, const double* n, const double* ux, const double* uy, const double* uz,
               const double* T, int on_device);

/* nsteps fused steps (pull, moments, Landau frame, equilibrium, relaxation),
 * asynchronous on the handle's stream. */
int rlbm3_step(rlbm3_handle* h, int nsteps);

/* Fields of the populations f(t) before the collision of step t (f*(t-1)
 * pulled; at t = 0 the initial equilibrium): out = [6][nz][ny][nx] doubles
 * (n, ux, uy, uz, T, eps; n is NaN where the cell has no Landau frame), host
 * (synchronous) or device (asynchronous). */
int rlbm3_moments(rlbm3_handle* h, double* out, int on_device);

/* Post-collision populations f*(t) (g + f_ref for FP32 storage), host array
 * [Q][nz][ny][nx] of doubles.  Synchronous. */
int rlbm3_get_populations(rlbm3_handle* h, double* f);

/* Synchronise; RLBM_ERR_NONPHYSICAL if cell updates were left unrelaxed since
 * the last call (their number in *count, nullable), else RLBM_OK. */
int rlbm3_sync_status(rlbm3_handle* h, long long* count);

/* Message of the last error on this handle (or of the last failed
 * rlbm3_create when h is NULL).  Never NULL. */
const char* rlbm3_last_error(const rlbm3_handle* h);

/* ------------------------------------------------------------------------
 * (1+1) dimensions: a one-dimensional massless gas on the App. H "(1+1)
 * dimensions" quadratures (Sec. 5-6 with d = 1).  Populations
 * p_{j,s} = p0_j (1, s), s = +-1, on the N shells of the order-N table
 * (order 4 read with its two printed columns exchanged: the printed weights
 * are the roots of L_4); each moves one cell per step in direction s.
 * Equilibrium: the massless limit of the order-N expansion (Sec. 5.2, Eq.
 * mj-expanded-1D-massless; the weight normalised with C = 1/(2 m K_1(m)),
 * whose constant member has no finite norm as m -> 0).  On these tables the
 * 2N populations and the 2N members (p0)^a sign(p^x)^b (a = 1..N, b = 0, 1)
 * of the limit basis form a square system that the quadrature integrates
 * exactly, so f^eq is the discrete distribution whose moments of those
 * members are the Maxwell-Juttner ones, n (a-1)! T^(a-1) {cosh, sinh}(a th)
 * with U = (cosh th, sinh th).  Landau frame of the 2 x 2 mixed tensor
 * (Sec. 4); EOS eps = P = n T (d = 1, m = 0).  FP64 storage computes in
 * FP64; FP32 storage (g = f - f_ref) computes in FP32 from differences to
 * the reference state, with compensated moment sums, and meets the 1e-5
 * parity bar up to order 4 (order 5: about 1.3e-5; use FP64 there).
 * A d = 2 stencil on an nx x 1 grid (rlbm_params.d = 1) is the other way to
 * run a one-dimensional problem: a two-dimensional gas with a 1-d flow.
 * Fields are arrays of nx doubles.
 * ------------------------------------------------------------------------ */
typedef struct rlbm1_handle rlbm1_handle;

/* Host-only tables for expansion order `order` (2 ... 5): Q = 2 order,
 * directions nvec (Q ints, +-1), momenta p (2Q: p0, px), weights w (Q; half
 * the printed per-direction value, the weight exp(-p0)/2 of dp/p0 spread
 * over both directions), H (Q x Q row-major, f^eq_i = sum_k H_ik M_k,
 * k = 2 (a - 1) + b).  Outputs but Q nullable. */
int rlbm1_plan(int order, int* Q, int* nvec, double* p, double* w, double* H);

/* nx cells; tau > 1/2 (units of Delta t); boundary RLBM_BC_PERIODIC,
 * RLBM_BC_FREEFLOW_X (pulls from beyond an end read the end cell) or
 * RLBM_BC_EQWALL_X (the end cells hold f^eq(n, rest, T_w) after each
 * collision, T_w = wall_T[0] / wall_T[1] or, where 0 or wall_T is NULL,
 * the cell's own T); precision RLBM_FP64 or RLBM_FP32_STORE (populations
 * stored as f - f_ref in FP32, f_ref the equilibrium of n = T = 1 at rest);
 * stream: the cudaStream_t work is issued on.  Allocates two population
 * buffers of 2 order (nx + 2) elements and field buffers.  Synchronous.
 * RLBM_ERR_QUADRATURE if the table lacks the direction symmetry the FP32
 * step uses (each pair's second H row the first with the odd members'
 * signs flipped; the built-in tables have it exactly). */
int rlbm1_create(int nx, int order, double tau, int boundary, const double* wall_T, int precision,
                 void* stream, rlbm1_handle** out);
void rlbm1_destroy(rlbm1_handle* h);

/* Q, directions (Q ints), momenta (2Q) and weights (Q); outputs but Q nullable. */
int rlbm1_stencil(const rlbm1_handle* h, int* Q, int* nvec, double* p, double* w);

/* f*(0) = f^eq(n, U(ux), T): nx doubles each, host (on_device = 0:
 * copied, synchronous) or device (borrowed, asynchronous). */
int rlbm1_init(rlbm1_handle* h, const double* n, const double* ux, const double* T, int on_device);

/* nsteps fused steps (pull, moments, Landau frame, equilibrium, relaxation),
 * asynchronous.  Cells without a Landau frame are left unrelaxed and
 * counted (rlbm1_sync_status). */
int rlbm1_step(rlbm1_handle* h, int nsteps);

/* Fields of f(t) (f*(t-1) streamed; at t = 0 the initial equilibrium):
 * out = [8][nx] doubles n, ux, T, eps, N^0, N^x, T^00, T^0x (n NaN without a
 * Landau frame), host (synchronous) or device (asynchronous). */
int rlbm1_moments(rlbm1_handle* h, double* out, int on_device);

/* Post-collision populations f*(t) (f_ref added back for FP32 storage),
 * host array [Q][nx] of doubles.  Synchronous. */
int rlbm1_get_populations(rlbm1_handle* h, double* f);

/* Synchronise; RLBM_ERR_NONPHYSICAL if cell updates were left unrelaxed
 * since the last call (their number in *count, nullable), else RLBM_OK. */
int rlbm1_sync_status(rlbm1_handle* h, long long* count);

/* Message of the last error on this handle (or of the last failed
 * rlbm1_create / rlbm1_plan when h is NULL).  Never NULL. */
const char* rlbm1_last_error(const rlbm1_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* RLBM_H */
