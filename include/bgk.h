/*
 * bgk.h - C ABI of libbgk.so, a GB300 (sm_103a) solver for the BGK model
 * kinetic equation on a regular phase-space grid.
 *
 * The method is the split step of Frezzotti, Ghiroldi, Gibelli, "Solving
 * Kinetic Equations on GPUs I: Model Kinetic Equations", Sec. 2.1: a
 * first-order upwind free-streaming sub-step (Eq. upwind, with the integer
 * Courant shift of Eq. exact), then per spatial cell the moments of
 * Eq. (macroscopic), the local Maxwellian of Eq. (Maxw) and the relaxation of
 * Eq. (relaxation).  Boundaries: the far-field inflow Maxwellians of
 * Eq. (bc_shock) and the diffuse (fully accommodating) walls of
 * Eq. (bc_cavity) with the zero-net-mass-flux wall density below it; specular
 * walls are added.
 *
 * Units (Sec. 4.1): velocity c = v / sqrt(2 R T0), temperature
 * theta = T / T0, density n / n0, lengths in mean free paths, time in
 * 1 / nu0.  The collision frequency of Eqs. (frequency) and (viscosity) is
 * nu = n * theta^(1 - omega).
 *
 * Velocity space is reduced by integrating out the components the flow does
 * not depend on (the reduction cited at the end of Sec. 4.1 and in Sec. 6):
 *   dim 1: g(x, c_x) = int f dc_y dc_z,  h = int (c_y^2 + c_z^2) f dc_y dc_z
 *   dim 2: g(x, y, c_x, c_y) = int f dc_z,  h = int c_z^2 f dc_z
 * One "point" of the phase space is one (cell, velocity) pair; it holds g
 * and h.
 *
 * STATE LAYOUT (the layout of every state buffer crossing this ABI):
 *   double f[ny][nx][nvy][nvx][2], component 0 = g, 1 = h;
 *   cell = iy*nx + ix, velocity v = jy*nvx + jx (jx fastest);
 *   cell centres x = x0 + (ix + 1/2) lx/nx, c_x = vx_min + (jx + 1/2) dcx.
 * For dim 1, ny = nvy = 1.
 *
 * CONVENTIONS
 *  - Every function returns bgk_status; nothing throws or aborts across the
 *    ABI.  On failure bgk_last_error() describes the cause.
 *  - The library owns the device state buffers of a solver.  The caller owns
 *    every array passed in or out; "on_device" flags say whether a pointer is
 *    a device pointer (non-zero) or a host pointer (zero).
 *  - Work is enqueued on the stream given in bgk_config.cuda_stream (NULL is
 *    the legacy default stream).  bgk_step is asynchronous; bgk_moments,
 *    bgk_wall_fluxes, bgk_get_state and bgk_sync synchronise that stream and
 *    report numerical failures detected by the kernels (BGK_ERR_NUMERIC).
 *  - A solver is not thread-safe: one host thread and one stream per handle.
 *  - The library computes in the kernels it ships for sm_103a; there is no
 *    CPU fallback.  Without a usable GPU the calls fail with BGK_ERR_CUDA.
 */
#ifndef BGK_H
#define BGK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BGK_ABI_VERSION 1

#if defined(__GNUC__)
#define BGK_API __attribute__((visibility("default")))
#else
#define BGK_API
#endif

typedef enum {
  BGK_OK = 0,
  BGK_ERR_INVALID_ARG = 1, /* bad pointer, size or configuration value */
  BGK_ERR_UNSUPPORTED = 2, /* valid request this build does not implement */
  BGK_ERR_OOM = 3,         /* device or host allocation failed */
  BGK_ERR_CUDA = 4,        /* CUDA runtime error (no device, launch failure) */
  BGK_ERR_NUMERIC = 5,     /* a cell produced n <= 0, theta <= 0, a non-finite
                              moment, or the effective-parameter iteration
                              failed; the state is then not trustworthy */
  BGK_ERR_TIMEOUT = 6      /* a bounded wait inside a kernel ran out */
} bgk_status;

typedef enum {
  BGK_F64 = 0,     /* state stored and computed in FP64 */
  BGK_F32 = 1,     /* state stored and computed in FP32; per-cell moment sums
                      carried in float-float (about 48 bits), rounded once to
                      FP32 for the step and finished in FP64 by bgk_moments */
  BGK_BF16_DEV = 2 /* state stored as BF16 deviation from the absolute
                      Maxwellian (n = 1, U = 0, theta = 1), computed as for
                      BGK_F32 */
} bgk_precision;

typedef enum {
  BGK_BC_INFLOW = 0,  /* Eq. (bc_shock): Maxwellian (n, ux, uy, theta) enters */
  BGK_BC_DIFFUSE = 1, /* Eq. (bc_cavity): wall velocity (ux, uy), temperature
                         theta; n is ignored (n_W from zero net mass flux) */
  BGK_BC_SPECULAR = 2 /* mirror reflection; needs a velocity grid symmetric
                         about 0 in the wall-normal component */
} bgk_bc_kind;

typedef enum { BGK_FACE_XLO = 0, BGK_FACE_XHI = 1, BGK_FACE_YLO = 2, BGK_FACE_YHI = 3 } bgk_face;

typedef struct {
  int32_t kind; /* bgk_bc_kind */
  int32_t reserved;
  double n, ux, uy, theta;
} bgk_bc;

typedef struct {
  int32_t dim;          /* 1 or 2 spatial dimensions */
  int32_t nx, ny;       /* cells; ny must be 1 when dim = 1 */
  int32_t nvx, nvy;     /* velocity cells; nvy must be 1 when dim = 1 */
  int32_t conservative; /* 1: Maxwellian built from effective parameters whose
                           discrete moments equal the cell's (Sec. 2.1,
                           remark after Eq. exact): exact conservation */
  int32_t relax_exact;  /* 1: Eq. (relaxation); 0: f += dt nu (Phi - f) */
  int32_t precision;    /* bgk_precision */
  int32_t tile_cells;   /* spatial cells per CTA of the step kernel: 0 = chosen
                           by the library, else 1, 2, 4 or 8 (tuning knob; the
                           results do not depend on it beyond rounding: the
                           order of the per-cell sums and, in FP64, how the
                           per-cell Gaussian factors are formed; for 2D FP32 and
                           BF16 states, 1 runs the pipelined one-cell kernel
                           when its buffers fit, with the one-cell block's
                           results) */
  int32_t reserved0;    /* must be 0 */
  double x0, lx;        /* domain [x0, x0 + lx] */
  double y0, ly;        /* domain [y0, y0 + ly] (dim 2) */
  double vx_min, vx_max;
  double vy_min, vy_max; /* dim 2 */
  double omega;         /* viscosity exponent: nu = n theta^(1 - omega) */
  double dt;            /* time step; 0 = derive from cfl */
  double cfl;           /* dim 1: max|c_x| dt/dx; dim 2: (max|c_x|/dx +
                           max|c_y|/dy) dt */
  bgk_bc bc[4];         /* per face, indexed by bgk_face (dim 1: XLO, XHI) */
  void* cuda_stream;    /* cudaStream_t; NULL = legacy default stream */
} bgk_config;

typedef struct {
  double dt, dx, dy, dcx, dcy, dv; /* dv = velocity-cell volume (reduced) */
  double max_courant;              /* dim 1: max|C|; dim 2: max(|Cx|+|Cy|) */
  int64_t ncell, nv;               /* spatial cells, velocities per cell */
  int64_t state_doubles;           /* ncell * nv * 2 */
  int64_t steps_done;              /* steps enqueued since the last init */
  int64_t device_bytes;            /* device memory held by the solver */
  int32_t precision;
  int32_t tile_cells;              /* cells per CTA the step kernel uses */
} bgk_info;

typedef struct bgk_solver bgk_solver;

/* The problem statement of Sec. 2.1 (phase-space grid, time step) with the
 * boundary conditions of Sec. 4.1 (Eq. bc_shock) or Sec. 5.1 (Eq. bc_cavity).
 * Validate cfg (all checks happen before any CUDA call), build the grids and
 * boundary tables on the current CUDA device, and allocate two state buffers
 * (ping-pong) plus per-cell moment storage.  The state is zero until an
 * init or set_state call.  *out receives the handle (NULL on failure).
 * Errors: INVALID_ARG (bad value), UNSUPPORTED (e.g. 2D Courant number above
 * 1, more than 4096 velocities per cell, walls with |C| > 1), OOM, CUDA. */
BGK_API bgk_status bgk_create(const bgk_config* cfg, bgk_solver** out);

/* Free everything the solver holds (synchronises its stream first).
 * NULL is accepted and ignored. */
BGK_API bgk_status bgk_destroy(bgk_solver* s);

/* Derived grid values and bookkeeping. */
BGK_API bgk_status bgk_get_info(const bgk_solver* s, bgk_info* out);

/* Initial step profile (Sec. 4.1, initial condition of the shock problem):
 * cells with x < x_split get the Maxwellian of left = (n, ux, uy, theta),
 * the others that of right.  Enqueued on the stream; resets steps_done and
 * the numerical-error flag. */
BGK_API bgk_status bgk_init_maxwellian_step(bgk_solver* s, double x_split, const double left[4],
                                    const double right[4]);

/* Uniform Maxwellian of state = (n, ux, uy, theta), multiplied point by point
 * by (1 + amplitude * xi) with xi in the state layout (ncell*nv*2 doubles,
 * host or device per xi_on_device; NULL = no perturbation).  Used for the
 * cavity's perturbed rest state. */
BGK_API bgk_status bgk_init_uniform(bgk_solver* s, const double state[4], const double* xi,
                            int xi_on_device, double amplitude);

/* Copy a state (STATE LAYOUT, ncell*nv*2 doubles) in or out.  get_state
 * synchronises the stream. */
BGK_API bgk_status bgk_set_state(bgk_solver* s, const double* f, int on_device);
BGK_API bgk_status bgk_get_state(bgk_solver* s, double* f, int on_device);

/* Enqueue nsteps time steps of the split scheme of Sec. 2.1: free streaming
 * by Eq. (upwind) (with the integer shift of Eq. (exact) in 1D), the moments
 * of Eq. (macroscopic), the Maxwellian of Eq. (Maxw) and the relaxation of
 * Eq. (relaxation); each step is one fused kernel, and batches of steps
 * replay a captured CUDA graph.
 * Asynchronous.  nsteps = 0 is a no-op; negative is INVALID_ARG. */
BGK_API bgk_status bgk_step(bgk_solver* s, int64_t nsteps);

/* Per-cell moments mom[cell][4] = (n, ux, uy, theta) of Eq. (macroscopic).
 * which = 0: of the current state; which = 1: of the post-streaming state of
 * the last step (the values the relaxation used).  Synchronises. */
BGK_API bgk_status bgk_moments(bgk_solver* s, int which, double* mom, int on_device);

/* Fluxes through one face for each of its cells (the wall fluxes behind the
 * drag of Sec. 5.2, "Results and discussion"; ny cells for x faces, nx
 * for y faces; 1 for dim 1), out[k][4] = (mass, shear, normal momentum,
 * energy) = sum over velocities of (c_n, c_t c_n, c_n^2, c_n (|c|^2 g + h))
 * times the crossing value times dv, where c_n is along the inward normal
 * (+x at XLO, -x at XHI, +y at YLO, -y at YHI) and c_t is c_y on x faces,
 * c_x on y faces.  The crossing value is the wall-adjacent cell's state for
 * c_n < 0 and the boundary value the next step would use for c_n > 0.
 * Synchronises. */
BGK_API bgk_status bgk_wall_fluxes(bgk_solver* s, int face, double* out, int on_device);

/* Lid-integrated shear of the current state (2D only): *J = dx * sum over
 * the face cells k of the lid (face YHI) of the shear flux tau_k of
 * bgk_wall_fluxes, summed in the order k = 0 .. nx-1.  This is the drag of
 * Sec. 5.2, "Results and discussion", before its normalisation, and the
 * objective that bgk_adjoint_lid_shear differentiates.  J is a host pointer.
 * Synchronises.  Errors: INVALID_ARG (null pointer), UNSUPPORTED (dim 1). */
BGK_API bgk_status bgk_lid_shear(bgk_solver* s, double* J);

/* Wait for the solver's stream; report a kernel-detected numerical failure. */
BGK_API bgk_status bgk_sync(bgk_solver* s);

/* Rankine-Hugoniot states of Eq. (RH) for upstream Mach number mach with the
 * normalisation of Sec. 4.1 (n- = 1, theta- = 1, u- = mach*sqrt(gamma/2)):
 * up and down receive (n, u, 0, theta).  Host-only arithmetic. */
BGK_API bgk_status bgk_rankine_hugoniot(double mach, double gamma, double up[4], double down[4]);

/* Message of the calling thread's last failure ("" if none); never NULL. */
BGK_API const char* bgk_last_error(void);

/* Name of a status code; never NULL. */
BGK_API const char* bgk_status_string(bgk_status st);

/* BGK_ABI_VERSION of the loaded library. */
BGK_API int bgk_abi_version(void);

/* ---- batches and tuning ------------------------------------------------ */

typedef struct bgk_batch bgk_batch;

/* Many independent problems (any mix of sizes, velocity grids, dimensions
 * and precisions) stepped together.  Each instance is a full solver created
 * from cfgs[i] with its cuda_stream replaced by `cuda_stream`;
 * bgk_batch_step advances every instance by nsteps with one CUDA-graph
 * launch per 64 steps in which each instance is an independent branch, so
 * the GPU runs the instances' step kernels concurrently.  Instances are
 * reached with bgk_batch_solver for init, state, moments and wall fluxes
 * (the batch owns them: do not bgk_destroy them).  On failure *out is NULL
 * and the message names the failing instance. */
BGK_API bgk_status bgk_batch_create(const bgk_config* cfgs, int count, void* cuda_stream,
                                    bgk_batch** out);
BGK_API bgk_status bgk_batch_solver(bgk_batch* b, int index, bgk_solver** out);
BGK_API bgk_status bgk_batch_step(bgk_batch* b, int64_t nsteps);
/* Wait for the batch stream; BGK_ERR_NUMERIC if any instance failed,
 * BGK_ERR_TIMEOUT if a persistent launch gave up at a grid barrier. */
BGK_API bgk_status bgk_batch_sync(bgk_batch* b);
BGK_API bgk_status bgk_batch_destroy(bgk_batch* b);

/* Persistent mode (enable = 1): each bgk_batch_step call becomes one
 * cooperative launch, captured in a CUDA graph, in which every CTA of a
 * resident grid walks the work units (blocks of cells of every instance)
 * of one step, then waits at a grid barrier before the next step.  FP32
 * instances only (2D and 1D); a 2D instance whose tile needs more than 16
 * velocities per lane gets a smaller tile.  A barrier wait longer than
 * timeout_s seconds records a timeout and ends the launch, leaving the
 * steps incomplete: bgk_batch_sync then returns BGK_ERR_TIMEOUT (and clears
 * the record).  enable = 0 returns to one graph branch per instance.
 * Results equal those of the instances stepped alone with the same tiles. */
BGK_API bgk_status bgk_batch_set_persistent(bgk_batch* b, int enable, double timeout_s);

/* Autotuner: time trial_steps steps for every admissible tile_cells value
 * (cells per CTA: 1, 2, 4, 8) on the solver's own state, which is saved
 * before and restored after the trials (the call allocates one temporary
 * state copy), and keep the fastest.  *tile_out (may be NULL) receives it.
 * Results do not depend on the tile beyond rounding order.  Synchronises. */
BGK_API bgk_status bgk_autotune(bgk_solver* s, int trial_steps, int* tile_out);
/* Tune every instance of a batch; instances with the same shape (dim, cells,
 * velocity grid, precision) share one tuning run. */
BGK_API bgk_status bgk_batch_autotune(bgk_batch* b, int trial_steps);

/* ---- full three-dimensional velocity grid ------------------------------- */

/* The normal shock of Sec. 4.1 as the paper computed it: one spatial
 * dimension and the full velocity grid (the Chu reduction is not made), so
 * the state of a spatial cell is f on N_vx x N_vy x N_vz velocity cells.
 * Streaming along x uses the integer shift of Eq. (exact) and the upwind
 * remainder of Eq. (upwind) (any Courant number); the relaxation target is
 * the 3D Maxwellian of Eq. (Maxw), Phi = n (pi theta)^(-3/2)
 * exp(-|c - U|^2 / theta), from effective parameters when conservative.
 * FP64 only.
 *
 * STATE LAYOUT (3V): f[cell][v], v = (jz * nvy + jy) * nvx + jx, one double
 * per point; c_a = vmin[a] + (j_a + 1/2) (vmax[a] - vmin[a]) / nv_a.
 * Moments: (n, ux, uy, uz, theta) per cell. */
typedef struct {
  int32_t nx;                 /* spatial cells on [x0, x0 + lx] */
  int32_t nvx, nvy, nvz;      /* velocity cells per component (each 1..256) */
  int32_t conservative;       /* 1: effective Maxwellian parameters (exact conservation) */
  int32_t relax_exact;        /* 1: Eq. (relaxation); 0: f += dt nu (Phi - f) */
  int32_t reserved0, reserved1; /* must be 0 */
  double x0, lx;
  double vmin[3], vmax[3];    /* velocity box per component */
  double omega;               /* nu = n theta^(1 - omega) */
  double dt;                  /* time step; 0 = derive from cfl */
  double cfl;                 /* max|c_x| dt / dx when dt = 0 */
  double inflow[2][5];        /* (n, ux, uy, uz, theta) held beyond XLO and XHI */
  void* cuda_stream;          /* cudaStream_t; NULL = legacy default stream */
} bgk3v_config;

typedef struct {
  double dt, dx, dv;          /* dv = dc_x dc_y dc_z */
  double max_courant;         /* max |c_x| dt / dx (may exceed 1) */
  int64_t ncell, nv;
  int64_t steps_done;
  int64_t device_bytes;
} bgk3v_info;

typedef struct bgk3v_solver bgk3v_solver;

/* Validate (before any CUDA call), build tables, allocate two state buffers.
 * Errors: INVALID_ARG, UNSUPPORTED (more than 2^24 velocities per cell or a
 * component above 256 cells), OOM, CUDA. */
BGK_API bgk_status bgk3v_create(const bgk3v_config* cfg, bgk3v_solver** out);
BGK_API bgk_status bgk3v_destroy(bgk3v_solver* s);
BGK_API bgk_status bgk3v_get_info(const bgk3v_solver* s, bgk3v_info* out);
/* Step profile: Maxwellian of left (n, ux, uy, uz, theta) for x < x_split,
 * of right beyond.  Enqueued; resets steps_done and the error flag. */
BGK_API bgk_status bgk3v_init_step(bgk3v_solver* s, double x_split, const double left[5], const double right[5]);
/* Copy a state (STATE LAYOUT (3V), ncell*nv doubles) in or out; get
 * synchronises. */
BGK_API bgk_status bgk3v_set_state(bgk3v_solver* s, const double* f, int on_device);
BGK_API bgk_status bgk3v_get_state(bgk3v_solver* s, double* f, int on_device);
/* Enqueue nsteps steps (one kernel per step).  Asynchronous. */
BGK_API bgk_status bgk3v_step(bgk3v_solver* s, int64_t nsteps);
/* mom[cell][5] = (n, ux, uy, uz, theta): which = 0 of the current state,
 * which = 1 of the last step's post-streaming state.  Synchronises. */
BGK_API bgk_status bgk3v_moments(bgk3v_solver* s, int which, double* mom, int on_device);
/* Wait for the stream; BGK_ERR_NUMERIC if a cell failed. */
BGK_API bgk_status bgk3v_sync(bgk3v_solver* s);

/* ---- adjoint -------------------------------------------------------------- */

/* Gradient of the lid-integrated shear by the adjoint of the split step.
 * J = sum over the cells of face YHI of dx * tau_k, tau_k the shear flux of
 * bgk_wall_fluxes (the drag of Sec. 5.2 up to its normalisation), after
 * nsteps steps from the solver's current state f0.  Runs the steps forward
 * (saving the state every checkpoint_every steps), then backward segment by
 * segment, recomputing each segment's states from its checkpoint: device
 * memory of about (nsteps / checkpoint_every + checkpoint_every + 3) states;
 * checkpoint_every = 0 takes ceil(sqrt(nsteps)), which minimises it (about
 * 92 states instead of 123 for 2000 steps at 100).  The checkpoint spacing does
 * not change the results.
 * Outputs: out = {J, dJ/d ln L, dJ/dU_W}, where L scales the domain and,
 * through the Courant rule, the time step together (Kn = 1/L for the
 * cavity: dJ/dKn = -(dJ/d ln L)/Kn) and U_W is the lid's (YHI) x speed;
 * dJ_df0 (STATE LAYOUT, host or device per on_device; may be NULL) receives
 * dJ/df0.  The map from moments to effective Maxwellian parameters is
 * linearised by the identity (exact up to the quadrature residual of the
 * velocity grid).  On return the solver holds the state after nsteps.
 * Requires dim 2, BGK_F64, exact relaxation, a diffuse lid (YHI) and a time
 * step derived from cfl (dt = 0).  Synchronises; allocates its buffers. */
BGK_API bgk_status bgk_adjoint_lid_shear(bgk_solver* s, int64_t nsteps, int checkpoint_every, double* dJ_df0,
                                         int on_device, double out[3]);

/* One time step with no device allocation (the paper has no counterpart:
 * this entry point exists for callers, not for the method).
 *
 * Some callers cannot let a library call cudaMalloc: code that runs under a
 * fixed device-memory budget handed out by its host framework, or code on a
 * path where cudaMalloc's implicit device-wide synchronisation is not
 * allowed.  For them this call advances one state by one step using only
 * the buffers the caller passes plus a fixed 384 KiB scratch array compiled
 * into the library (held on every GPU that loads libbgk.so until the process
 * exits).  The scratch holds the per-velocity tables (about 120 bytes per
 * velocity) and the error flag, which limits this call to about 3260
 * velocities per cell (48x48 fits, 64x64 does not); larger configurations
 * get BGK_ERR_UNSUPPORTED before any GPU work.
 *
 *   cfg     as for bgk_create (validated the same way; tile_cells honoured);
 *           the work goes to cfg->cuda_stream
 *   f_in    device pointer, state at time level n (STATE LAYOUT), read
 *           only, 16-byte aligned
 *   f_out   device pointer, state at level n+1 (same size, must not overlap
 *           f_in), 16-byte aligned
 *   mom_out device pointer, ncell*4 doubles, 32-byte aligned: moments
 *           (n, ux, uy, theta) of the post-streaming state, as
 *           bgk_moments(which = 1)
 * The library cannot see the buffers' sizes: the caller guarantees them.
 * A misaligned pointer gets BGK_ERR_INVALID_ARG before any GPU work.
 * The result equals bgk_set_state(f_in) + bgk_step(1) on a solver made from
 * cfg.  The call synchronises cfg->cuda_stream before returning and reports
 * BGK_ERR_NUMERIC like bgk_sync.  The first call on a device looks up the
 * scratch array's device address for that device; make that first call
 * before any stream capture begins.  All calls share the one scratch array and it
 * keeps the last call's contents (the error flag is cleared and the tables
 * rebuilt on every call): calls whose work overlaps on the GPU, from several
 * threads or streams, race and must be serialised by the caller. */
BGK_API bgk_status bgk_step_noalloc(const bgk_config* cfg, const double* f_in, double* f_out,
                                    double* mom_out);

#ifdef __cplusplus
}
#endif
#endif /* BGK_H */
