// bgk_internal.h - structures shared by the host runtime and the kernels of
// libbgk.so (not part of the public ABI; see include/bgk.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bgk {

constexpr int kMaxNv = 4096;   // velocities per cell handled by one CTA
constexpr int kFaces = 4;
enum { XLO = 0, XHI = 1, YLO = 2, YHI = 3 };
enum { BC_INFLOW = 0, BC_DIFFUSE = 1, BC_SPECULAR = 2 };
enum { PREC_F64 = 0, PREC_F32 = 1, PREC_BF16 = 2 };  // as bgk_precision

// Error bits written by kernels into the solver's device flag.
enum { ERR_MOMENT = 1, ERR_EFFECTIVE = 2, ERR_TIMEOUT = 4 };

// Effective-parameter iteration (Sec. 2.1, remark on exact conservation):
// p <- p + (q - D(p)) until an update is below kEffTol, at most kEffMaxIt
// updates; a run that ends above kEffFail is a failure.
constexpr double kEffTol = 1e-13;
constexpr int kEffMaxIt = 20;
constexpr double kEffFail = 1e-9;
// The GPU evaluates the Gaussians once per cell and moves them to a nearby
// parameter point to first order; beyond this relative distance it
// re-evaluates (the neglected second-order terms stay below 1e-15).
constexpr double kLinMax = 1e-8;

// Scalar description of one problem, passed by value to every kernel.
struct Params {
  int dim, nx, ny, nvx, nvy, nv;
  int tile;  // spatial cells per CTA of the step kernel (1, 2, 4 or 8)
  int mgl;   // reduced precisions: groups of 4 velocities per lane (2, 4 or 6)
  int conservative, relax_exact;
  int bc_kind[kFaces];
  double dt, dx, dy, dcx, dcy, dv;
  double x0, vx_min, vy_min;
  double omega;
  double bc_state[kFaces][4];  // n, ux, uy, theta
};

// Per-velocity tables built once on the device (build_tables).
struct Tables {
  const double* cx;       // [nvx] velocity-cell centres
  const double* cy;       // [nvy] (dim 1: one entry, 0)
  const double* cy2;      // [nvy] c_y^2 (stored right after cy)
  const double4_32a* coef;    // [nv] (a0, ax, ay, |c|^2): streaming weights, 2D
                          //      (w_near, w_far, 0, c_x^2): 1D
  const int* shift;       // [nv] 1D integer Courant shift [C] (0 in 2D)
  const double2* cxy;     // [nv] (c_x, c_y) per velocity
  const int* vinfo;       // [nv] jx | jy << 12 | (sgn c_x + 1) << 24 | (sgn c_y + 1) << 26
  const double2* ghost;   // [kFaces][nv] inflow Maxwellian, or the unit-density
                          //   wall Maxwellian for diffuse faces
  const double* emitted;  // [kFaces] sum_{c_n>0} c_n G_W(n=1) dv (diffuse)
};

// FP32 tables of the reduced-precision step (bgk_mixed.cu).
struct MixedTables {
  const float4* coef;       // [nv] (ax, ay, c_x, c_y): flux-form streaming weights
  const int* vinfo;         // [nv] as Tables::vinfo
  const float* cx;          // [nvx]
  const float* cy;          // [nvy]
  const float* ax;          // [nvx] 2D flux-form weight |c_x| dt / dx per column (= coef.x)
  const float* ay;          // [nvy] |c_y| dt / dy per row (= coef.y)
  const float2* ghost;      // [kFaces][nv] FP32 boundary Maxwellians
  const float2* mabs;       // [nv] absolute Maxwellian (n = 1, U = 0, theta = 1) in FP32
  const double* mabs_sums;  // [4] FP64 sums of mabs: g, c_x g, c_y g, |c|^2 g + h
  const float2* mabs_ff;    // [4] the same sums as float-float pairs
  const double* emitted;    // [kFaces] sum_{c_n>0} c_n ghost_g dv of the FP32 ghosts
  const int* shift;         // [nv] 1D integer Courant shift (as Tables::shift)
  unsigned* step_ctr;       // [2] steps taken: the kernel of buffer parity p reads word p and
                            //   writes word 1 - p (the BF16 dither varies with it)
};

// Launchers (bgk_step.cu, bgk_aux.cu, bgk_mixed.cu).  All enqueue on `stream`.
// One FP64 step fin -> fout; mom[cell] receives the moments (n, ux, uy,
// theta) of the post-streaming state, par[cell] (when not null) the
// effective Maxwellian parameters the relaxation used.
cudaError_t launch_step_f64(const Params& P, const Tables& T, const double2* fin, double2* fout,
                            double4_32a* mom, int* err, cudaStream_t stream, double4_32a* par = nullptr);
cudaError_t launch_build_tables(const Params& P, double* cx, double* cy, double4_32a* coef, int* shift,
                                double2* cxy, int* vinfo, double2* ghost, double* emitted,
                                cudaStream_t stream);
size_t step_f64_smem_bytes(const Params& P, int tile);
cudaError_t prepare_step_f64(const Params& P);
cudaError_t launch_init_step(const Params& P, double2* f, double x_split, const double left[4],
                             const double right[4], cudaStream_t stream);
cudaError_t launch_init_uniform(const Params& P, double2* f, const double state[4],
                                const double2* xi, double amplitude, cudaStream_t stream);
cudaError_t launch_moments(const Params& P, const Tables& T, const double2* f, double4_32a* mom,
                           cudaStream_t stream);
cudaError_t launch_wall_fluxes(const Params& P, const Tables& T, const double2* f, int face,
                               double4_32a* out, cudaStream_t stream);
cudaError_t launch_build_mixed_tables(const Params& P, const Tables& T, const MixedTables& M,
                                      cudaStream_t stream);
size_t step_mixed_smem_bytes(const Params& P, int tile, int prec);
int mixed_groups_per_lane(const Params& P, int tile);
// Persistent batch (bgk_mixed.cu): one kernel advances many FP32
// instances by several steps, a grid barrier between steps.
enum {
  PK_2D_G1_M2 = 0, PK_2D_G1_M4, PK_2D_G2_M2, PK_2D_G2_M4, PK_2D_G4_M2, PK_2D_G4_M4, PK_2D_G8_M2,
  PK_1D_K1, PK_1D_K2, PK_1D_K4, PK_KINDS
};
struct PInstance {
  Params P;
  MixedTables M;
  const void* f_even;  // input of even steps (output of odd steps)
  void* f_odd;         // output of even steps
  float2* msum;
  int* err;
  int kind;            // PK_*
  int unit0, units;    // first work unit, work units per step
  int pad;
};
struct GridBarrier {
  unsigned int count;
  unsigned int gen;
};
// Kind of an FP32 instance for the persistent kernel (-1: not supported).
int persistent_kind(const Params& P);
int persistent_units(const Params& P, int kind);
size_t persistent_smem(const Params& P);
// Resident CTAs of the persistent kernel for dynamic shared memory smem.
cudaError_t persistent_grid(size_t smem, int* grid);
constexpr int kMaxPersistInstances = 144;
static_assert(sizeof(PInstance) * kMaxPersistInstances <= 60 * 1024, "persistent descriptors exceed constant memory");
// Copy ninst descriptors (device memory) to the kernel's constant array.
cudaError_t upload_persistent(const PInstance* d_inst, int ninst, cudaStream_t stream);
cudaError_t launch_persistent(int ninst, int total_units, int nsteps, GridBarrier* bar, int* gerr,
                              long long spin_limit, int grid, size_t smem, cudaStream_t stream);

// Full 3D velocity grid, one spatial dimension (bgk_step3v.cu).
struct Params3v {
  int nx, nvx, nvy, nvz, nv;
  int conservative, relax_exact;
  double x0, dx, dt, dv, omega;
  double dc[3], vmin[3];
};
struct Tables3v {
  const double* c[3];    // [nvx], [nvy], [nvz] velocity-cell centres
  const double* c2;      // [nv] |c|^2
  const int* shift;      // [nvx] [C], C = c_x dt/dx, toward zero
  const int* upwind;     // [nvx] +1 for C > 0, else -1
  const double* rem;     // [nvx] |C - [C]|
  const double* ghost;   // [2][nv] inflow Maxwellians at XLO, XHI
};
struct Inflow3v {
  double s[2][5];  // (n, ux, uy, uz, theta)
};
cudaError_t launch_tables3v(const Params3v& P, double* c0, double* c1, double* c2, double* cc, int* shift,
                            int* upwind, double* rem, double* ghost, const Inflow3v& inflow, cudaStream_t stream);
cudaError_t launch_init3v(const Params3v& P, const Tables3v& T, double x_split, const Inflow3v& lr, double* f,
                          cudaStream_t stream);
cudaError_t launch_step3v(const Params3v& P, const Tables3v& T, const double* fin, double* fout, double* mom,
                          int* err, cudaStream_t stream);
cudaError_t launch_moments3v(const Params3v& P, const Tables3v& T, const double* f, double* mom,
                             cudaStream_t stream);

// Reverse pass of the lid shear (bgk_adjoint.cu).
cudaError_t launch_adj_lid_table(const Params& P, const Tables& T, double2* dghost, double* demit,
                                 cudaStream_t stream);
cudaError_t launch_adj_seed(const Params& P, const Tables& T, const double2* f, double2* lam,
                            const double2* dghost, double demit, double* Jk, double* duw, cudaStream_t stream);
cudaError_t launch_adj_step(const Params& P, const Tables& T, const double2* fn1,
                            const double4_32a* qn, const double4_32a* pn, const double2* lam_in, int tilde,
                            int collide, double2* out, const double2* dghost, double demit, double* dlnl,
                            double* duw, cudaStream_t stream);
cudaError_t launch_msum_moments(const Params& P, int prec, const MixedTables& M, const float2* msum,
                                double4_32a* mom, cudaStream_t stream);
cudaError_t prepare_step_mixed(const Params& P, int prec);
// True when tile 1 runs the pipelined kernel with at least 3 groups of 4
// velocities per streaming thread (FP32 state, 2D).
bool mixed_pipe_preferred(const Params& P);
cudaError_t launch_step_mixed(const Params& P, int prec, const MixedTables& M, const void* fin, void* fout,
                              double4_32a* mom, int* err, cudaStream_t stream, int parity);
cudaError_t launch_to_f64(const Params& P, int prec, const MixedTables& M, const void* f, double2* out,
                          cudaStream_t stream);
cudaError_t launch_from_f64(const Params& P, int prec, const MixedTables& M, const double2* in, void* f,
                            cudaStream_t stream);

}  // namespace bgk
