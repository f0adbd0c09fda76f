/*
 * bgk_oracle.h - plain FP64 CPU oracle of the BGK phase-space step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link,
 * load or call this code; only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg do.  It shares no header, helper, table or
 * constant with the CUDA library: every formula here is written out again
 * from the paper (Frezzotti, Ghiroldi, Gibelli, "Solving Kinetic Equations on
 * GPUs I: Model Kinetic Equations"), section and equation cited per function.
 *
 * Units (Sec. 4.1, normalisation): velocity c = v / sqrt(2 R T0), temperature
 * theta = T / T0, density n / n0, x in mean free paths, t in 1/nu0.  The
 * collision frequency of Eq. (frequency) with the power-law viscosity of
 * Eq. (viscosity) is then nu = n * theta^(1 - omega).
 *
 * The velocity space is reduced (Chu reduction, cited at the end of Sec. 4.1
 * and in Sec. 6): for a 1D flow the state per (cell, c_x) is
 *   g = int f dc_y dc_z,  h = int (c_y^2 + c_z^2) f dc_y dc_z,
 * for a 2D flow the state per (cell, c_x, c_y) is
 *   g = int f dc_z,       h = int c_z^2 f dc_z.
 *
 * Storage of the oracle's own state: two arrays g[cell][v], h[cell][v] with
 * cell = iy * nx + ix and v = jy * nvx + jx (jx fastest).
 */
#ifndef BGK_ORACLE_H
#define BGK_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_BC_INFLOW = 0, ORC_BC_DIFFUSE = 1, ORC_BC_SPECULAR = 2 };
enum { ORC_XLO = 0, ORC_XHI = 1, ORC_YLO = 2, ORC_YHI = 3 };

typedef struct {
  int dim;                 /* 1 or 2 spatial dimensions */
  int nx, ny;              /* cells; ny = 1 when dim = 1 */
  double x0, lx, y0, ly;   /* domain [x0, x0+lx] x [y0, y0+ly] */
  int nvx, nvy;            /* velocity cells; nvy = 1 when dim = 1 */
  double vx_min, vx_max, vy_min, vy_max;
  double omega;            /* viscosity exponent: nu = n theta^(1-omega) */
  double dt;               /* time step */
  int conservative;        /* 1: effective Maxwellian parameters (Sec. 2.1) */
  int relax_exact;         /* 1: Eq. (relaxation); 0: explicit Euler */
  int bc_kind[4];          /* per face xlo, xhi, ylo, yhi: ORC_BC_* */
  double bc_state[4][4];   /* per face: n, ux, uy, theta (inflow state, or
                              wall velocity and temperature; n unused) */
} orc_config;

/* Grid helpers (Sec. 2.1: cell-centred phase-space grid). */
int orc_nv(const orc_config* c);
int orc_ncell(const orc_config* c);
double orc_cx(const orc_config* c, int jx);
double orc_cy(const orc_config* c, int jy);
double orc_dv(const orc_config* c);
double orc_dt_from_cfl(const orc_config* c, double cfl);

/* Eq. (Maxw) reduced over the unresolved velocity components. */
void orc_maxwellian(const orc_config* c, const double p[4], double* G, double* H);

/* Eq. (macroscopic): moments (n, ux, uy, theta) of one cell's (g, h). */
void orc_moments(const orc_config* c, const double* g, const double* h, double out[4]);

/* Effective Maxwellian parameters whose discrete moments equal q (Sec. 2.1,
 * the remark on exact conservation).  Returns iterations used, or -1 if the
 * iteration failed to converge or left the admissible set. */
int orc_effective_params(const orc_config* c, const double q[4], double p_out[4]);

/* Rankine-Hugoniot states, Eq. (RH): up/down = (n, u, 0, theta). */
void orc_rankine_hugoniot(double mach, double gamma, double up[4], double down[4]);

/* Initial states. */
void orc_init_step(const orc_config* c, double x_split, const double left[4],
                   const double right[4], double* g, double* h);
void orc_init_uniform(const orc_config* c, const double s[4], const double* xi,
                      double amp, double* g, double* h);

/* Free-streaming sub-step, Eq. (upwind) with the integer shift of Eq. (exact)
 * and the boundary values of Eqs. (bc_shock) and (bc_cavity).  Returns 0, or
 * -1 if a diffuse wall sees zero incident flux. */
int orc_stream(const orc_config* c, const double* g, const double* h,
               double* gt, double* ht);

/* Collision sub-step, Eq. (relaxation) (or its Euler form) applied in place;
 * writes the moments of the pre-relaxation state per cell into mom[cell][4]
 * when mom is not NULL.  Returns 0, or -1 on a non-physical moment. */
int orc_relax(const orc_config* c, double* g, double* h, double* mom);

/* Full step(s): stream then relax.  mom (may be NULL) holds the moments of
 * the last step's post-streaming state.  Returns 0 or -1. */
int orc_step(const orc_config* c, double* g, double* h, long nsteps, double* mom);

/* Wall fluxes across one face for every face cell (length nx or ny):
 * mass = sum c_n F dV, shear = sum c_t c_n F dV, normal = sum c_n^2 F dV,
 * energy = sum c_n (|c|^2 F_g + F_h) dV, where c_n is the velocity component
 * along the inward normal, c_t the tangential one (c_x on y faces, c_y on x
 * faces), and F is the cell's own value for particles moving into the wall
 * and the boundary value for particles leaving it. */
int orc_wall_fluxes(const orc_config* c, const double* g, const double* h, int face,
                    double* mass, double* shear, double* normal, double* energy);

/* Threads used by the OpenMP loops over cells (1 when built without it). */
int orc_threads(void);
/* Threads of the OpenMP loops from now on (n > 0). */
void orc_set_threads(int n);

/* Objective of the adjoint: the lid-integrated shear J = sum over the cells
 * of face YHI of dx * tau_k, tau_k the shear flux of orc_wall_fluxes (the
 * drag of Sec. 5.2 up to its normalisation). */
double orc_lid_shear(const orc_config* c, const double* g, const double* h);

/* Reverse pass of nsteps split steps (2D, exact relaxation) from (g0, h0):
 * out = {J, dJ/d ln L, dJ/dU_W} and dJ/dg0, dJ/dh0 (same layout as g, h).
 * L scales the domain and, through the Courant rule, the time step together
 * (Kn = 1/L for the cavity); U_W is the x velocity of face YHI.  The
 * effective-parameter map p(q) is linearised by the identity (its Jacobian
 * differs from it by the quadrature residual).  Stores every state.
 * Returns 0, or -1 on an unsupported configuration or a failed step. */
int orc_adjoint_lid_shear(const orc_config* c, const double* g0, const double* h0, long nsteps,
                          double* dg0, double* dh0, double out[3]);

#ifdef __cplusplus
}
#endif
#endif
