/*
 * bgk_oracle3v.h - plain FP64 CPU oracle of the BGK step on a full
 * three-dimensional velocity grid, one spatial dimension (the normal shock
 * of Sec. 4.1 as the paper computed it: the Chu reduction is not made, so
 * the state per spatial cell is f on N_vx x N_vy x N_vz velocity cells).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link,
 * load or call this code; only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg do.  It shares no header, helper, table or
 * constant with the CUDA library.
 *
 * Units as in bgk_oracle.h: c = v / sqrt(2 R T0), theta = T / T0, density
 * n / n0, x in mean free paths, t in 1/nu0, nu = n theta^(1 - omega).
 *
 * Storage: f[cell][v], v = (jz * nvy + jy) * nvx + jx (jx fastest).
 * Moments per cell: (n, ux, uy, uz, theta).
 */
#ifndef BGK_ORACLE3V_H
#define BGK_ORACLE3V_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int nx;                   /* spatial cells on [x0, x0 + lx] */
  double x0, lx;
  int nvx, nvy, nvz;        /* velocity cells per component */
  double vmin[3], vmax[3];  /* velocity box per component */
  double omega;             /* nu = n theta^(1-omega) */
  double dt;                /* time step */
  int conservative;         /* 1: effective Maxwellian parameters (Sec. 2.1) */
  int relax_exact;          /* 1: Eq. (relaxation); 0: explicit Euler */
  double inflow[2][5];      /* left and right inflow states (n, ux, uy, uz, theta) */
} orc3_config;

int orc3_nv(const orc3_config* c);
double orc3_c(const orc3_config* c, int axis, int j); /* cell centre of component axis */
double orc3_dv(const orc3_config* c);                  /* velocity-cell volume */
double orc3_dt_from_cfl(const orc3_config* c, double cfl);

/* Eq. (Maxw): Phi = n (pi theta)^(-3/2) exp(-|c - U|^2 / theta) at every
 * velocity cell, p = (n, ux, uy, uz, theta). */
void orc3_maxwellian(const orc3_config* c, const double p[5], double* phi);

/* Eq. (macroscopic) by midpoint quadrature: out = (n, ux, uy, uz, theta). */
void orc3_moments(const orc3_config* c, const double* f, double out[5]);

/* Effective parameters whose discrete moments equal q (Sec. 2.1 remark).
 * Returns iterations used or -1. */
int orc3_effective_params(const orc3_config* c, const double q[5], double p_out[5]);

/* Initial step profile: Maxwellian of left for x < x_split, right beyond. */
void orc3_init_step(const orc3_config* c, double x_split, const double left[5], const double right[5],
                    double* f);

/* Free streaming along x: integer shift of Eq. (exact) and the upwind
 * remainder of Eq. (upwind); cells beyond the ends take the inflow
 * Maxwellians. */
void orc3_stream(const orc3_config* c, const double* f, double* ft);

/* Relaxation (Eq. relaxation or Euler) in place; mom (may be NULL) gets the
 * moments of the pre-relaxation state, 5 per cell.  Returns 0 or -1. */
int orc3_relax(const orc3_config* c, double* f, double* mom);

/* nsteps steps; mom of the last step as in orc3_relax.  Returns 0 or -1. */
int orc3_step(const orc3_config* c, double* f, long nsteps, double* mom);

#ifdef __cplusplus
}
#endif
#endif
