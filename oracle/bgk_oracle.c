/*
 * bgk_oracle.c - plain FP64 CPU oracle of the BGK phase-space step.
 *
 * TEST INFRASTRUCTURE ONLY (see bgk_oracle.h).  Written for a reader who
 * checks it against the paper by eye: naive loops, one formula per line, no
 * blocking or fusion.  The only liberty taken is that the Gaussian of
 * Eq. (Maxw) is evaluated as the product of its one-dimensional factors
 * (exp(a + b) = exp(a) exp(b)), which is the same function.
 *
 * Compile with -ffp-contract=off so that x86 and Arm give the same sums.
 */
#include "bgk_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static const double ORC_PI = 3.14159265358979323846;

/* Effective-parameter iteration (Sec. 2.1, exact-conservation remark):
 * stop once an update is below ORC_EFF_TOL (relative); give up after
 * ORC_EFF_MAXIT updates. */
#define ORC_EFF_TOL 1e-13
#define ORC_EFF_MAXIT 20
#define ORC_EFF_FAIL 1e-9

/* ------------------------------------------------------------------------ */
/* Grid (Sec. 2.1): N_x cells of width dx; velocity box split into equal     */
/* cells; values live at cell centres.                                       */
/* ------------------------------------------------------------------------ */
int orc_nv(const orc_config* c) { return c->nvx * (c->dim == 2 ? c->nvy : 1); }
int orc_ncell(const orc_config* c) { return c->nx * (c->dim == 2 ? c->ny : 1); }

static double orc_dcx(const orc_config* c) { return (c->vx_max - c->vx_min) / c->nvx; }
static double orc_dcy(const orc_config* c) { return (c->vy_max - c->vy_min) / c->nvy; }
static double orc_dx(const orc_config* c) { return c->lx / c->nx; }
static double orc_dy(const orc_config* c) { return c->ly / c->ny; }

double orc_cx(const orc_config* c, int jx) { return c->vx_min + (jx + 0.5) * orc_dcx(c); }
double orc_cy(const orc_config* c, int jy) {
  if (c->dim == 1) return 0.0;
  return c->vy_min + (jy + 0.5) * orc_dcy(c);
}
/* Volume of one velocity cell, Delta V of Sec. 2.1 (reduced dimensions). */
double orc_dv(const orc_config* c) {
  if (c->dim == 1) return orc_dcx(c);
  return orc_dcx(c) * orc_dcy(c);
}

static double orc_max_abs_cx(const orc_config* c) {
  double m = 0.0;
  for (int jx = 0; jx < c->nvx; ++jx) {
    double a = fabs(orc_cx(c, jx));
    if (a > m) m = a;
  }
  return m;
}
static double orc_max_abs_cy(const orc_config* c) {
  double m = 0.0;
  for (int jy = 0; jy < c->nvy; ++jy) {
    double a = fabs(orc_cy(c, jy));
    if (a > m) m = a;
  }
  return m;
}

/* Time step from a Courant number: 1D cfl = max|c_x| dt/dx; 2D (unsplit
 * donor cell) cfl = (max|c_x|/dx + max|c_y|/dy) dt. */
double orc_dt_from_cfl(const orc_config* c, double cfl) {
  if (c->dim == 1) return cfl * orc_dx(c) / orc_max_abs_cx(c);
  return cfl / (orc_max_abs_cx(c) / orc_dx(c) + orc_max_abs_cy(c) / orc_dy(c));
}

int orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* Eq. (Maxw) in normalised units:                                           */
/*   Phi = n (pi theta)^(-3/2) exp(-|c - U|^2 / theta).                      */
/* Integrated over the unresolved components (Chu reduction):                */
/*   1D: G = n (pi theta)^(-1/2) exp(-(c_x-U_x)^2/theta),  H = theta G       */
/*   2D: G = n (pi theta)^(-1) exp(-|c-U|^2/theta),        H = theta/2 G     */
/* (each unresolved component contributes int c^2 e^{-c^2/theta} dc /        */
/*  int e^{-c^2/theta} dc = theta/2 to H/G).                                 */
/* p = (n, ux, uy, theta).                                                   */
/* ------------------------------------------------------------------------ */
void orc_maxwellian(const orc_config* c, const double p[4], double* G, double* H) {
  const double n = p[0], ux = p[1], uy = p[2], th = p[3];
  if (c->dim == 1) {
    const double pref = n / sqrt(ORC_PI * th);
    for (int jx = 0; jx < c->nvx; ++jx) {
      const double d = orc_cx(c, jx) - ux;
      G[jx] = pref * exp(-d * d / th);
      H[jx] = th * G[jx];
    }
    return;
  }
  const double pref = n / (ORC_PI * th);
  for (int jy = 0; jy < c->nvy; ++jy) {
    const double dy = orc_cy(c, jy) - uy;
    const double ey = exp(-dy * dy / th);
    for (int jx = 0; jx < c->nvx; ++jx) {
      const double dx = orc_cx(c, jx) - ux;
      const double ex = exp(-dx * dx / th);
      const int j = jy * c->nvx + jx;
      G[j] = pref * ex * ey;
      H[j] = 0.5 * th * G[j];
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Eq. (macroscopic) by midpoint quadrature over the velocity cells:         */
/*   n = sum g dV,  n U = sum c g dV,                                        */
/*   (3/2) n theta = sum (|c - U|^2 g + h) dV                                */
/* evaluated as theta = (2/3) (E/n - |U|^2) with E = sum (|c|^2 g + h) dV.   */
/* ------------------------------------------------------------------------ */
void orc_moments(const orc_config* c, const double* g, const double* h, double out[4]) {
  const double dv = orc_dv(c);
  double s0 = 0.0, sx = 0.0, sy = 0.0, se = 0.0;
  for (int jy = 0; jy < (c->dim == 2 ? c->nvy : 1); ++jy) {
    const double cy = orc_cy(c, jy);
    for (int jx = 0; jx < c->nvx; ++jx) {
      const double cx = orc_cx(c, jx);
      const int j = jy * c->nvx + jx;
      s0 += g[j];
      sx += cx * g[j];
      sy += cy * g[j];
      se += (cx * cx + cy * cy) * g[j] + h[j];
    }
  }
  const double n = s0 * dv;
  const double ux = sx * dv / n;
  const double uy = sy * dv / n;
  const double e = se * dv;
  out[0] = n;
  out[1] = ux;
  out[2] = uy;
  out[3] = (2.0 / 3.0) * (e / n - (ux * ux + uy * uy));
}

/* ------------------------------------------------------------------------ */
/* Effective parameters (Sec. 2.1, remark after Eq. (exact)): find p such    */
/* that the moments of the DISCRETISED Maxwellian Phi(p) equal the target q. */
/* The map D(p) = moments(Phi(p)) is the identity up to the quadrature       */
/* error, so the iteration p <- p + (q - D(p)) contracts at the rate of that */
/* error (it is Newton's method with the Jacobian of the continuous map).    */
/* ------------------------------------------------------------------------ */
int orc_effective_params(const orc_config* c, const double q[4], double p_out[4]) {
  const int nv = orc_nv(c);
  double* G = (double*)malloc(sizeof(double) * nv);
  double* H = (double*)malloc(sizeof(double) * nv);
  double p[4] = {q[0], q[1], q[2], q[3]};
  int it = 0, ok = 0;
  double r = 0.0;
  for (it = 1; it <= ORC_EFF_MAXIT; ++it) {
    double d[4];
    orc_maxwellian(c, p, G, H);
    orc_moments(c, G, H, d);
    double delta[4];
    for (int k = 0; k < 4; ++k) delta[k] = q[k] - d[k];
    for (int k = 0; k < 4; ++k) p[k] += delta[k];
    const double vs = sqrt(q[3]);
    r = fabs(delta[0]) / q[0];
    if (fabs(delta[1]) / vs > r) r = fabs(delta[1]) / vs;
    if (fabs(delta[2]) / vs > r) r = fabs(delta[2]) / vs;
    if (fabs(delta[3]) / q[3] > r) r = fabs(delta[3]) / q[3];
    if (!(p[0] > 0.0) || !(p[3] > 0.0) || !isfinite(r)) break;
    if (r < ORC_EFF_TOL) {
      ok = 1;
      break;
    }
  }
  if (!ok && it > ORC_EFF_MAXIT && r < ORC_EFF_FAIL) {
    ok = 1; /* stalled at round-off level */
    it = ORC_EFF_MAXIT;
  }
  for (int k = 0; k < 4; ++k) p_out[k] = p[k];
  free(G);
  free(H);
  return ok ? it : -1;
}

/* ------------------------------------------------------------------------ */
/* Eq. (RH): V-/V+ = n+/n- = 4M^2/(M^2+3), T+/T- = (5M^2-1)(M^2+3)/(16M^2), */
/* with the upstream state n- = 1, T- = 1 (normalisation of Sec. 4.1) and   */
/* V- = M sqrt(gamma R T-) = M sqrt(gamma/2) in units of sqrt(2 R T-).       */
/* ------------------------------------------------------------------------ */
void orc_rankine_hugoniot(double mach, double gamma, double up[4], double down[4]) {
  const double m2 = mach * mach;
  const double ratio = 4.0 * m2 / (m2 + 3.0);
  const double tratio = (5.0 * m2 - 1.0) * (m2 + 3.0) / (16.0 * m2);
  up[0] = 1.0;
  up[1] = mach * sqrt(gamma / 2.0);
  up[2] = 0.0;
  up[3] = 1.0;
  down[0] = up[0] * ratio;
  down[1] = up[1] / ratio;
  down[2] = 0.0;
  down[3] = up[3] * tratio;
}

/* ------------------------------------------------------------------------ */
/* Initial states.                                                           */
/* Shock (Sec. 4.1): f = Phi- for x < 0 and Phi+ for x > 0 (split point is   */
/* a parameter).                                                             */
/* ------------------------------------------------------------------------ */
void orc_init_step(const orc_config* c, double x_split, const double left[4],
                   const double right[4], double* g, double* h) {
  const int nv = orc_nv(c);
  const double dx = orc_dx(c);
  for (int cell = 0; cell < orc_ncell(c); ++cell) {
    const int ix = cell % c->nx;
    const double x = c->x0 + (ix + 0.5) * dx;
    orc_maxwellian(c, x < x_split ? left : right, g + (size_t)cell * nv, h + (size_t)cell * nv);
  }
}

/* Uniform Maxwellian times (1 + amp xi), xi[(cell*nv + j)*2 + {0: g, 1: h}]. */
void orc_init_uniform(const orc_config* c, const double s[4], const double* xi,
                      double amp, double* g, double* h) {
  const int nv = orc_nv(c);
  for (int cell = 0; cell < orc_ncell(c); ++cell) {
    double* gc = g + (size_t)cell * nv;
    double* hc = h + (size_t)cell * nv;
    orc_maxwellian(c, s, gc, hc);
    if (xi == NULL) continue;
    for (int j = 0; j < nv; ++j) {
      gc[j] = gc[j] * (1.0 + amp * xi[((size_t)cell * nv + j) * 2 + 0]);
      hc[j] = hc[j] * (1.0 + amp * xi[((size_t)cell * nv + j) * 2 + 1]);
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Boundary values.                                                          */
/* Inward normals: xlo +x, xhi -x, ylo +y, yhi -y.  Particles with c_n > 0   */
/* leave the wall and take the boundary value; particles with c_n < 0 hit    */
/* the wall and carry the wall-adjacent cell's value.                        */
/* ------------------------------------------------------------------------ */
static double orc_cn(const orc_config* c, int face, int j) {
  const int jx = j % c->nvx, jy = j / c->nvx;
  switch (face) {
    case ORC_XLO: return orc_cx(c, jx);
    case ORC_XHI: return -orc_cx(c, jx);
    case ORC_YLO: return orc_cy(c, jy);
    default: return -orc_cy(c, jy);
  }
}
static double orc_ct(const orc_config* c, int face, int j) {
  const int jx = j % c->nvx, jy = j / c->nvx;
  return (face == ORC_XLO || face == ORC_XHI) ? orc_cy(c, jy) : orc_cx(c, jx);
}
static int orc_face_cells(const orc_config* c, int face) {
  return (face == ORC_XLO || face == ORC_XHI) ? (c->dim == 2 ? c->ny : 1) : c->nx;
}
/* Cell adjacent to face cell k of a face. */
static int orc_face_cell(const orc_config* c, int face, int k) {
  switch (face) {
    case ORC_XLO: return k * c->nx;
    case ORC_XHI: return k * c->nx + c->nx - 1;
    case ORC_YLO: return k;
    default: return (c->ny - 1) * c->nx + k;
  }
}
/* Velocity index with the normal component reversed (specular reflection). */
static int orc_reflect(const orc_config* c, int face, int j) {
  const int jx = j % c->nvx, jy = j / c->nvx;
  if (face == ORC_XLO || face == ORC_XHI) return jy * c->nvx + (c->nvx - 1 - jx);
  return (c->nvy - 1 - jy) * c->nvx + jx;
}

/* Boundary tables for one step.  For each face: the unit-density boundary  */
/* Maxwellian (inflow: the given state), and for diffuse walls the wall      */
/* density n_W per face cell from the zero-net-mass-flux condition below     */
/* Eq. (bc_cavity), written for the discrete velocity set:                   */
/*   n_W sum_{c_n>0} c_n G_W(n=1) dV = sum_{c_n<0} |c_n| g_cell dV.          */
typedef struct {
  double* G[4];
  double* H[4];
  double* nw[4];
} orc_bnd;

static int orc_faces(const orc_config* c) { return c->dim == 2 ? 4 : 2; }

static int orc_bnd_build(const orc_config* c, const double* g, orc_bnd* b) {
  const int nv = orc_nv(c);
  const double dv = orc_dv(c);
  memset(b, 0, sizeof(*b));
  for (int face = 0; face < orc_faces(c); ++face) {
    b->G[face] = (double*)malloc(sizeof(double) * nv);
    b->H[face] = (double*)malloc(sizeof(double) * nv);
    const double* s = c->bc_state[face];
    if (c->bc_kind[face] == ORC_BC_INFLOW) {
      orc_maxwellian(c, s, b->G[face], b->H[face]);
    } else if (c->bc_kind[face] == ORC_BC_DIFFUSE) {
      const double unit[4] = {1.0, s[1], s[2], s[3]};
      orc_maxwellian(c, unit, b->G[face], b->H[face]);
      const int nf = orc_face_cells(c, face);
      b->nw[face] = (double*)malloc(sizeof(double) * nf);
      double emitted = 0.0;
      for (int j = 0; j < nv; ++j) {
        const double cn = orc_cn(c, face, j);
        if (cn > 0.0) emitted += cn * b->G[face][j] * dv;
      }
      for (int k = 0; k < nf; ++k) {
        const double* gc = g + (size_t)orc_face_cell(c, face, k) * nv;
        double incident = 0.0;
        for (int j = 0; j < nv; ++j) {
          const double cn = orc_cn(c, face, j);
          if (cn < 0.0) incident += -cn * gc[j] * dv;
        }
        if (!(emitted > 0.0)) return -1;
        b->nw[face][k] = incident / emitted;
      }
    }
  }
  return 0;
}
static void orc_bnd_free(orc_bnd* b) {
  for (int face = 0; face < 4; ++face) {
    free(b->G[face]);
    free(b->H[face]);
    free(b->nw[face]);
  }
}

/* Value of (g, h) at velocity j just outside face cell k of a face. */
static void orc_ghost(const orc_config* c, const orc_bnd* b, const double* g, const double* h,
                      int face, int k, int j, double* go, double* ho) {
  const int nv = orc_nv(c);
  switch (c->bc_kind[face]) {
    case ORC_BC_INFLOW:
      *go = b->G[face][j];
      *ho = b->H[face][j];
      return;
    case ORC_BC_DIFFUSE:
      *go = b->nw[face][k] * b->G[face][j];
      *ho = b->nw[face][k] * b->H[face][j];
      return;
    default: {
      const size_t cell = (size_t)orc_face_cell(c, face, k);
      const int jr = orc_reflect(c, face, j);
      *go = g[cell * nv + jr];
      *ho = h[cell * nv + jr];
      return;
    }
  }
}

/* (g, h) of cell (ix, iy) at velocity j, or the boundary value when the     */
/* index lies outside the domain (any distance: used by the integer shift).  */
static void orc_fetch(const orc_config* c, const orc_bnd* b, const double* g, const double* h,
                      int ix, int iy, int j, double* go, double* ho) {
  const int nv = orc_nv(c);
  if (ix < 0) {
    orc_ghost(c, b, g, h, ORC_XLO, iy, j, go, ho);
  } else if (ix >= c->nx) {
    orc_ghost(c, b, g, h, ORC_XHI, iy, j, go, ho);
  } else if (iy < 0) {
    orc_ghost(c, b, g, h, ORC_YLO, ix, j, go, ho);
  } else if (iy >= (c->dim == 2 ? c->ny : 1)) {
    orc_ghost(c, b, g, h, ORC_YHI, ix, j, go, ho);
  } else {
    const size_t cell = (size_t)iy * c->nx + ix;
    *go = g[cell * nv + j];
    *ho = h[cell * nv + j];
  }
}

/* ------------------------------------------------------------------------ */
/* Free streaming, Eq. (freestreaming), by the first-order upwind scheme of  */
/* Eq. (upwind).  1D: for Courant numbers C = c_x dt/dx with |C| >= 1 the    */
/* state is first translated by [C] whole cells, Eq. (exact), and the        */
/* fractional remainder is then applied with Eq. (upwind).  2D: the same     */
/* donor-cell update with both fluxes taken from time level n (unsplit):     */
/*   f~ = (1 - |Cx| - |Cy|) f + |Cx| f_(upwind in x) + |Cy| f_(upwind in y). */
/* ------------------------------------------------------------------------ */
int orc_stream(const orc_config* c, const double* g, const double* h, double* gt, double* ht) {
  const int nv = orc_nv(c);
  const int ncell = orc_ncell(c);
  const double dx = orc_dx(c);
  const double dt = c->dt;
  orc_bnd b;
  if (orc_bnd_build(c, g, &b) != 0) {
    orc_bnd_free(&b);
    return -1;
  }
  if (c->dim == 1) {
#pragma omp parallel for schedule(static) if (ncell >= 64)
    for (int ix = 0; ix < c->nx; ++ix) {
      for (int j = 0; j < nv; ++j) {
        const double C = orc_cx(c, j) * dt / dx;
        const int s = (int)C;           /* [C], toward zero */
        const double r = C - s;         /* residual Courant number */
        const int up = C > 0.0 ? 1 : -1; /* upwind direction */
        double g1, h1, g2, h2;
        orc_fetch(c, &b, g, h, ix - s, 0, j, &g1, &h1);
        orc_fetch(c, &b, g, h, ix - s - up, 0, j, &g2, &h2);
        const double a = fabs(r);
        gt[(size_t)ix * nv + j] = (1.0 - a) * g1 + a * g2;
        ht[(size_t)ix * nv + j] = (1.0 - a) * h1 + a * h2;
      }
    }
  } else {
    const double dy = orc_dy(c);
#pragma omp parallel for schedule(static) if (ncell >= 64)
    for (int cell = 0; cell < ncell; ++cell) {
      const int ix = cell % c->nx, iy = cell / c->nx;
      for (int j = 0; j < nv; ++j) {
        const int jx = j % c->nvx, jy = j / c->nvx;
        const double cx = orc_cx(c, jx), cy = orc_cy(c, jy);
        const double ax = fabs(cx) * dt / dx;
        const double ay = fabs(cy) * dt / dy;
        const double g0 = g[(size_t)cell * nv + j], h0 = h[(size_t)cell * nv + j];
        double gx = g0, hx = h0, gy = g0, hy = h0;
        if (cx != 0.0) orc_fetch(c, &b, g, h, ix - (cx > 0.0 ? 1 : -1), iy, j, &gx, &hx);
        if (cy != 0.0) orc_fetch(c, &b, g, h, ix, iy - (cy > 0.0 ? 1 : -1), j, &gy, &hy);
        gt[(size_t)cell * nv + j] = (1.0 - ax - ay) * g0 + ax * gx + ay * gy;
        ht[(size_t)cell * nv + j] = (1.0 - ax - ay) * h0 + ax * hx + ay * hy;
      }
    }
  }
  orc_bnd_free(&b);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Collision sub-step, Eq. (homrel), solved exactly by Eq. (relaxation):     */
/*   f^{n+1} = [1 - exp(-nu dt)] Phi + exp(-nu dt) f~                         */
/* or, when relax_exact = 0, by the explicit Euler step                      */
/*   f^{n+1} = f~ + dt nu (Phi - f~).                                         */
/* n, U, theta and nu come from the post-streaming state f~ of the same cell */
/* (Sec. 2.1); nu = n theta^(1-omega) from Eqs. (frequency), (viscosity).    */
/* ------------------------------------------------------------------------ */
int orc_relax(const orc_config* c, double* g, double* h, double* mom) {
  const int nv = orc_nv(c);
  const int ncell = orc_ncell(c);
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad) if (ncell >= 64)
  for (int cell = 0; cell < ncell; ++cell) {
    double* gc = g + (size_t)cell * nv;
    double* hc = h + (size_t)cell * nv;
    double q[4];
    orc_moments(c, gc, hc, q);
    if (mom) {
      for (int k = 0; k < 4; ++k) mom[(size_t)cell * 4 + k] = q[k];
    }
    if (!(q[0] > 0.0) || !(q[3] > 0.0) || !isfinite(q[1]) || !isfinite(q[2])) {
      bad = 1;
      continue;
    }
    const double nu = q[0] * pow(q[3], 1.0 - c->omega);
    double p[4] = {q[0], q[1], q[2], q[3]};
    if (c->conservative && orc_effective_params(c, q, p) < 0) {
      bad = 1;
      continue;
    }
    double* G = (double*)malloc(sizeof(double) * nv);
    double* H = (double*)malloc(sizeof(double) * nv);
    orc_maxwellian(c, p, G, H);
    if (c->relax_exact) {
      const double e = exp(-nu * c->dt);
      for (int j = 0; j < nv; ++j) {
        gc[j] = (1.0 - e) * G[j] + e * gc[j];
        hc[j] = (1.0 - e) * H[j] + e * hc[j];
      }
    } else {
      const double a = c->dt * nu;
      for (int j = 0; j < nv; ++j) {
        gc[j] = gc[j] + a * (G[j] - gc[j]);
        hc[j] = hc[j] + a * (H[j] - hc[j]);
      }
    }
    free(G);
    free(H);
  }
  return bad ? -1 : 0;
}

/* Time splitting of Sec. 2.1: streaming sub-step, then collision sub-step. */
int orc_step(const orc_config* c, double* g, double* h, long nsteps, double* mom) {
  const size_t total = (size_t)orc_ncell(c) * orc_nv(c);
  double* gt = (double*)malloc(sizeof(double) * total);
  double* ht = (double*)malloc(sizeof(double) * total);
  int rc = 0;
  for (long s = 0; s < nsteps && rc == 0; ++s) {
    rc = orc_stream(c, g, h, gt, ht);
    if (rc == 0) rc = orc_relax(c, gt, ht, mom);
    memcpy(g, gt, sizeof(double) * total);
    memcpy(h, ht, sizeof(double) * total);
  }
  free(gt);
  free(ht);
  return rc;
}

/* Wall fluxes across one face, from the current state and the boundary     */
/* values the next streaming sub-step would use.                             */
int orc_wall_fluxes(const orc_config* c, const double* g, const double* h, int face,
                    double* mass, double* shear, double* normal, double* energy) {
  if (face < 0 || face >= orc_faces(c)) return -1;
  const int nv = orc_nv(c);
  const double dv = orc_dv(c);
  orc_bnd b;
  if (orc_bnd_build(c, g, &b) != 0) {
    orc_bnd_free(&b);
    return -1;
  }
  for (int k = 0; k < orc_face_cells(c, face); ++k) {
    const size_t cell = (size_t)orc_face_cell(c, face, k);
    double m = 0.0, s = 0.0, p = 0.0, e = 0.0;
    for (int j = 0; j < nv; ++j) {
      const double cn = orc_cn(c, face, j), ct = orc_ct(c, face, j);
      const int jx = j % c->nvx, jy = j / c->nvx;
      const double cx = orc_cx(c, jx), cy = orc_cy(c, jy);
      double fg, fh;
      if (cn < 0.0) {
        fg = g[cell * nv + j];
        fh = h[cell * nv + j];
      } else {
        orc_ghost(c, &b, g, h, face, k, j, &fg, &fh);
      }
      m += cn * fg * dv;
      s += ct * cn * fg * dv;
      p += cn * cn * fg * dv;
      e += cn * ((cx * cx + cy * cy) * fg + fh) * dv;
    }
    mass[k] = m;
    shear[k] = s;
    normal[k] = p;
    energy[k] = e;
  }
  orc_bnd_free(&b);
  return 0;
}

/* ======================================================================== */
/* Adjoint of the split step for the lid-integrated shear (2D cavity).      */
/* ======================================================================== */

/* J = sum_k dx tau_k over the face cells of YHI (inward normal -y, tangent
 * c_x): tau_k = dV [ sum_{c_y>0} c_x (-c_y) g_k + sum_{c_y<0} c_x (-c_y) n_W G_W ]. */
double orc_lid_shear(const orc_config* c, const double* g, const double* h) {
  const int nf = c->nx;
  double* m = (double*)malloc(sizeof(double) * nf * 4);
  orc_wall_fluxes(c, g, h, ORC_YHI, m, m + nf, m + 2 * nf, m + 3 * nf);
  double J = 0.0;
  for (int k = 0; k < nf; ++k) J += orc_dx(c) * m[nf + k];
  free(m);
  return J;
}

/* Unit wall Maxwellian of a face and its derivative in the wall's x speed. */
static void orc_wall_unit(const orc_config* c, int face, double* G, double* H, double* dG, double* dH) {
  const double* s = c->bc_state[face];
  const double unit[4] = {1.0, s[1], s[2], s[3]};
  orc_maxwellian(c, unit, G, H);
  for (int j = 0; j < orc_nv(c); ++j) {
    const double cx = orc_cx(c, j % c->nvx);
    dG[j] = G[j] * 2.0 * (cx - s[1]) / s[3];
    dH[j] = 0.5 * s[3] * dG[j];
  }
}

int orc_adjoint_lid_shear(const orc_config* c, const double* g0, const double* h0, long nsteps,
                          double* dg0, double* dh0, double out[3]) {
  if (c->dim != 2 || !c->relax_exact || c->bc_kind[ORC_YHI] != ORC_BC_DIFFUSE) return -1;
  const int nv = orc_nv(c), ncell = orc_ncell(c), nx = c->nx, ny = c->ny;
  const size_t sz = (size_t)ncell * nv;
  const double dv = orc_dv(c), dt = c->dt, dx = orc_dx(c), dy = orc_dy(c);
  double* Gs = (double*)malloc(sizeof(double) * sz * (nsteps + 1));
  double* Hs = (double*)malloc(sizeof(double) * sz * (nsteps + 1));
  memcpy(Gs, g0, sizeof(double) * sz);
  memcpy(Hs, h0, sizeof(double) * sz);
  for (long n = 0; n < nsteps; ++n) {
    double* gn = Gs + sz * n;
    double* hn = Hs + sz * n;
    if (orc_stream(c, gn, hn, gn + sz, hn + sz) != 0 || orc_relax(c, gn + sz, hn + sz, NULL) != 0) {
      free(Gs);
      free(Hs);
      return -1;
    }
  }
  const double* gN = Gs + sz * nsteps;
  const double* hN = Hs + sz * nsteps;

  /* lid tables: unit wall Maxwellian, its U_W derivative, emitted flux */
  double *GW = malloc(sizeof(double) * nv), *HW = malloc(sizeof(double) * nv);
  double *dGW = malloc(sizeof(double) * nv), *dHW = malloc(sizeof(double) * nv);
  orc_wall_unit(c, ORC_YHI, GW, HW, dGW, dHW);
  double emit = 0.0, demit = 0.0, shear_w = 0.0, dshear_w = 0.0;
  for (int j = 0; j < nv; ++j) {
    const double cn = orc_cn(c, ORC_YHI, j), ct = orc_ct(c, ORC_YHI, j);
    if (cn > 0.0) {
      emit += cn * GW[j] * dv;
      demit += cn * dGW[j] * dv;
      shear_w += ct * cn * GW[j] * dv;
      dshear_w += ct * cn * dGW[j] * dv;
    }
  }

  /* objective and its explicit derivatives */
  const double J = orc_lid_shear(c, gN, hN);
  double dlnL = J, dUW = 0.0;
  double* lg = (double*)calloc(sz, sizeof(double));
  double* lh = (double*)calloc(sz, sizeof(double));
  for (int k = 0; k < nx; ++k) {
    const size_t cell = (size_t)(ny - 1) * nx + k;
    double inc = 0.0;
    for (int j = 0; j < nv; ++j) {
      const double cn = orc_cn(c, ORC_YHI, j);
      if (cn < 0.0) inc += -cn * gN[cell * nv + j] * dv;
    }
    const double nw = inc / emit;
    dUW += dx * nw * (dshear_w - shear_w * demit / emit);
    for (int j = 0; j < nv; ++j) {
      const double cn = orc_cn(c, ORC_YHI, j), ct = orc_ct(c, ORC_YHI, j);
      if (cn < 0.0) lg[cell * nv + j] = dx * (ct * cn * dv + shear_w * (-cn) * dv / emit);
    }
  }

  /* reverse sweep */
  double* ltg = (double*)malloc(sizeof(double) * sz);  /* adjoint of f~ */
  double* lth = (double*)malloc(sizeof(double) * sz);
  double* ng = (double*)malloc(sizeof(double) * sz);
  double* nh = (double*)malloc(sizeof(double) * sz);
  double* ftg = (double*)malloc(sizeof(double) * sz);
  double* fth = (double*)malloc(sizeof(double) * sz);
  double* G = (double*)malloc(sizeof(double) * nv);
  double* H = (double*)malloc(sizeof(double) * nv);
  double* Gf[4], *Hf[4], *dGf[4], *dHf[4];
  double emitf[4] = {0, 0, 0, 0};
  for (int f = 0; f < 4; ++f) {
    Gf[f] = malloc(sizeof(double) * nv);
    Hf[f] = malloc(sizeof(double) * nv);
    dGf[f] = malloc(sizeof(double) * nv);
    dHf[f] = malloc(sizeof(double) * nv);
    orc_wall_unit(c, f, Gf[f], Hf[f], dGf[f], dHf[f]);
    for (int j = 0; j < nv; ++j)
      if (orc_cn(c, f, j) > 0.0) emitf[f] += orc_cn(c, f, j) * Gf[f][j] * dv;
  }
  int rc = 0;
  for (long n = nsteps - 1; n >= 0 && rc == 0; --n) {
    const double* gn = Gs + sz * n;
    const double* hn = Hs + sz * n;
    orc_stream(c, gn, hn, ftg, fth);
    /* collision adjoint, cell by cell (Eq. relaxation differentiated) */
    for (int cell = 0; cell < ncell; ++cell) {
      const double* gt = ftg + (size_t)cell * nv;
      const double* ht = fth + (size_t)cell * nv;
      double q[4], p[4];
      orc_moments(c, gt, ht, q);
      for (int k = 0; k < 4; ++k) p[k] = q[k];
      if (c->conservative && orc_effective_params(c, q, p) < 0) {
        rc = -1;
        break;
      }
      orc_maxwellian(c, p, G, H);
      const double nu = q[0] * pow(q[3], 1.0 - c->omega);
      const double e = exp(-nu * dt);
      const double a = 1.0 - e;
      const double* lgc = lg + (size_t)cell * nv;
      const double* lhc = lh + (size_t)cell * nv;
      double sa = 0.0, sp[4] = {0, 0, 0, 0};
      double E = 0.0;
      for (int j = 0; j < nv; ++j) {
        const double cx = orc_cx(c, j % c->nvx), cy = orc_cy(c, j / c->nvx);
        E += ((cx * cx + cy * cy) * gt[j] + ht[j]) * dv;
        sa += lgc[j] * (G[j] - gt[j]) + lhc[j] * (H[j] - ht[j]);
        const double dxp = cx - p[1], dyp = cy - p[2];
        const double dG[4] = {G[j] / p[0], G[j] * 2.0 * dxp / p[3], G[j] * 2.0 * dyp / p[3],
                              G[j] * ((dxp * dxp + dyp * dyp) / (p[3] * p[3]) - 1.0 / p[3])};
        for (int k = 0; k < 4; ++k) {
          const double dH = 0.5 * p[3] * dG[k] + (k == 3 ? 0.5 * G[j] : 0.0);
          sp[k] += lgc[j] * dG[k] + lhc[j] * dH;
        }
      }
      /* adjoint of q: Phi through p (dp/dq = identity), a through nu */
      const double da_dn = dt * e * pow(q[3], 1.0 - c->omega);
      const double da_dth = dt * e * (1.0 - c->omega) * q[0] * pow(q[3], -c->omega);
      const double mu[4] = {a * sp[0] + da_dn * sa, a * sp[1], a * sp[2], a * sp[3] + da_dth * sa};
      dlnL += sa * nu * dt * e; /* dt scales with L */
      const double n_ = q[0], ux = q[1], uy = q[2];
      for (int j = 0; j < nv; ++j) {
        const double cx = orc_cx(c, j % c->nvx), cy = orc_cy(c, j / c->nvx);
        const double dn = dv;
        const double dux = dv * (cx - ux) / n_;
        const double duy = dv * (cy - uy) / n_;
        const double dth = (2.0 / 3.0) * (dv / n_) * ((cx * cx + cy * cy) - E / n_ - 2.0 * (ux * (cx - ux) + uy * (cy - uy)));
        ltg[(size_t)cell * nv + j] = (1.0 - a) * lgc[j] + mu[0] * dn + mu[1] * dux + mu[2] * duy + mu[3] * dth;
        lth[(size_t)cell * nv + j] = (1.0 - a) * lhc[j] + mu[3] * (2.0 / 3.0) * dv / n_;
      }
    }
    if (rc) break;
    /* streaming adjoint: scatter each f~ back to its sources (transposed
       donor cell); boundary sources feed the wall density n_W */
    memset(ng, 0, sizeof(double) * sz);
    memset(nh, 0, sizeof(double) * sz);
    for (int cell = 0; cell < ncell; ++cell) {
      const int ix = cell % nx, iy = cell / nx;
      double lam_face[4] = {0, 0, 0, 0};
      double inc[4] = {0, 0, 0, 0};
      for (int j = 0; j < nv; ++j) {
        for (int f = 0; f < 4; ++f)
          if (orc_cn(c, f, j) < 0.0) inc[f] += -orc_cn(c, f, j) * gn[(size_t)cell * nv + j] * dv;
      }
      for (int j = 0; j < nv; ++j) {
        const double cx = orc_cx(c, j % c->nvx), cy = orc_cy(c, j / c->nvx);
        const double ax = fabs(cx) * dt / dx, ay = fabs(cy) * dt / dy;
        const size_t id = (size_t)cell * nv + j;
        ng[id] += (1.0 - ax - ay) * ltg[id];
        nh[id] += (1.0 - ax - ay) * lth[id];
        for (int axis = 0; axis < 2; ++axis) {
          const double cc = axis == 0 ? cx : cy, w = axis == 0 ? ax : ay;
          if (cc == 0.0) continue;
          const int sx = axis == 0 ? (cc > 0.0 ? -1 : 1) : 0, sy = axis == 1 ? (cc > 0.0 ? -1 : 1) : 0;
          const int jx2 = ix + sx, iy2 = iy + sy;
          if (jx2 >= 0 && jx2 < nx && iy2 >= 0 && iy2 < ny) {
            const size_t src = ((size_t)iy2 * nx + jx2) * nv + j;
            ng[src] += w * ltg[id];
            nh[src] += w * lth[id];
          } else {
            const int face = axis == 0 ? (cc > 0.0 ? ORC_XLO : ORC_XHI) : (cc > 0.0 ? ORC_YLO : ORC_YHI);
            if (c->bc_kind[face] == ORC_BC_DIFFUSE) {
              lam_face[face] += w * (ltg[id] * Gf[face][j] + lth[id] * Hf[face][j]);
              if (face == ORC_YHI) {
                const double nw = inc[face] / emitf[face];
                const double dgh = nw * (dGf[face][j] - Gf[face][j] * demit / emitf[face]);
                const double dhh = nw * (dHf[face][j] - Hf[face][j] * demit / emitf[face]);
                dUW += w * (ltg[id] * dgh + lth[id] * dhh);
              }
            } else if (c->bc_kind[face] == ORC_BC_SPECULAR) {
              const size_t src = (size_t)cell * nv + orc_reflect(c, face, j);
              ng[src] += w * ltg[id];
              nh[src] += w * lth[id];
            }
          }
        }
      }
      /* n_W = dv sum_{c_n<0} |c_n| g / emitted */
      for (int f = 0; f < 4; ++f) {
        if (lam_face[f] == 0.0) continue;
        for (int j = 0; j < nv; ++j)
          if (orc_cn(c, f, j) < 0.0) ng[(size_t)cell * nv + j] += lam_face[f] * (-orc_cn(c, f, j)) * dv / emitf[f];
      }
    }
    memcpy(lg, ng, sizeof(double) * sz);
    memcpy(lh, nh, sizeof(double) * sz);
  }
  if (rc == 0) {
    memcpy(dg0, lg, sizeof(double) * sz);
    memcpy(dh0, lh, sizeof(double) * sz);
    out[0] = J;
    out[1] = dlnL;
    out[2] = dUW;
  }
  for (int f = 0; f < 4; ++f) {
    free(Gf[f]);
    free(Hf[f]);
    free(dGf[f]);
    free(dHf[f]);
  }
  free(G); free(H); free(ftg); free(fth); free(ng); free(nh); free(ltg); free(lth);
  free(lg); free(lh); free(GW); free(HW); free(dGW); free(dHW); free(Gs); free(Hs);
  return rc;
}
