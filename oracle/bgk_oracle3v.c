/*
 * bgk_oracle3v.c - plain FP64 CPU oracle of the BGK step with a full 3D
 * velocity grid and one spatial dimension.
 *
 * TEST INFRASTRUCTURE ONLY (see bgk_oracle3v.h).  Naive loops, one formula
 * per line; the Gaussian is evaluated as the product of its three
 * one-dimensional factors, which is the same function.  Compile with
 * -ffp-contract=off.
 */
#include "bgk_oracle3v.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static const double O3_PI = 3.14159265358979323846;

#define O3_EFF_TOL 1e-13
#define O3_EFF_MAXIT 20
#define O3_EFF_FAIL 1e-9

static int o3_n(const orc3_config* c, int axis) { return axis == 0 ? c->nvx : axis == 1 ? c->nvy : c->nvz; }
static double o3_dc(const orc3_config* c, int axis) { return (c->vmax[axis] - c->vmin[axis]) / o3_n(c, axis); }

int orc3_nv(const orc3_config* c) { return c->nvx * c->nvy * c->nvz; }
double orc3_c(const orc3_config* c, int axis, int j) { return c->vmin[axis] + (j + 0.5) * o3_dc(c, axis); }
double orc3_dv(const orc3_config* c) { return o3_dc(c, 0) * o3_dc(c, 1) * o3_dc(c, 2); }

/* Largest |c_x| over the cell centres. */
static double o3_max_abs_cx(const orc3_config* c) {
  double m = 0.0;
  for (int j = 0; j < c->nvx; ++j) {
    const double a = fabs(orc3_c(c, 0, j));
    if (a > m) m = a;
  }
  return m;
}

double orc3_dt_from_cfl(const orc3_config* c, double cfl) { return cfl * (c->lx / c->nx) / o3_max_abs_cx(c); }

/* Eq. (Maxw), normalised: n (pi theta)^(-3/2) exp(-|c - U|^2 / theta). */
void orc3_maxwellian(const orc3_config* c, const double p[5], double* phi) {
  const double n = p[0], th = p[4];
  const double pref = n / pow(O3_PI * th, 1.5);
  for (int jz = 0; jz < c->nvz; ++jz) {
    const double dz = orc3_c(c, 2, jz) - p[3];
    const double ez = exp(-dz * dz / th);
    for (int jy = 0; jy < c->nvy; ++jy) {
      const double dy = orc3_c(c, 1, jy) - p[2];
      const double ey = exp(-dy * dy / th);
      for (int jx = 0; jx < c->nvx; ++jx) {
        const double dx = orc3_c(c, 0, jx) - p[1];
        const double ex = exp(-dx * dx / th);
        phi[(jz * c->nvy + jy) * c->nvx + jx] = pref * ex * ey * ez;
      }
    }
  }
}

/* Eq. (macroscopic): n = sum f dV, n U = sum c f dV,
 * theta = (2/3) (E/n - |U|^2), E = sum |c|^2 f dV. */
void orc3_moments(const orc3_config* c, const double* f, double out[5]) {
  const double dv = orc3_dv(c);
  double s0 = 0.0, sx = 0.0, sy = 0.0, sz = 0.0, se = 0.0;
  for (int jz = 0; jz < c->nvz; ++jz) {
    const double cz = orc3_c(c, 2, jz);
    for (int jy = 0; jy < c->nvy; ++jy) {
      const double cy = orc3_c(c, 1, jy);
      for (int jx = 0; jx < c->nvx; ++jx) {
        const double cx = orc3_c(c, 0, jx);
        const double v = f[(jz * c->nvy + jy) * c->nvx + jx];
        s0 += v;
        sx += cx * v;
        sy += cy * v;
        sz += cz * v;
        se += (cx * cx + cy * cy + cz * cz) * v;
      }
    }
  }
  const double n = s0 * dv;
  const double ux = sx * dv / n, uy = sy * dv / n, uz = sz * dv / n;
  out[0] = n;
  out[1] = ux;
  out[2] = uy;
  out[3] = uz;
  out[4] = (2.0 / 3.0) * (se * dv / n - (ux * ux + uy * uy + uz * uz));
}

/* Sec. 2.1 remark: p <- p + (q - D(p)), D(p) the discrete moments of the
 * discrete Maxwellian of p, until the update is below O3_EFF_TOL. */
int orc3_effective_params(const orc3_config* c, const double q[5], double p_out[5]) {
  const int nv = orc3_nv(c);
  double* phi = (double*)malloc(sizeof(double) * nv);
  double p[5];
  for (int k = 0; k < 5; ++k) p[k] = q[k];
  int it = 0, ok = 0;
  double r = 0.0;
  for (it = 1; it <= O3_EFF_MAXIT; ++it) {
    double d[5];
    orc3_maxwellian(c, p, phi);
    orc3_moments(c, phi, d);
    const double vs = sqrt(q[4]);
    r = 0.0;
    for (int k = 0; k < 5; ++k) {
      const double delta = q[k] - d[k];
      p[k] += delta;
      const double scale = k == 0 ? q[0] : k == 4 ? q[4] : vs;
      if (fabs(delta) / scale > r) r = fabs(delta) / scale;
    }
    if (!(p[0] > 0.0) || !(p[4] > 0.0) || !isfinite(r)) break;
    if (r < O3_EFF_TOL) {
      ok = 1;
      break;
    }
  }
  if (!ok && it > O3_EFF_MAXIT && r < O3_EFF_FAIL) {
    ok = 1; /* stalled at round-off level */
    it = O3_EFF_MAXIT;
  }
  for (int k = 0; k < 5; ++k) p_out[k] = p[k];
  free(phi);
  return ok ? it : -1;
}

void orc3_init_step(const orc3_config* c, double x_split, const double left[5], const double right[5],
                    double* f) {
  const int nv = orc3_nv(c);
  double* pl = (double*)malloc(sizeof(double) * nv);
  double* pr = (double*)malloc(sizeof(double) * nv);
  orc3_maxwellian(c, left, pl);
  orc3_maxwellian(c, right, pr);
  const double dx = c->lx / c->nx;
  for (int i = 0; i < c->nx; ++i) {
    const double x = c->x0 + (i + 0.5) * dx;
    memcpy(f + (size_t)i * nv, x < x_split ? pl : pr, sizeof(double) * nv);
  }
  free(pl);
  free(pr);
}

/* Eq. (exact) then Eq. (upwind) along x: C = c_x dt/dx, shift by [C]
 * (toward zero) and upwind the remainder; indices beyond the ends read the
 * inflow Maxwellian of that end. */
void orc3_stream(const orc3_config* c, const double* f, double* ft) {
  const int nv = orc3_nv(c);
  double* gl = (double*)malloc(sizeof(double) * nv);
  double* gr = (double*)malloc(sizeof(double) * nv);
  orc3_maxwellian(c, c->inflow[0], gl);
  orc3_maxwellian(c, c->inflow[1], gr);
  const double dx = c->lx / c->nx;
#pragma omp parallel for schedule(static) if (c->nx >= 64)
  for (int i = 0; i < c->nx; ++i) {
    for (int j = 0; j < nv; ++j) {
      const int jx = j % c->nvx;
      const double C = orc3_c(c, 0, jx) * c->dt / dx;
      const int s = (int)C;
      const double r = C - s;
      const int up = C > 0.0 ? 1 : -1;
      const int i1 = i - s, i2 = i - s - up;
      const double f1 = i1 < 0 ? gl[j] : i1 >= c->nx ? gr[j] : f[(size_t)i1 * nv + j];
      const double f2 = i2 < 0 ? gl[j] : i2 >= c->nx ? gr[j] : f[(size_t)i2 * nv + j];
      const double a = fabs(r);
      ft[(size_t)i * nv + j] = (1.0 - a) * f1 + a * f2;
    }
  }
  free(gl);
  free(gr);
}

/* Eq. (relaxation): f <- (1 - e^{-nu dt}) Phi + e^{-nu dt} f~ (or Euler),
 * nu = n theta^(1-omega) from the post-streaming moments of the cell. */
int orc3_relax(const orc3_config* c, double* f, double* mom) {
  const int nv = orc3_nv(c);
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad) if (c->nx >= 16)
  for (int i = 0; i < c->nx; ++i) {
    double* fc = f + (size_t)i * nv;
    double q[5], p[5];
    orc3_moments(c, fc, q);
    if (mom)
      for (int k = 0; k < 5; ++k) mom[(size_t)i * 5 + k] = q[k];
    if (!(q[0] > 0.0) || !(q[4] > 0.0) || !isfinite(q[1]) || !isfinite(q[2]) || !isfinite(q[3])) {
      bad = 1;
      continue;
    }
    for (int k = 0; k < 5; ++k) p[k] = q[k];
    if (c->conservative && orc3_effective_params(c, q, p) < 0) {
      bad = 1;
      continue;
    }
    double* phi = (double*)malloc(sizeof(double) * nv);
    orc3_maxwellian(c, p, phi);
    const double nu = q[0] * pow(q[4], 1.0 - c->omega);
    const double a = c->relax_exact ? 1.0 - exp(-nu * c->dt) : nu * c->dt;
    for (int j = 0; j < nv; ++j) fc[j] = fc[j] + a * (phi[j] - fc[j]);
    free(phi);
  }
  return bad ? -1 : 0;
}

int orc3_step(const orc3_config* c, double* f, long nsteps, double* mom) {
  const int nv = orc3_nv(c);
  double* ft = (double*)malloc(sizeof(double) * (size_t)c->nx * nv);
  int rc = 0;
  for (long n = 0; n < nsteps && rc == 0; ++n) {
    orc3_stream(c, f, ft);
    rc = orc3_relax(c, ft, mom);
    memcpy(f, ft, sizeof(double) * (size_t)c->nx * nv);
  }
  free(ft);
  return rc;
}
