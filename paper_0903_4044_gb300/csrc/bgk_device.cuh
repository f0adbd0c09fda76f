// bgk_device.cuh - device helpers of libbgk.so: warp/block reductions, the
// reduced Maxwellian, boundary values and the effective-parameter solve.
#pragma once

#include "bgk_internal.h"

namespace bgk {

__device__ __forceinline__ double kPi() { return 3.14159265358979323846; }

// ---------------------------------------------------------------------------
// Reductions.  FP64 adds run on the (slow) FP64 pipe of sm_103, so sums of
// several values use recursive halving: at each xor level a lane keeps half
// of its values and adds the partner's copy of them, instead of reducing
// every value across all 32 lanes.
// ---------------------------------------------------------------------------

// Four values per lane -> lane L ends with the warp total of value
// (L >> 3) & 3.  6 FP64 adds per lane instead of 20.
__device__ __forceinline__ double warp_reduce4(double v0, double v1, double v2, double v3) {
  const int lane = threadIdx.x & 31;
  const bool b4 = lane & 16, b3 = lane & 8;
  double ra = __shfl_xor_sync(0xffffffffu, b4 ? v0 : v2, 16);
  double rb = __shfl_xor_sync(0xffffffffu, b4 ? v1 : v3, 16);
  const double a = (b4 ? v2 : v0) + ra;
  const double b = (b4 ? v3 : v1) + rb;
  const double r = __shfl_xor_sync(0xffffffffu, b3 ? a : b, 8);
  double x = (b3 ? b : a) + r;
  x += __shfl_xor_sync(0xffffffffu, x, 4);
  x += __shfl_xor_sync(0xffffffffu, x, 2);
  x += __shfl_xor_sync(0xffffffffu, x, 1);
  return x;
}

// Eight values per lane -> lane L ends with the warp total of value
// (L >> 2) & 7.  9 FP64 adds per lane.
__device__ __forceinline__ double warp_reduce8(const double (&v)[8]) {
  const int lane = threadIdx.x & 31;
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
  double a[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double r = __shfl_xor_sync(0xffffffffu, b4 ? v[k] : v[k + 4], 16);
    a[k] = (b4 ? v[k + 4] : v[k]) + r;
  }
  double b[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const double r = __shfl_xor_sync(0xffffffffu, b3 ? a[k] : a[k + 2], 8);
    b[k] = (b3 ? a[k + 2] : a[k]) + r;
  }
  const double r = __shfl_xor_sync(0xffffffffu, b2 ? b[0] : b[1], 4);
  double x = (b2 ? b[1] : b[0]) + r;
  x += __shfl_xor_sync(0xffffffffu, x, 2);
  x += __shfl_xor_sync(0xffffffffu, x, 1);
  return x;
}

// Block sum of four values; the totals land in out[0..3] (shared memory)
// and are valid for every thread after the call.  `red` holds
// 4 * (BLOCK/32) doubles.  Fixed summation order (deterministic).
template <int BLOCK>
__device__ __forceinline__ void block_reduce4(double v0, double v1, double v2, double v3,
                                              double* red, double* out) {
  constexpr int NW = BLOCK / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double w = warp_reduce4(v0, v1, v2, v3);
  if ((lane & 7) == 0) red[warp * 4 + (lane >> 3)] = w;
  __syncthreads();
  if (warp == 0) {
    double x = (lane >> 2) < NW ? red[(lane >> 2) * 4 + (lane & 3)] : 0.0;
    if (NW > 1) x += __shfl_xor_sync(0xffffffffu, x, 4);
    if (NW > 2) x += __shfl_xor_sync(0xffffffffu, x, 8);
    if (NW > 4) x += __shfl_xor_sync(0xffffffffu, x, 16);
    if (lane < 4) out[lane] = x;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Eq. (Maxw) reduced over the unresolved components (Chu):
//   dim 1: G = n (pi theta)^(-1/2) e^{-(cx-ux)^2/theta}, H = theta G
//   dim 2: G = n (pi theta)^(-1) e^{-|c-U|^2/theta},     H = theta/2 G
// ---------------------------------------------------------------------------
__device__ __forceinline__ double2 maxwell_point(int dim, const double p[4], double cx, double cy) {
  const double th = p[3];
  const double dx = cx - p[1];
  double G;
  if (dim == 1) {
    G = p[0] / sqrt(kPi() * th) * exp(-dx * dx / th);
    return make_double2(G, th * G);
  }
  const double dy = cy - p[2];
  G = p[0] / (kPi() * th) * exp(-dx * dx / th) * exp(-dy * dy / th);
  return make_double2(G, 0.5 * th * G);
}

// Eq. (macroscopic) from the velocity sums s0 = sum g, sx = sum cx g,
// sy = sum cy g, se = sum (|c|^2 g + h):  n, ux, uy, theta.
__device__ __forceinline__ void moments_from_sums(double s0, double sx, double sy, double se,
                                                  double dv, double q[4]) {
  const double n = s0 * dv;
  const double in = dv / n;  // one division
  const double ux = sx * in;
  const double uy = sy * in;
  q[0] = n;
  q[1] = ux;
  q[2] = uy;
  q[3] = (2.0 / 3.0) * (se * in - (ux * ux + uy * uy));
}

__device__ __forceinline__ bool moments_ok(const double q[4]) {
  return q[0] > 0.0 && q[3] > 0.0 && isfinite(q[0]) && isfinite(q[1]) && isfinite(q[2]) &&
         isfinite(q[3]);
}

// ---------------------------------------------------------------------------
// Effective Maxwellian parameters (Sec. 2.1, remark after Eq. exact): find p
// with D(p) = q, D = discrete moments of the reduced Maxwellian, by
// p <- p + (q - D(p)) from p = q.  D is evaluated from central sums
// M_m = sum_j d^m e_j, d = c_j - u_b, e_j = exp(-d^2/theta_b) of each axis,
// taken at a base point b, and moved to p to first order:
//   e_j(p) = e_j(b) (1 + d (w1 + d w2)), w1 = 2 (u - u_b)/theta_b,
//   w2 = (theta - theta_b)/theta_b^2,
// so that with S_m = M_m + w1 M_{m+1} + w2 M_{m+2} per axis
//   n_d = n (pi theta)^(-d/2) dv Sx0 Sy0,  U_d = u_b + S1/S0,
//   theta_d = (2/3) (sum over axes of (S2/S0 - (S1/S0)^2) + kappa),
// kappa = theta (dim 1) or theta/2 (dim 2) being the h part per unit
// density.  When p has moved more than kLinMax from b the caller
// re-evaluates the Gaussians at b = p (reeval).  Every lane runs its own
// cell; the loop has no cross-lane operations.
// ---------------------------------------------------------------------------
struct EffState {
  double base[4], p[4];
  double ib0, ith, isq;  // 1 / n_b, 1 / theta_b, 1 / sqrt(theta_b)
  double iq0, iq3, ivs;  // the same at the target q (the first base point)
  int it;
  bool conv, fail, reeval;
};

// Reciprocals of the base point, taken once per base (the FP64 pipe
// charges a division about ten instructions, so both come from one: 1 / n_b
// = theta_b / (n_b theta_b), within two roundings), and 1 / sqrt(theta_b)
// from the reciprocal square root (within one ulp).
__device__ __forceinline__ void eff_set_base(EffState& E) {
  const double r = 1.0 / (E.base[0] * E.base[3]);
  E.ib0 = E.base[3] * r;
  E.ith = E.base[0] * r;
  E.isq = rsqrt(E.base[3]);
}

__device__ __forceinline__ void eff_init(EffState& E, const double q[4], bool done) {
  for (int k = 0; k < 4; ++k) E.base[k] = E.p[k] = q[k];
  eff_set_base(E);
  E.iq0 = E.ib0;
  E.iq3 = E.ith;
  E.ivs = E.isq;
  E.it = 0;
  E.conv = done;
  E.fail = false;
  E.reeval = false;
}

template <int DIM>
__device__ __forceinline__ void eff_iterate(const Params& P, const double q[4], const double Mx[5],
                                            const double My[5], EffState& E, double lin_max = kLinMax,
                                            double tol = kEffTol) {
  // the convergence test scales n by q_n, U by sqrt(q_theta), theta by q_theta
  const double iq0 = E.iq0, iq3 = E.iq3, ivs = E.ivs;
  double* p = E.p;
  double* b = E.base;
  while (!E.conv && !E.fail && !E.reeval) {
    ++E.it;
    const double ith = E.ith;
    const double w2 = (p[3] - b[3]) * ith * ith;
    double Sx[3], Sy[3] = {1.0, 0.0, 0.0};
    const double w1x = 2.0 * (p[1] - b[1]) * ith;
#pragma unroll
    for (int m = 0; m < 3; ++m) Sx[m] = Mx[m] + w1x * Mx[m + 1] + w2 * Mx[m + 2];
    if (DIM == 2) {
      const double w1y = 2.0 * (p[2] - b[2]) * ith;
#pragma unroll
      for (int m = 0; m < 3; ++m) Sy[m] = My[m] + w1y * My[m + 1] + w2 * My[m + 2];
    }
    const double pref = (DIM == 1) ? p[0] * rsqrt(kPi() * p[3]) : p[0] / (kPi() * p[3]);
    const double rxy = 1.0 / (Sx[0] * Sy[0]);  // one division for 1/Sx0 and 1/Sy0
    const double rx = Sy[0] * rxy, ry = Sx[0] * rxy;
    const double mux = Sx[1] * rx, muy = Sy[1] * ry;
    double d[4];
    d[0] = pref * P.dv * Sx[0] * Sy[0];
    d[1] = b[1] + mux;
    d[2] = (DIM == 2) ? b[2] + muy : 0.0;
    const double kappa = (DIM == 1) ? p[3] : 0.5 * p[3];
    const double var = (Sx[2] * rx - mux * mux) + ((DIM == 2) ? (Sy[2] * ry - muy * muy) : 0.0);
    d[3] = (2.0 / 3.0) * (var + kappa);
    double r = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const double delta = q[k] - d[k];
      p[k] += delta;
      const double iscale = (k == 0) ? iq0 : (k == 3) ? iq3 : ivs;
      r = fmax(r, fabs(delta) * iscale);
    }
    if (!(p[0] > 0.0) || !(p[3] > 0.0) || !isfinite(r)) {
      E.fail = true;
    } else if (r < tol || (E.it == 1 && 100.0 * r * r < tol)) {
      // the map p -> D(p) - p changes by the quadrature defect, so the
      // iteration contracts by about the size r of its first update: after a
      // first update r the next one is about r^2, below the tolerance here
      E.conv = true;
    } else if (E.it >= kEffMaxIt) {
      if (r < kEffFail) E.conv = true;
      else E.fail = true;
    }
    if (!E.fail) {
      const double drift = fmax(fmax(fabs(p[0] - b[0]) * E.ib0, fabs(p[3] - b[3]) * ith),
                                fmax(fabs(p[1] - b[1]), fabs(p[2] - b[2])) * E.isq);
      if (drift > lin_max) {
        for (int k = 0; k < 4; ++k) b[k] = p[k];
        eff_set_base(E);
        E.reeval = true;
      }
    }
  }
}

// First-order factors that move the Gaussians from E.base to E.p.
__device__ __forceinline__ void eff_lin(const EffState& E, double& w1x, double& w1y, double& w2) {
  const double ith = E.ith;
  w2 = (E.p[3] - E.base[3]) * ith * ith;
  w1x = 2.0 * (E.p[1] - E.base[1]) * ith;
  w1y = 2.0 * (E.p[2] - E.base[2]) * ith;
}

// Relaxation weights from nu = n theta^(1-omega): exact (Eq. relaxation)
// b = exp(-nu dt), a = 1 - b; Euler a = nu dt, b = 1 - a.
__device__ __forceinline__ void relax_weights(const Params& P, const double q[4], double& a, double& b) {
  const double nu = q[0] * (P.omega == 0.5 ? sqrt(q[3]) : pow(q[3], 1.0 - P.omega));
  if (P.relax_exact) {
    b = exp(-nu * P.dt);
    a = 1.0 - b;
  } else {
    a = P.dt * nu;
    b = 1.0 - a;
  }
}

// Boundary value (g, h) just outside `face` at velocity j: the inflow
// Maxwellian, n_W times the unit wall Maxwellian, or the mirror image of the
// wall-adjacent cell's own state `fc` (specular).
__device__ __forceinline__ double2 ghost_value(const Params& P, const Tables& T, int face, int j,
                                               double nw, const double2* __restrict__ fc) {
  const int kind = P.bc_kind[face];
  if (kind == BC_SPECULAR) {
    const int jx = j % P.nvx, jy = j / P.nvx;
    const int jr = (face == XLO || face == XHI) ? jy * P.nvx + (P.nvx - 1 - jx)
                                                : (P.nvy - 1 - jy) * P.nvx + jx;
    return fc[jr];
  }
  const double2 gv = T.ghost[face * P.nv + j];
  if (kind == BC_DIFFUSE) return make_double2(nw * gv.x, nw * gv.y);
  return gv;
}

}  // namespace bgk
