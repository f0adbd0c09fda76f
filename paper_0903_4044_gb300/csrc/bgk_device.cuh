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
  const double ux = sx * dv / n;
  const double uy = sy * dv / n;
  const double e = se * dv;
  q[0] = n;
  q[1] = ux;
  q[2] = uy;
  q[3] = (2.0 / 3.0) * (e / n - (ux * ux + uy * uy));
}

__device__ __forceinline__ bool moments_ok(const double q[4]) {
  return q[0] > 0.0 && q[3] > 0.0 && isfinite(q[0]) && isfinite(q[1]) && isfinite(q[2]) &&
         isfinite(q[3]);
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
