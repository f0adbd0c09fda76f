// bgk_aux.cu - set-up and diagnostic kernels of libbgk.so: velocity and
// boundary tables, initial states, moments of the current state and wall
// fluxes.  None of these is on the per-step path.
#include "bgk_device.cuh"

namespace bgk {

// Cell-centred velocity of index j along one axis (Sec. 2.1), without FMA
// contraction so that the grid is the plain expression vmin + (j + 1/2) dc.
__device__ __forceinline__ double centre(double vmin, int j, double dc) {
  return __dadd_rn(vmin, __dmul_rn((double)j + 0.5, dc));
}

// Per-velocity streaming weights and boundary Maxwellians.
__global__ void tables_kernel(const Params P, double* cx, double* cy, double4_32a* coef, int* shift,
                              double2* cxy, int* vinfo, double2* ghost) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= P.nv) return;
  const int jx = j % P.nvx, jy = j / P.nvx;
  const double cxj = centre(P.vx_min, jx, P.dcx);
  const double cyj = (P.dim == 2) ? centre(P.vy_min, jy, P.dcy) : 0.0;
  if (jy == 0) cx[jx] = cxj;
  if (jx == 0) cy[jy] = cyj;
  if (jx == 0) cy[P.nvy + jy] = __dmul_rn(cyj, cyj);  // c_y^2 after the centres
  const double c2 = __dadd_rn(__dmul_rn(cxj, cxj), __dmul_rn(cyj, cyj));
  cxy[j] = make_double2(cxj, cyj);
  const int sgx = cxj > 0.0 ? 1 : (cxj < 0.0 ? -1 : 0);
  const int sgy = cyj > 0.0 ? 1 : (cyj < 0.0 ? -1 : 0);
  vinfo[j] = jx | (jy << 12) | ((sgx + 1) << 24) | ((sgy + 1) << 26);
  if (P.dim == 2) {
    // unsplit donor cell: f~ = (1 - |Cx| - |Cy|) f + |Cx| f_upx + |Cy| f_upy
    const double ax = fabs(cxj) * P.dt / P.dx;
    const double ay = fabs(cyj) * P.dt / P.dy;
    coef[j] = make_double4_32a(1.0 - ax - ay, ax, ay, c2);
    shift[j] = 0;
  } else {
    // Eq. (exact) shift by [C], then Eq. (upwind) with the remainder r
    const double C = cxj * P.dt / P.dx;
    const int s = (int)C;
    const double r = fabs(C - s);
    coef[j] = make_double4_32a(1.0 - r, r, 0.0, c2);
    shift[j] = s;
  }
  const int nfaces = (P.dim == 2) ? 4 : 2;
  for (int face = 0; face < nfaces; ++face) {
    const double* s = P.bc_state[face];
    double2 v = make_double2(0.0, 0.0);
    if (P.bc_kind[face] == BC_INFLOW) {
      v = maxwell_point(P.dim, s, cxj, cyj);
    } else if (P.bc_kind[face] == BC_DIFFUSE) {
      const double unit[4] = {1.0, s[1], s[2], s[3]};
      v = maxwell_point(P.dim, unit, cxj, cyj);
    }
    ghost[face * P.nv + j] = v;
  }
}

// emitted[face] = sum_{c_n > 0} c_n G_W(n = 1) dv for diffuse faces.
__global__ void __launch_bounds__(256) emitted_kernel(const Params P, const double* cx,
                                                      const double* cy, const double2* ghost,
                                                      double* emitted) {
  __shared__ double red[4 * 8];
  __shared__ double tot[4];
  double e[4] = {0.0, 0.0, 0.0, 0.0};
  for (int j = threadIdx.x; j < P.nv; j += 256) {
    const double cxj = cx[j % P.nvx];
    const double cyj = cy[j / P.nvx];
    const double cn[4] = {cxj, -cxj, cyj, -cyj};
    for (int face = 0; face < 4; ++face) {
      if (P.bc_kind[face] == BC_DIFFUSE && (P.dim == 2 || face < 2) && cn[face] > 0.0)
        e[face] = fma(cn[face], ghost[face * P.nv + j].x, e[face]);
    }
  }
  block_reduce4<256>(e[0], e[1], e[2], e[3], red, tot);
  if (threadIdx.x < 4) emitted[threadIdx.x] = tot[threadIdx.x] * P.dv;
}

cudaError_t launch_build_tables(const Params& P, double* cx, double* cy, double4_32a* coef, int* shift,
                                double2* cxy, int* vinfo, double2* ghost, double* emitted,
                                cudaStream_t stream) {
  tables_kernel<<<(P.nv + 255) / 256, 256, 0, stream>>>(P, cx, cy, coef, shift, cxy, vinfo, ghost);
  emitted_kernel<<<1, 256, 0, stream>>>(P, cx, cy, ghost, emitted);
  return cudaGetLastError();
}

// Shock initial condition (Sec. 4.1): Maxwellian step at x_split.
__global__ void init_step_kernel(const Params P, double2* f, double x_split, const double4_32a left,
                                 const double4_32a right) {
  const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  const size_t total = (size_t)P.nx * P.ny * P.nv;
  if (idx >= total) return;
  const int cell = (int)(idx / P.nv), j = (int)(idx % P.nv);
  const int ix = cell % P.nx;
  const double x = __dadd_rn(P.x0, __dmul_rn((double)ix + 0.5, P.dx));
  const double4_32a s = (x < x_split) ? left : right;
  const double p[4] = {s.x, s.y, s.z, s.w};
  const double cxj = centre(P.vx_min, j % P.nvx, P.dcx);
  const double cyj = (P.dim == 2) ? centre(P.vy_min, j / P.nvx, P.dcy) : 0.0;
  f[idx] = maxwell_point(P.dim, p, cxj, cyj);
}

cudaError_t launch_init_step(const Params& P, double2* f, double x_split, const double left[4],
                             const double right[4], cudaStream_t stream) {
  const size_t total = (size_t)P.nx * P.ny * P.nv;
  const double4_32a l = make_double4_32a(left[0], left[1], left[2], left[3]);
  const double4_32a r = make_double4_32a(right[0], right[1], right[2], right[3]);
  init_step_kernel<<<(unsigned)((total + 255) / 256), 256, 0, stream>>>(P, f, x_split, l, r);
  return cudaGetLastError();
}

// Uniform Maxwellian times (1 + amplitude xi).
__global__ void init_uniform_kernel(const Params P, double2* f, const double4_32a st, const double2* xi,
                                    double amplitude) {
  const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  const size_t total = (size_t)P.nx * P.ny * P.nv;
  if (idx >= total) return;
  const int j = (int)(idx % P.nv);
  const double p[4] = {st.x, st.y, st.z, st.w};
  const double cxj = centre(P.vx_min, j % P.nvx, P.dcx);
  const double cyj = (P.dim == 2) ? centre(P.vy_min, j / P.nvx, P.dcy) : 0.0;
  double2 v = maxwell_point(P.dim, p, cxj, cyj);
  if (xi != nullptr) {
    const double2 x = xi[idx];
    v.x = __dmul_rn(v.x, __dadd_rn(1.0, __dmul_rn(amplitude, x.x)));
    v.y = __dmul_rn(v.y, __dadd_rn(1.0, __dmul_rn(amplitude, x.y)));
  }
  f[idx] = v;
}

cudaError_t launch_init_uniform(const Params& P, double2* f, const double state[4],
                                const double2* xi, double amplitude, cudaStream_t stream) {
  const size_t total = (size_t)P.nx * P.ny * P.nv;
  const double4_32a s = make_double4_32a(state[0], state[1], state[2], state[3]);
  init_uniform_kernel<<<(unsigned)((total + 255) / 256), 256, 0, stream>>>(P, f, s, xi, amplitude);
  return cudaGetLastError();
}

// Moments of the current state, one CTA per cell.
__global__ void __launch_bounds__(256) moments_kernel(const Params P, const Tables T,
                                                      const double2* __restrict__ f,
                                                      double4_32a* __restrict__ mom) {
  __shared__ double red[4 * 8];
  __shared__ double tot[4];
  const int cell = blockIdx.x;
  const double2* fc = f + (size_t)cell * P.nv;
  double s0 = 0.0, sx = 0.0, sy = 0.0, se = 0.0;
  for (int j = threadIdx.x; j < P.nv; j += 256) {
    const double2 v = fc[j];
    const double cx = T.cx[j % P.nvx], cy = T.cy[j / P.nvx];
    s0 += v.x;
    sx = fma(cx, v.x, sx);
    sy = fma(cy, v.x, sy);
    se = fma(T.coef[j].w, v.x, se) + v.y;
  }
  block_reduce4<256>(s0, sx, sy, se, red, tot);
  if (threadIdx.x == 0) {
    double q[4];
    moments_from_sums(tot[0], tot[1], tot[2], tot[3], P.dv, q);
    mom[cell] = make_double4_32a(q[0], q[1], q[2], q[3]);
  }
}

cudaError_t launch_moments(const Params& P, const Tables& T, const double2* f, double4_32a* mom,
                           cudaStream_t stream) {
  moments_kernel<<<P.nx * P.ny, 256, 0, stream>>>(P, T, f, mom);
  return cudaGetLastError();
}

// Fluxes through one face, one CTA per face cell.  The crossing value is the
// cell's own state for c_n < 0 and the boundary value for c_n > 0; diffuse
// faces first get n_W from the incident flux (zero net mass flux).
__global__ void __launch_bounds__(256) wall_flux_kernel(const Params P, const Tables T,
                                                        const double2* __restrict__ f, int face,
                                                        double4_32a* __restrict__ out) {
  __shared__ double red[4 * 8];
  __shared__ double tot[4];
  const int k = blockIdx.x;
  int cell;
  switch (face) {
    case XLO: cell = k * P.nx; break;
    case XHI: cell = k * P.nx + P.nx - 1; break;
    case YLO: cell = k; break;
    default: cell = (P.ny - 1) * P.nx + k; break;
  }
  const double2* fc = f + (size_t)cell * P.nv;
  auto cn_of = [&](int j) {
    const double cx = T.cx[j % P.nvx], cy = T.cy[j / P.nvx];
    return face == XLO ? cx : face == XHI ? -cx : face == YLO ? cy : -cy;
  };
  double nw = 0.0;
  if (P.bc_kind[face] == BC_DIFFUSE) {
    double inc = 0.0;
    for (int j = threadIdx.x; j < P.nv; j += 256) {
      const double cn = cn_of(j);
      if (cn < 0.0) inc = fma(-cn, fc[j].x, inc);
    }
    block_reduce4<256>(inc, 0.0, 0.0, 0.0, red, tot);
    nw = tot[0] * P.dv / T.emitted[face];
  }
  double m = 0.0, s = 0.0, pn = 0.0, e = 0.0;
  for (int j = threadIdx.x; j < P.nv; j += 256) {
    const double cx = T.cx[j % P.nvx], cy = T.cy[j / P.nvx];
    const double cn = cn_of(j);
    const double ct = (face == XLO || face == XHI) ? cy : cx;
    const double2 F = (cn < 0.0) ? fc[j] : ghost_value(P, T, face, j, nw, fc);
    m = fma(cn, F.x, m);
    s = fma(ct * cn, F.x, s);
    pn = fma(cn * cn, F.x, pn);
    e = fma(cn, fma(T.coef[j].w, F.x, F.y), e);
  }
  block_reduce4<256>(m, s, pn, e, red, tot);
  if (threadIdx.x == 0) out[k] = make_double4_32a(tot[0] * P.dv, tot[1] * P.dv, tot[2] * P.dv, tot[3] * P.dv);
}

cudaError_t launch_wall_fluxes(const Params& P, const Tables& T, const double2* f, int face,
                               double4_32a* out, cudaStream_t stream) {
  const int ncells = (face == XLO || face == XHI) ? P.ny : P.nx;
  wall_flux_kernel<<<ncells, 256, 0, stream>>>(P, T, f, face, out);
  return cudaGetLastError();
}

}  // namespace bgk
