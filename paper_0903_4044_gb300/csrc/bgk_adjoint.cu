// bgk_adjoint.cu - reverse pass of the FP64 2D split step for the
// lid-integrated shear J = sum over the cells of face YHI of dx * tau_k, with
// tau_k = dv sum_j c_t c_n F_j the shear flux through the lid (F the cell's
// state for c_n < 0, the diffuse-wall value n_W Phi_W for c_n > 0).
//
// Per step n (f^n -> f~ -> f^{n+1}) the adjoint lambda^{n+1} of f^{n+1} is
// carried back in two kernels:
//   adj_collide  f^{n+1} = f~ + a (Phi(p) - f~), a = 1 - exp(-nu dt),
//                nu = n theta^(1-omega), p the effective parameters of the
//                moments q of f~ (the map p(q) is linearised by the identity:
//                its exact Jacobian differs from it by the quadrature
//                residual of the velocity grid):
//                  lambda~ = (1 - a) lambda' + (dq/df~)^T mu,
//                  mu = a (dPhi/dp)^T lambda' + (da/dq)^T <lambda', Phi - f~>;
//   adj_stream   the transposed donor cell: each f^n value receives the
//                adjoints of the f~ values it fed (its own cell with a0, the
//                downwind neighbours with ax, ay), and wall-adjacent cells
//                receive the adjoint of the diffuse-wall density n_W, which
//                is linear in their incident half; specular walls mirror.
// Derivatives with respect to the domain scale L (lengths and the Courant
// time step scale together, Kn = 1/L) and the lid speed U_W accumulate per
// cell in fixed order, so results are deterministic.
#include "bgk_device.cuh"

namespace bgk {

namespace {

constexpr int kB = 256;  // threads per CTA, one CTA per cell

__device__ __forceinline__ double face_cn(int face, double cx, double cy) {
  return face == XLO ? cx : face == XHI ? -cx : face == YLO ? cy : -cy;
}
__device__ __forceinline__ int reflect(const Params& P, int face, int j) {
  const int jx = j % P.nvx, jy = j / P.nvx;
  return (face == XLO || face == XHI) ? jy * P.nvx + (P.nvx - 1 - jx) : (P.nvy - 1 - jy) * P.nvx + jx;
}

// Block sum of 8 values (two block_reduce4 calls); totals in out[0..7].
__device__ __forceinline__ void block_reduce8(const double (&v)[8], double* red, double* out) {
  block_reduce4<kB>(v[0], v[1], v[2], v[3], red, out);
  double a[4] = {out[0], out[1], out[2], out[3]};
  __syncthreads();
  block_reduce4<kB>(v[4], v[5], v[6], v[7], red, out + 4);
  if (threadIdx.x < 4) out[threadIdx.x] = a[threadIdx.x];
  __syncthreads();
}

// n_W of every diffuse face the cell touches, from its own f (all threads).
__device__ void wall_densities(const Params& P, const Tables& T, const double2* fc, int ix, int iy,
                               double* red, double* tot, double nw[4]) {
  double inc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int j = threadIdx.x; j < P.nv; j += kB) {
    const double2 c = T.cxy[j];
    const double g = fc[j].x;
    for (int f = 0; f < 4; ++f) {
      const double cn = face_cn(f, c.x, c.y);
      if (cn < 0.0) inc[f] = fma(-cn, g, inc[f]);
    }
  }
  block_reduce4<kB>(inc[0], inc[1], inc[2], inc[3], red, tot);
  const bool touch[4] = {ix == 0, ix == P.nx - 1, iy == 0, iy == P.ny - 1};
  for (int f = 0; f < 4; ++f)
    nw[f] = (touch[f] && P.bc_kind[f] == BC_DIFFUSE) ? tot[f] * P.dv / T.emitted[f] : 0.0;
}

// f~ at velocity j of cell (ix, iy) (the forward's donor-cell update).
__device__ __forceinline__ double2 stream_point(const Params& P, const Tables& T, const double2* fin,
                                                int cell, int ix, int iy, int j, const double nw[4]) {
  const double2* fc = fin + (size_t)cell * P.nv;
  const double2 c = T.cxy[j];
  const double4_32a co = T.coef[j];
  const double2 f0 = fc[j];
  double2 fx = f0, fy = f0;
  auto ghost = [&](int face) {
    const int kind = P.bc_kind[face];
    if (kind == BC_SPECULAR) return fc[reflect(P, face, j)];
    const double2 gv = T.ghost[face * P.nv + j];
    return kind == BC_DIFFUSE ? make_double2(nw[face] * gv.x, nw[face] * gv.y) : gv;
  };
  if (c.x > 0.0) fx = ix > 0 ? fc[j - P.nv] : ghost(XLO);
  else if (c.x < 0.0) fx = ix < P.nx - 1 ? fc[j + P.nv] : ghost(XHI);
  const size_t row = (size_t)P.nx * P.nv;
  if (c.y > 0.0) fy = iy > 0 ? fc[j - row] : ghost(YLO);
  else if (c.y < 0.0) fy = iy < P.ny - 1 ? fc[j + row] : ghost(YHI);
  double2 ft;
  ft.x = fma(co.z, fy.x, fma(co.y, fx.x, co.x * f0.x));
  ft.y = fma(co.z, fy.y, fma(co.y, fx.y, co.x * f0.y));
  return ft;
}

// Effective parameters p with D(p) = q (one warp, exact Gaussians per
// iteration, the same stopping rule as the forward); factors in ex, ey.
__device__ bool effective_warp(const Params& P, const Tables& T, const double q[4], double p[4],
                               double* ex, double* ey) {
  const int lane = threadIdx.x & 31;
  for (int k = 0; k < 4; ++k) p[k] = q[k];
  const double vs = sqrt(q[3]);
  double r = 1.0;
  for (int it = 1; it <= kEffMaxIt && P.conservative; ++it) {
    const double inv = 1.0 / p[3];
    double s[6] = {0, 0, 0, 0, 0, 0};
    for (int j = lane; j < P.nvx; j += 32) {
      const double d = T.cx[j] - p[1], e = exp(-(d * d) * inv);
      s[0] += e;
      s[1] = fma(d, e, s[1]);
      s[2] = fma(d * d, e, s[2]);
    }
    for (int j = lane; j < P.nvy; j += 32) {
      const double d = T.cy[j] - p[2], e = exp(-(d * d) * inv);
      s[3] += e;
      s[4] = fma(d, e, s[4]);
      s[5] = fma(d * d, e, s[5]);
    }
    for (int k = 0; k < 6; ++k)
      for (int m = 16; m > 0; m >>= 1) s[k] += __shfl_xor_sync(0xffffffffu, s[k], m);
    const double mux = s[1] / s[0], muy = s[4] / s[3];
    double d[4];
    d[0] = p[0] / (kPi() * p[3]) * P.dv * s[0] * s[3];
    d[1] = p[1] + mux;
    d[2] = p[2] + muy;
    d[3] = (2.0 / 3.0) * ((s[2] / s[0] - mux * mux) + (s[5] / s[3] - muy * muy) + 0.5 * p[3]);
    r = 0.0;
    for (int k = 0; k < 4; ++k) {
      const double delta = q[k] - d[k];
      p[k] += delta;
      r = fmax(r, fabs(delta) / (k == 0 ? q[0] : k == 3 ? q[3] : vs));
    }
    if (!(p[0] > 0.0) || !(p[3] > 0.0) || !isfinite(r)) return false;
    if (r < kEffTol) break;
    if (it == kEffMaxIt && r >= kEffFail) return false;
  }
  const double inv = 1.0 / p[3], pref = p[0] / (kPi() * p[3]);
  for (int j = lane; j < P.nvx; j += 32) {
    const double d = T.cx[j] - p[1];
    ex[j] = pref * exp(-(d * d) * inv);
  }
  for (int j = lane; j < P.nvy; j += 32) {
    const double d = T.cy[j] - p[2];
    ey[j] = exp(-(d * d) * inv);
  }
  return true;
}

}  // namespace

// lambda~ from lambda^{n+1} for one cell; dlnl[cell] accumulates the
// domain-scale derivative (dt scales with L).
__global__ void __launch_bounds__(kB) adj_collide_kernel(const Params P, const Tables T,
                                                         const double2* __restrict__ fin,
                                                         const double2* __restrict__ lam,
                                                         double2* __restrict__ lamt, double* __restrict__ dlnl,
                                                         int* __restrict__ err) {
  extern __shared__ double sh[];
  double* ex = sh;
  double* ey = sh + P.nvx;
  __shared__ double red[32], tot[8], sc[8];
  const int cell = blockIdx.x, ix = cell % P.nx, iy = cell / P.nx;
  const double2* fc = fin + (size_t)cell * P.nv;
  double nw[4];
  wall_densities(P, T, fc, ix, iy, red, tot, nw);
  // moments of f~
  double s0 = 0.0, sx = 0.0, sy = 0.0, se = 0.0;
  for (int j = threadIdx.x; j < P.nv; j += kB) {
    const double2 ft = stream_point(P, T, fin, cell, ix, iy, j, nw);
    const double2 c = T.cxy[j];
    s0 += ft.x;
    sx = fma(c.x, ft.x, sx);
    sy = fma(c.y, ft.x, sy);
    se = fma(T.coef[j].w, ft.x, se) + ft.y;
  }
  block_reduce4<kB>(s0, sx, sy, se, red, tot);
  double q[4];
  moments_from_sums(tot[0], tot[1], tot[2], tot[3], P.dv, q);
  const double E = tot[3] * P.dv;
  if (threadIdx.x < 32) {
    double p[4] = {q[0], q[1], q[2], q[3]};
    const bool ok = moments_ok(q) && effective_warp(P, T, q, p, ex, ey);
    if (threadIdx.x == 0) {
      sc[0] = p[0];
      sc[1] = p[1];
      sc[2] = p[2];
      sc[3] = p[3];
      sc[4] = ok ? 1.0 : 0.0;
      if (!ok) atomicOr(err, ERR_MOMENT);
    }
  }
  __syncthreads();
  const double p0 = sc[0], p1 = sc[1], p2 = sc[2], p3 = sc[3];
  const double nu = q[0] * pow(q[3], 1.0 - P.omega);
  const double e = exp(-nu * P.dt), a = 1.0 - e;
  // s_a = <lambda', Phi - f~>, s_p = (dPhi/dp)^T lambda'
  double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const double2* lc = lam + (size_t)cell * P.nv;
  for (int j = threadIdx.x; j < P.nv; j += kB) {
    const double2 ft = stream_point(P, T, fin, cell, ix, iy, j, nw);
    const double2 c = T.cxy[j];
    const double G = ex[j % P.nvx] * ey[j / P.nvx], H = 0.5 * p3 * G;
    const double2 l = lc[j];
    v[0] += l.x * (G - ft.x) + l.y * (H - ft.y);
    const double dxp = c.x - p1, dyp = c.y - p2;
    const double dG[4] = {G / p0, G * 2.0 * dxp / p3, G * 2.0 * dyp / p3,
                          G * ((dxp * dxp + dyp * dyp) / (p3 * p3) - 1.0 / p3)};
    for (int k = 0; k < 4; ++k) {
      const double dH = 0.5 * p3 * dG[k] + (k == 3 ? 0.5 * G : 0.0);
      v[1 + k] += l.x * dG[k] + l.y * dH;
    }
  }
  __syncthreads();
  block_reduce8(v, red, tot);
  const double sa = tot[0];
  const double da_dn = P.dt * e * pow(q[3], 1.0 - P.omega);
  const double da_dth = P.dt * e * (1.0 - P.omega) * q[0] * pow(q[3], -P.omega);
  const double mu[4] = {a * tot[1] + da_dn * sa, a * tot[2], a * tot[3], a * tot[4] + da_dth * sa};
  if (threadIdx.x == 0) dlnl[cell] += sa * nu * P.dt * e;
  const double n = q[0], ux = q[1], uy = q[2];
  double2* lt = lamt + (size_t)cell * P.nv;
  for (int j = threadIdx.x; j < P.nv; j += kB) {
    const double2 c = T.cxy[j];
    const double2 l = lc[j];
    const double dux = P.dv * (c.x - ux) / n, duy = P.dv * (c.y - uy) / n;
    const double dth = (2.0 / 3.0) * (P.dv / n) *
                       (T.coef[j].w - E / n - 2.0 * (ux * (c.x - ux) + uy * (c.y - uy)));
    lt[j] = make_double2((1.0 - a) * l.x + mu[0] * P.dv + mu[1] * dux + mu[2] * duy + mu[3] * dth,
                         (1.0 - a) * l.y + mu[3] * (2.0 / 3.0) * P.dv / n);
  }
}

// lambda^n from lambda~ for one cell (transposed streaming); duw[ix]
// accumulates the lid-speed derivative for lid cells.
__global__ void __launch_bounds__(kB) adj_stream_kernel(const Params P, const Tables T,
                                                        const double2* __restrict__ fin,
                                                        const double2* __restrict__ lamt,
                                                        double2* __restrict__ lam_out,
                                                        const double2* __restrict__ dghost_lid, double demit_lid,
                                                        double* __restrict__ duw) {
  __shared__ double red[32], tot[8];
  const int cell = blockIdx.x, ix = cell % P.nx, iy = cell / P.nx;
  const double2* fc = fin + (size_t)cell * P.nv;
  const size_t row = (size_t)P.nx * P.nv;
  const double2* lt = lamt + (size_t)cell * P.nv;
  const bool touch[4] = {ix == 0, ix == P.nx - 1, iy == 0, iy == P.ny - 1};
  double nw[4];
  wall_densities(P, T, fc, ix, iy, red, tot, nw);
  // adjoints of the diffuse-wall values this cell used, and the lid speed
  double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int j = threadIdx.x; j < P.nv; j += kB) {
    const double2 c = T.cxy[j];
    const double4_32a co = T.coef[j];
    const double2 l = lt[j];
    for (int f = 0; f < 4; ++f) {
      if (!touch[f] || P.bc_kind[f] != BC_DIFFUSE) continue;
      if (face_cn(f, c.x, c.y) <= 0.0) continue;  // entering from face f
      const double w = (f < 2) ? co.y : co.z;
      const double2 gw = T.ghost[f * P.nv + j];
      v[f] += w * (l.x * gw.x + l.y * gw.y);
      if (f == YHI) {
        const double2 dg = dghost_lid[j];
        const double egx = dg.x - gw.x * demit_lid / T.emitted[YHI];
        const double egy = dg.y - gw.y * demit_lid / T.emitted[YHI];
        v[4] += w * nw[YHI] * (l.x * egx + l.y * egy);
      }
    }
  }
  block_reduce8(v, red, tot);
  if (threadIdx.x == 0 && touch[YHI] && P.bc_kind[YHI] == BC_DIFFUSE) duw[ix] += tot[4];
  double2* lo = lam_out + (size_t)cell * P.nv;
  for (int j = threadIdx.x; j < P.nv; j += kB) {
    const double2 c = T.cxy[j];
    const double4_32a co = T.coef[j];
    double2 r = make_double2(co.x * lt[j].x, co.x * lt[j].y);
    // downwind neighbours used this value as their upwind source
    if (c.x > 0.0 && ix < P.nx - 1) {
      const double2 d = lt[j + P.nv];
      r.x = fma(co.y, d.x, r.x);
      r.y = fma(co.y, d.y, r.y);
    } else if (c.x < 0.0 && ix > 0) {
      const double2 d = lt[(ptrdiff_t)j - P.nv];
      r.x = fma(co.y, d.x, r.x);
      r.y = fma(co.y, d.y, r.y);
    }
    if (c.y > 0.0 && iy < P.ny - 1) {
      const double2 d = lt[j + row];
      r.x = fma(co.z, d.x, r.x);
      r.y = fma(co.z, d.y, r.y);
    } else if (c.y < 0.0 && iy > 0) {
      const double2 d = lt[(ptrdiff_t)j - (ptrdiff_t)row];
      r.x = fma(co.z, d.x, r.x);
      r.y = fma(co.z, d.y, r.y);
    }
    for (int f = 0; f < 4; ++f) {
      if (!touch[f]) continue;
      const double cn = face_cn(f, c.x, c.y);
      if (P.bc_kind[f] == BC_DIFFUSE && cn < 0.0) {
        // n_W = dv sum_{c_n<0} |c_n| g / emitted
        r.x = fma(tot[f] * P.dv / T.emitted[f], -cn, r.x);
      } else if (P.bc_kind[f] == BC_SPECULAR && cn < 0.0) {
        // this value was mirrored into the entering velocity reflect(j)
        const int jr = reflect(P, f, j);
        const double w = (f < 2) ? T.coef[jr].y : T.coef[jr].z;
        r.x = fma(w, lt[jr].x, r.x);
        r.y = fma(w, lt[jr].y, r.y);
      }
    }
    lo[j] = r;
  }
}

// Objective seed on f^N: lambda^N = dJ/df^N (lid cells), J_k = dx tau_k and
// the explicit lid-speed derivative per lid cell.  One CTA per lid cell.
__global__ void __launch_bounds__(kB) adj_seed_kernel(const Params P, const Tables T,
                                                      const double2* __restrict__ f, double2* __restrict__ lam,
                                                      const double2* __restrict__ dghost_lid, double demit_lid,
                                                      double* __restrict__ Jk, double* __restrict__ duw) {
  __shared__ double red[32], tot[8];
  const int k = blockIdx.x;
  const int cell = (P.ny - 1) * P.nx + k;
  const double2* fc = f + (size_t)cell * P.nv;
  double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int j = threadIdx.x; j < P.nv; j += kB) {
    const double2 c = T.cxy[j];
    const double cn = -c.y, ct = c.x;
    if (cn < 0.0) {
      v[0] = fma(-cn, fc[j].x, v[0]);     // incident flux
      v[1] = fma(ct * cn, fc[j].x, v[1]);  // incident shear
    } else {
      const double2 gw = T.ghost[YHI * P.nv + j];
      v[2] = fma(ct * cn, gw.x, v[2]);          // emitted shear per unit n_W
      v[3] = fma(ct * cn, dghost_lid[j].x, v[3]);
    }
  }
  block_reduce8(v, red, tot);
  const double emit = T.emitted[YHI];
  const double nw = tot[0] * P.dv / emit;
  const double shear_w = tot[2] * P.dv, dshear_w = tot[3] * P.dv;
  if (threadIdx.x == 0) {
    Jk[k] = P.dx * P.dv * (tot[1] + nw * tot[2]);
    duw[k] = P.dx * nw * (dshear_w - shear_w * demit_lid / emit);
  }
  double2* lc = lam + (size_t)cell * P.nv;
  for (int j = threadIdx.x; j < P.nv; j += kB) {
    const double2 c = T.cxy[j];
    const double cn = -c.y, ct = c.x;
    if (cn < 0.0) lc[j] = make_double2(P.dx * (ct * cn * P.dv + shear_w * (-cn) * P.dv / emit), 0.0);
  }
}

// d Phi_W / d U_W of the lid (unit density) and its emitted-flux derivative.
__global__ void __launch_bounds__(kB) adj_lid_table_kernel(const Params P, const Tables T, double2* dghost,
                                                           double* demit) {
  __shared__ double red[32], tot[4];
  const double th = P.bc_state[YHI][3], uw = P.bc_state[YHI][1];
  double s = 0.0;
  for (int j = threadIdx.x; j < P.nv; j += kB) {
    const double2 c = T.cxy[j];
    const double2 gw = T.ghost[YHI * P.nv + j];
    const double dg = gw.x * 2.0 * (c.x - uw) / th;
    dghost[j] = make_double2(dg, 0.5 * th * dg);
    if (-c.y > 0.0) s = fma(-c.y, dg, s);
  }
  block_reduce4<kB>(s, 0.0, 0.0, 0.0, red, tot);
  if (threadIdx.x == 0) *demit = tot[0] * P.dv;
}

cudaError_t launch_adj_lid_table(const Params& P, const Tables& T, double2* dghost, double* demit,
                                 cudaStream_t stream) {
  adj_lid_table_kernel<<<1, kB, 0, stream>>>(P, T, dghost, demit);
  return cudaGetLastError();
}

cudaError_t launch_adj_seed(const Params& P, const Tables& T, const double2* f, double2* lam,
                            const double2* dghost, double demit, double* Jk, double* duw, cudaStream_t stream) {
  adj_seed_kernel<<<P.nx, kB, 0, stream>>>(P, T, f, lam, dghost, demit, Jk, duw);
  return cudaGetLastError();
}

cudaError_t launch_adj_step(const Params& P, const Tables& T, const double2* fn, const double2* lam_next,
                            double2* lamt, double2* lam_out, const double2* dghost, double demit,
                            double* dlnl, double* duw, int* err, cudaStream_t stream) {
  const int ncell = P.nx * P.ny;
  adj_collide_kernel<<<ncell, kB, sizeof(double) * (P.nvx + P.nvy), stream>>>(P, T, fn, lam_next, lamt, dlnl,
                                                                              err);
  adj_stream_kernel<<<ncell, kB, 0, stream>>>(P, T, fn, lamt, lam_out, dghost, demit, duw);
  return cudaGetLastError();
}

}  // namespace bgk
