// bgk_adjoint.cu - reverse pass of the FP64 2D split step for the
// lid-integrated shear J = sum over the cells of face YHI of dx * tau_k, with
// tau_k = dv sum_j c_t c_n F_j the shear flux through the lid (F the cell's
// state for c_n < 0, the diffuse-wall value n_W Phi_W for c_n > 0).
//
// Step n maps f^n -> f~ (donor-cell streaming, Eq. upwind in its unsplit 2D
// form, with the wall values of Eq. bc_cavity) -> f^{n+1} (relaxation,
// Eq. relaxation).  With lambda the adjoint of f, one reverse launch per
// step and cell does
//   1. the streaming adjoint of step n+1: lambda^{n+1} at this cell gathers
//      lambda~^{n+1} of the cells its values fed (itself with a0, the
//      downwind neighbours with ax, ay) plus, at walls, the adjoint of the
//      diffuse-wall density n_W (linear in the cell's incident half of
//      f^{n+1}) and of the specular mirror;
//   2. the collision adjoint of step n, f^{n+1} = f~ + a (Phi(p) - f~),
//      a = 1 - exp(-nu dt), nu = n theta^(1-omega), p the effective
//      parameters of the moments q of f~ (the map p(q) linearised by the
//      identity: its Jacobian differs from it by the quadrature residual of
//      the velocity grid):
//        lambda~ = (1 - a) lambda + (dq/df~)^T mu,
//        mu = a (dPhi/dp)^T lambda + (da/dq)^T <lambda, Phi - f~>.
//      (dPhi/dp)^T lambda needs only the sums of G L (1, c_x, c_y, |c|^2)
//      and of G lambda_h, with L = lambda_g + theta_p/2 lambda_h, and
//      (dq/df~)^T mu is a polynomial in (1, c_x, c_y, |c|^2) per cell, so
//      the per-velocity work is a few FMAs.  q and p of step n come from the
//      forward kernel of the recomputed segment.
// Derivatives with respect to the domain scale L (lengths and the Courant
// time step scale together, Kn = 1/L) and the lid speed U_W accumulate per
// cell in a fixed order, so results are deterministic.
#include "bgk_device.cuh"

namespace bgk {

namespace {

constexpr int kB = 256;  // threads per CTA, one CTA per cell
constexpr int kNW = kB / 32;

__device__ __forceinline__ double face_cn(int face, double cx, double cy) {
  return face == XLO ? cx : face == XHI ? -cx : face == YLO ? cy : -cy;
}
__device__ __forceinline__ int reflect(const Params& P, int face, int j) {
  const int jx = j % P.nvx, jy = j / P.nvx;
  return (face == XLO || face == XHI) ? jy * P.nvx + (P.nvx - 1 - jx) : (P.nvy - 1 - jy) * P.nvx + jx;
}

// Block sums of N values in a fixed order; totals in out[0..N-1] (all threads).
template <int N>
__device__ __forceinline__ void block_sum(double (&v)[N], double* red, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < N; ++k)
    for (int m = 16; m > 0; m >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], m);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < N; ++k) red[warp * N + k] = v[k];
  __syncthreads();
  if (threadIdx.x < N) {
    double t = 0.0;
    for (int w = 0; w < kNW; ++w) t += red[w * N + threadIdx.x];
    out[threadIdx.x] = t;
  }
  __syncthreads();
}

// Faces of the cell that are diffuse walls (bit f set).
__device__ __forceinline__ int diffuse_faces(const Params& P, int ix, int iy) {
  const bool touch[4] = {ix == 0, ix == P.nx - 1, iy == 0, iy == P.ny - 1};
  int m = 0;
  for (int f = 0; f < 4; ++f)
    if (touch[f] && P.bc_kind[f] == BC_DIFFUSE) m |= 1 << f;
  return m;
}

// Warp totals of eight values, valid in every lane (recursive halving, then
// a broadcast from the lane holding each total).
__device__ __forceinline__ void warp_total8(const double (&v)[8], double (&t)[8]) {
  const double x = warp_reduce8(v);
#pragma unroll
  for (int k = 0; k < 8; ++k) t[k] = __shfl_sync(0xffffffffu, x, 4 * k);
}

// n_W of every diffuse face the cell touches, from its own f (Eq. bc_cavity:
// the emitted flux equals the incident one).  One warp, all lanes.
__device__ void wall_densities(const Params& P, const Tables& T, const double2* fc, int dmask, double nw[4]) {
  const int lane = threadIdx.x & 31;
  double inc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int j = lane; j < P.nv; j += 32) {
    const double2 c = T.cxy[j];
    const double g = fc[j].x;
    for (int f = 0; f < 4; ++f) {
      const double cn = face_cn(f, c.x, c.y);
      if (cn < 0.0) inc[f] = fma(-cn, g, inc[f]);
    }
  }
  double t[8];
  warp_total8(inc, t);
  for (int f = 0; f < 4; ++f) nw[f] = (dmask >> f & 1) ? t[f] * P.dv / T.emitted[f] : 0.0;
}

// Signs of c_x, c_y of velocity j from its vinfo entry (-1, 0, 1): integer
// tests keep the branches off the FP64 pipe.
__device__ __forceinline__ int sgn_x(int vi) { return ((vi >> 24) & 3) - 1; }
__device__ __forceinline__ int sgn_y(int vi) { return ((vi >> 26) & 3) - 1; }

// lambda at every velocity of one cell from lambda~ (the transposed
// donor-cell update); adjw: adjoint of each diffuse face's n_W per unit
// incident flux.  EDGE as in stream_point.
template <bool EDGE>
__device__ __forceinline__ void gather_adjoint(const Params& P, const Tables& T, int ix, int iy,
                                               const double2* __restrict__ lt, const double adjw[4], int dmask,
                                               double2* dst) {
  const int lane = threadIdx.x & 31;
  const size_t row = (size_t)P.nx * P.nv;
  const bool touch[4] = {ix == 0, ix == P.nx - 1, iy == 0, iy == P.ny - 1};
  for (int j = lane; j < P.nv; j += 32) {
    const int vi = T.vinfo[j];
    const int sx = sgn_x(vi), sy = sgn_y(vi);
    const double4_32a co = T.coef[j];
    const double2 l0 = lt[j];
    double2 r = make_double2(co.x * l0.x, co.x * l0.y);
    // downwind neighbours used this value as their upwind source
    if (!EDGE) {
      if (sx != 0) {
        const double2 d = lt[sx > 0 ? (ptrdiff_t)j + P.nv : (ptrdiff_t)j - P.nv];
        r.x = fma(co.y, d.x, r.x);
        r.y = fma(co.y, d.y, r.y);
      }
      if (sy != 0) {
        const double2 d = lt[sy > 0 ? (ptrdiff_t)j + (ptrdiff_t)row : (ptrdiff_t)j - (ptrdiff_t)row];
        r.x = fma(co.z, d.x, r.x);
        r.y = fma(co.z, d.y, r.y);
      }
    } else {
      if (sx > 0 && ix < P.nx - 1) {
        const double2 d = lt[j + P.nv];
        r.x = fma(co.y, d.x, r.x);
        r.y = fma(co.y, d.y, r.y);
      } else if (sx < 0 && ix > 0) {
        const double2 d = lt[(ptrdiff_t)j - P.nv];
        r.x = fma(co.y, d.x, r.x);
        r.y = fma(co.y, d.y, r.y);
      }
      if (sy > 0 && iy < P.ny - 1) {
        const double2 d = lt[j + row];
        r.x = fma(co.z, d.x, r.x);
        r.y = fma(co.z, d.y, r.y);
      } else if (sy < 0 && iy > 0) {
        const double2 d = lt[(ptrdiff_t)j - (ptrdiff_t)row];
        r.x = fma(co.z, d.x, r.x);
        r.y = fma(co.z, d.y, r.y);
      }
      for (int fc = 0; fc < 4; ++fc) {
        if (!touch[fc]) continue;
        const double2 c = T.cxy[j];
        const double cn = face_cn(fc, c.x, c.y);
        if (cn >= 0.0) continue;  // only incident values feed a wall
        if (dmask >> fc & 1) {
          r.x = fma(adjw[fc], -cn, r.x);
        } else if (P.bc_kind[fc] == BC_SPECULAR) {
          // mirrored into the entering velocity reflect(j)
          const int jr = reflect(P, fc, j);
          const double w = (fc < 2) ? T.coef[jr].y : T.coef[jr].z;
          r.x = fma(w, lt[jr].x, r.x);
          r.y = fma(w, lt[jr].y, r.y);
        }
      }
    }
    dst[j] = r;
  }
}

// Streaming adjoint of one step at one cell (one warp): lambda at every
// velocity of the cell from lambda~ of the cells its values fed, written to
// dst.  f = the step's input state (wall densities).
__device__ void stream_adjoint(const Params& P, const Tables& T, int cell, int ix, int iy, int dmask,
                               const double2* __restrict__ f, const double2* __restrict__ lam_t,
                               const double2* __restrict__ dghost, double demit, double* __restrict__ duw,
                               double2* dst) {
  const int lane = threadIdx.x & 31;
  const size_t base = (size_t)cell * P.nv;
  const double2* lt = lam_t + base;
  const bool edge = ix == 0 || ix == P.nx - 1 || iy == 0 || iy == P.ny - 1;
  double adjw[4] = {0.0, 0.0, 0.0, 0.0};  // adjoint of n_W per diffuse face, per unit incident flux
  if (dmask) {
    double nw[4];
    wall_densities(P, T, f + base, dmask, nw);
    double v[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int j = lane; j < P.nv; j += 32) {
      const double2 c = T.cxy[j];
      const double4_32a co = T.coef[j];
      const double2 l = lt[j];
      for (int fc = 0; fc < 4; ++fc) {
        if (!(dmask >> fc & 1) || face_cn(fc, c.x, c.y) <= 0.0) continue;  // entering from face fc
        const double w = (fc < 2) ? co.y : co.z;
        const double2 gw = T.ghost[fc * P.nv + j];
        v[fc] = fma(w, l.x * gw.x + l.y * gw.y, v[fc]);
        if (fc == YHI) {
          const double2 dg = dghost[j];
          const double r = demit / T.emitted[YHI];
          v[4] = fma(w * nw[YHI], l.x * (dg.x - gw.x * r) + l.y * (dg.y - gw.y * r), v[4]);
        }
      }
    }
    double t[8];
    warp_total8(v, t);
    if (lane == 0 && (dmask >> YHI & 1)) duw[ix] += t[4];
    for (int fc = 0; fc < 4; ++fc) adjw[fc] = (dmask >> fc & 1) ? t[fc] * P.dv / T.emitted[fc] : 0.0;
  }
  if (edge) gather_adjoint<true>(P, T, ix, iy, lt, adjw, dmask, dst);
  else gather_adjoint<false>(P, T, ix, iy, lt, adjw, dmask, dst);
}

// Sums over the velocities of one cell for the collision adjoint (one
// warp, lane partials): s = (G L, G L c_x, G L c_y, G L |c|^2, G lambda_h,
// <lambda, f^{n+1}>), L = lambda_g + theta_p/2 lambda_h.  Since
// f^{n+1} = f~ + a (Phi - f~), <lambda, Phi - f~> = <lambda, Phi - f^{n+1}> / e
// with e = 1 - a: the cell's own f^{n+1} replaces the streamed f~.
__device__ __forceinline__ void collide_sums(const Params& P, const Tables& T, const double2* f1, const double* ex,
                                             const double* ey, const double2* sl, double hp, double (&s)[8]) {
  const int lane = threadIdx.x & 31;
  for (int j = lane; j < P.nv; j += 32) {
    const int vi = T.vinfo[j];
    const double2 c = T.cxy[j];
    const double G = ex[vi & 0xfff] * ey[(vi >> 12) & 0xfff];  // jx, jy of velocity j
    const double2 l = sl[j];
    const double2 f = f1[j];
    const double GL = G * fma(hp, l.y, l.x);
    s[0] += GL;
    s[1] = fma(GL, c.x, s[1]);
    s[2] = fma(GL, c.y, s[2]);
    s[3] = fma(GL, T.coef[j].w, s[3]);
    s[4] = fma(G, l.y, s[4]);
    s[5] = fma(l.x, f.x, fma(l.y, f.y, s[5]));
  }
}

}  // namespace

// One reverse step, G cells per CTA, one warp per cell.
//   tilde = 0: lam_in holds lambda^{n+1} itself (the objective's seed);
//   tilde = 1: lam_in holds lambda~^{n+1}; fn1 = f^{n+1} feeds the wall terms.
//   collide = 1: out = lambda~^n (needs qn, pn of step n; fn1 = f^{n+1});
//   collide = 0: out = lambda^{n+1} (the last launch, giving lambda^0).
// dghost, demit: d/dU_W of the lid's unit Maxwellian and of its emitted flux.
// The per-cell coefficients are computed cells-in-lanes by warp 0.  Six
// CTAs per SM hold it to 80 registers without spills (105 unbounded):
// 3.881 -> 3.846 s per 128^2 x 32^2, 2000-step gradient.
template <int G>
__global__ void __launch_bounds__(32 * G, 6) adj_step_kernel(const Params P, const Tables T,
                                                          const double2* __restrict__ fn1,
                                                          const double4_32a* __restrict__ qn,
                                                          const double4_32a* __restrict__ pn,
                                                          const double2* __restrict__ lam_in, int tilde,
                                                          int collide, double2* __restrict__ out,
                                                          const double2* __restrict__ dghost, double demit,
                                                          double* __restrict__ dlnl, double* __restrict__ duw) {
  extern __shared__ double sh[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ncell = P.nx * P.ny, nvxy = P.nvx + P.nvy;
  double* ex = sh + (size_t)warp * nvxy;  // n/(pi theta) e^{-(c_x-u_x)^2/theta}
  double* ey = ex + P.nvx;                // e^{-(c_y-u_y)^2/theta}
  __shared__ double s_sum[G][8], s_cf[G][5];
  const int cell = blockIdx.x * G + warp;
  const bool live = cell < ncell;
  const int ix = cell % P.nx, iy = cell / P.nx;
  const size_t base = (size_t)cell * P.nv;
  const int dmask = live ? diffuse_faces(P, ix, iy) : 0;

  // 1. lambda^{n+1} at this cell, parked in the cell's output slots (each
  // lane rereads only what it wrote; shared-memory staging, 16 B per
  // velocity, held an SM to 3 CTAs)
  double2* sl = out + base;
  if (live) {
    double2* dst = sl;
    if (tilde) {
      stream_adjoint(P, T, cell, ix, iy, dmask, fn1, lam_in, dghost, demit, duw, dst);
    } else {
      for (int j = lane; j < P.nv; j += 32) dst[j] = lam_in[base + j];
    }
  }
  if (!collide) return;  // uniform over the grid

  // 2. collision adjoint of step n: sums over the velocities
  double4_32a p = make_double4_32a(1.0, 0.0, 0.0, 1.0);
  if (live) {
    p = pn[cell];
    const double inv = 1.0 / p.w, pref = p.x / (kPi() * p.w);
    for (int j = lane; j < nvxy; j += 32) {
      const bool isx = j < P.nvx;
      const double d = (isx ? T.cx[j] : T.cy[j - P.nvx]) - (isx ? p.y : p.z);
      const double g = exp(-(d * d) * inv);
      ex[j] = isx ? pref * g : g;  // ey = ex + nvx
    }
    __syncwarp();
    double s[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    collide_sums(P, T, fn1 + base, ex, ey, sl, 0.5 * p.w, s);
    const double x = warp_reduce8(s);
    if ((lane & 3) == 0) s_sum[warp][lane >> 2] = x;
  }
  __syncthreads();
  // per-cell coefficients, cells in lanes (FP64 pow/exp/divides are costly)
  if (warp == 0 && lane < G && blockIdx.x * G + lane < ncell) {
    const int c = blockIdx.x * G + lane;
    const double4_32a q = qn[c], pc = pn[c];
    const double* t = s_sum[lane];
    const double n = q.x, ux = q.y, uy = q.z, th = q.w;
    const double th1 = pow(th, 1.0 - P.omega);
    const double nu = n * th1;
    const double e = exp(-nu * P.dt), a = 1.0 - e;
    const double s0 = t[0], s1 = t[1], s2 = t[2], s3 = t[3], s4 = t[4];
    const double sa = (s0 - t[5]) / e;  // <lambda, Phi - f~>
    const double ip = 1.0 / pc.w;
    const double sp0 = s0 / pc.x;
    const double sp1 = 2.0 * (s1 - pc.y * s0) * ip;
    const double sp2 = 2.0 * (s2 - pc.z * s0) * ip;
    const double sp3 =
        (s3 - 2.0 * (pc.y * s1 + pc.z * s2) + (pc.y * pc.y + pc.z * pc.z) * s0) * ip * ip - s0 * ip + 0.5 * s4;
    const double da_dn = P.dt * e * th1;
    const double da_dth = P.dt * e * (1.0 - P.omega) * n * th1 / th;
    const double mu0 = a * sp0 + da_dn * sa, mu1 = a * sp1, mu2 = a * sp2, mu3 = a * sp3 + da_dth * sa;
    const double r = P.dv / n, eon = 1.5 * th + ux * ux + uy * uy;
    const double B = (2.0 / 3.0) * r * mu3;
    s_cf[lane][0] = e;
    s_cf[lane][1] = mu0 * P.dv - r * (mu1 * ux + mu2 * uy) + B * (2.0 * (ux * ux + uy * uy) - eon);
    s_cf[lane][2] = r * (mu1 - (4.0 / 3.0) * mu3 * ux);
    s_cf[lane][3] = r * (mu2 - (4.0 / 3.0) * mu3 * uy);
    s_cf[lane][4] = B;  // coefficient of |c|^2, and the h component
    dlnl[c] += sa * nu * P.dt * e;  // dt scales with L
  }
  __syncthreads();
  if (!live) return;
  // lambda~ = e lambda + (dq/df~)^T mu, a polynomial in (1, c_x, c_y, |c|^2)
  const double e = s_cf[warp][0], A0 = s_cf[warp][1], A1 = s_cf[warp][2], A2 = s_cf[warp][3], B = s_cf[warp][4];
  double2* o = out + base;
  for (int j = lane; j < P.nv; j += 32) {
    const double2 c = T.cxy[j];
    const double2 l = sl[j];
    const double poly = fma(B, T.coef[j].w, fma(A2, c.y, fma(A1, c.x, A0)));
    o[j] = make_double2(fma(e, l.x, poly), fma(e, l.y, B));
  }
}

// Objective seed on f^N: lambda^N = dJ/df^N (lid cells), J_k = dx tau_k and
// the explicit lid-speed derivative per lid cell.  One CTA per lid cell.
__global__ void __launch_bounds__(kB) adj_seed_kernel(const Params P, const Tables T,
                                                      const double2* __restrict__ f, double2* __restrict__ lam,
                                                      const double2* __restrict__ dghost_lid, double demit_lid,
                                                      double* __restrict__ Jk, double* __restrict__ duw) {
  __shared__ double red[kNW * 4], tot[4];
  const int k = blockIdx.x;
  const int cell = (P.ny - 1) * P.nx + k;
  const double2* fc = f + (size_t)cell * P.nv;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int j = threadIdx.x; j < P.nv; j += kB) {
    const double2 c = T.cxy[j];
    const double cn = -c.y, ct = c.x;
    if (cn < 0.0) {
      v[0] = fma(-cn, fc[j].x, v[0]);     // incident flux
      v[1] = fma(ct * cn, fc[j].x, v[1]);  // incident shear
    } else {
      const double2 gw = T.ghost[YHI * P.nv + j];
      v[2] = fma(ct * cn, gw.x, v[2]);  // emitted shear per unit n_W
      v[3] = fma(ct * cn, dghost_lid[j].x, v[3]);
    }
  }
  block_sum<4>(v, red, tot);
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
  __shared__ double red[kNW], tot[1];
  const double th = P.bc_state[YHI][3], uw = P.bc_state[YHI][1];
  double s[1] = {0.0};
  for (int j = threadIdx.x; j < P.nv; j += kB) {
    const double2 c = T.cxy[j];
    const double2 gw = T.ghost[YHI * P.nv + j];
    const double dg = gw.x * 2.0 * (c.x - uw) / th;
    dghost[j] = make_double2(dg, 0.5 * th * dg);
    if (-c.y > 0.0) s[0] = fma(-c.y, dg, s[0]);
  }
  block_sum<1>(s, red, tot);
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

namespace {

size_t adj_cell_bytes(const Params& P) { return sizeof(double) * (size_t)(P.nvx + P.nvy); }

template <int G>
cudaError_t launch_adj_g(const Params& P, const Tables& T, const double2* fn1,
                         const double4_32a* qn, const double4_32a* pn, const double2* lam_in, int tilde, int collide,
                         double2* out, const double2* dghost, double demit, double* dlnl, double* duw,
                         cudaStream_t stream) {
  const size_t smem = G * adj_cell_bytes(P);
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(adj_step_kernel<G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               226 * 1024);
    if (e != cudaSuccess) return e;
  }
  const unsigned grid = (unsigned)((P.nx * P.ny + G - 1) / G);
  adj_step_kernel<G><<<grid, 32 * G, smem, stream>>>(P, T, fn1, qn, pn, lam_in, tilde, collide, out, dghost,
                                                     demit, dlnl, duw);
  return cudaGetLastError();
}

}  // namespace

// Cells per CTA: 4 while four cells' Gaussian factors fit in 100 KB (two
// CTAs per SM), else 2, else 1.
cudaError_t launch_adj_step(const Params& P, const Tables& T, const double2* fn1,
                            const double4_32a* qn, const double4_32a* pn, const double2* lam_in, int tilde,
                            int collide, double2* out, const double2* dghost, double demit, double* dlnl,
                            double* duw, cudaStream_t stream) {
  const size_t cb = adj_cell_bytes(P);
  if (cb > 226 * 1024) return cudaErrorInvalidValue;
  if (4 * cb <= 100 * 1024)
    return launch_adj_g<4>(P, T, fn1, qn, pn, lam_in, tilde, collide, out, dghost, demit, dlnl, duw, stream);
  if (2 * cb <= 100 * 1024)
    return launch_adj_g<2>(P, T, fn1, qn, pn, lam_in, tilde, collide, out, dghost, demit, dlnl, duw, stream);
  return launch_adj_g<1>(P, T, fn1, qn, pn, lam_in, tilde, collide, out, dghost, demit, dlnl, duw, stream);
}

}  // namespace bgk
