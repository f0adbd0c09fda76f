// bgk_step.cu - the fused FP64 BGK phase-space step.
//
// A CTA owns G spatial cells, one warp per cell; lanes stride over the
// velocity index v = jy*nvx + jx with 16-byte (g, h) pairs.  Per step:
//   phase 1 (each warp, its cell)
//     A0  diffuse-wall densities n_W of the faces the cell touches, from the
//         cell's own f^n (zero net mass flux, below Eq. bc_cavity);
//     A1  streaming: f~ = a0 f + ax f_(upwind x) + ay f_(upwind y) (2D
//         unsplit donor cell), or f~ = (1-|r|) f_(i-[C]) + |r| f_(i-[C]-sgn C)
//         (1D, Eq. upwind after the integer shift of Eq. exact); upwind
//         neighbours come from L2, boundary values from the ghost tables;
//         f~ is parked in the cell's output slots until phase 3;
//     A2  FP64 velocity sums of f~ for Eq. (macroscopic), one warp reduction;
//   phase 2 (warp 0, the G cells in lanes; in 2D warp 1 takes the y axis of
//            the Gaussian sums and factors)
//     A3  moments, nu = n theta^(1-omega), relaxation weights and the
//         effective Maxwellian parameters (one set of exponentials per cell,
//         linearised updates), separable factors written to shared memory;
//   phase 3 (each warp, its cell)
//     A4  f^{n+1} = b f~ + a Phi (Eq. relaxation: b = e^{-nu dt}, a = 1 - b;
//         Euler: a = nu dt, b = 1 - a), stored to HBM.
// The FP64 pipe of sm_103 charges every warp instruction in full whatever the
// number of active lanes, so the per-cell scalar work of phase 2 runs with
// cells in lanes (G cells per instruction) and sign tests use integer tables.
#include "bgk_device.cuh"

namespace bgk {


namespace {

__device__ __forceinline__ int vi_jx(int vi) { return vi & 0xfff; }
__device__ __forceinline__ int vi_jy(int vi) { return (vi >> 12) & 0xfff; }
__device__ __forceinline__ int vi_sx(int vi) { return ((vi >> 24) & 3) - 1; }
__device__ __forceinline__ int vi_sy(int vi) { return ((vi >> 26) & 3) - 1; }

// Boundary value at velocity j (components jx, jy) for a face of the cell
// whose state starts at fc.
__device__ __forceinline__ double2 ghost_at(const Params& P, const Tables& T, int face, int j, int jx,
                                            int jy, double nw, const double2* __restrict__ fc) {
  const int kind = P.bc_kind[face];
  if (kind == BC_SPECULAR) {
    const int jr = (face == XLO || face == XHI) ? jy * P.nvx + (P.nvx - 1 - jx)
                                                : (P.nvy - 1 - jy) * P.nvx + jx;
    return fc[jr];
  }
  const double2 gv = T.ghost[face * P.nv + j];
  if (kind == BC_DIFFUSE) return make_double2(nw * gv.x, nw * gv.y);
  return gv;
}

// ---- phase 1 ---------------------------------------------------------------
// Interior cell of a 2D grid whose velocity rows hold NM x 16 columns (NM 3
// or 4): lane
// 16 h + l takes the rows jy = h, h + 2, ... and in each row the columns
// jx = l + 16 m (m < NM).  A lane's columns never change, so sum c_x g and
// the c_x^2 part of sum |c|^2 g follow from its column sums after the loop,
// and sum c_y g and the c_y^2 part (c_y^2 from a table) from its row sum once
// per row: per point one FP64 add into the column sum, one into the row sum
// (NM - 1 per row) and one for h, plus two per row: 10/3 at NM = 3 instead
// of 5.
template <int NM>
__device__ __forceinline__ void stream_interior_rows(const Params& P, const Tables& T,
                                                     const double2* __restrict__ fc, ptrdiff_t row,
                                                     double2* __restrict__ tile, double& s0, double& sx,
                                                     double& sy, double& se) {
  const int lane = threadIdx.x & 31, l = lane & 15;
  const int nv = P.nv, nvx = P.nvx;
  int offx[NM];
  double col[NM];
#pragma unroll
  for (int m = 0; m < NM; ++m) {
    offx[m] = -vi_sx(T.vinfo[l + 16 * m]) * nv;  // upwind in x: ix - sgn c_x
    col[m] = 0.0;
  }
  double sh = 0.0, syy = 0.0;
#pragma unroll 1
  for (int jy = lane >> 4; jy < P.nvy; jy += 2) {
    const int j0 = jy * nvx + l;
    const ptrdiff_t offy = -(ptrdiff_t)vi_sy(T.vinfo[j0]) * row;
    const double cy = T.cy[jy], cy2 = T.cy2[jy];
    double rg = 0.0;
#pragma unroll
    for (int m = 0; m < NM; ++m) {
      const int j = j0 + 16 * m;
      const double2 f0 = fc[j];
      const double2 fx = fc[j + offx[m]];
      const double2 fy = fc[j + offy];
      const double4_32a co = T.coef[j];
      double2 ft;
      ft.x = fma(co.z, fy.x, fma(co.y, fx.x, co.x * f0.x));
      ft.y = fma(co.z, fy.y, fma(co.y, fx.y, co.x * f0.y));
      tile[j] = ft;
      col[m] += ft.x;
      rg = m == 0 ? ft.x : rg + ft.x;
      sh += ft.y;
    }
    sy = fma(cy, rg, sy);
    syy = fma(cy2, rg, syy);
  }
  double sxx = 0.0;
#pragma unroll
  for (int m = 0; m < NM; ++m) {
    const double cx = T.cx[l + 16 * m];
    s0 += col[m];
    sx = fma(cx, col[m], sx);
    sxx = fma(cx * cx, col[m], sxx);
  }
  se = sxx + syy + sh;
}

template <int DIM>
__device__ __forceinline__ void stream_cell(const Params& P, const Tables& T,
                                            const double2* __restrict__ fin, int cell,
                                            double2* __restrict__ tile, double* __restrict__ sums) {
  const int lane = threadIdx.x & 31;
  const int nv = P.nv, nx = P.nx;
  const int ix = cell % nx, iy = cell / nx;
  const double2* __restrict__ fc = fin + (size_t)cell * nv;
  const bool bxlo = ix == 0, bxhi = ix == nx - 1;
  const bool bylo = DIM == 2 && iy == 0, byhi = DIM == 2 && iy == P.ny - 1;

  // A0: n_W for each diffuse face this cell touches (warp-uniform branch)
  unsigned diff = 0;
  if (bxlo && P.bc_kind[XLO] == BC_DIFFUSE) diff |= 1u;
  if (bxhi && P.bc_kind[XHI] == BC_DIFFUSE) diff |= 2u;
  if (bylo && P.bc_kind[YLO] == BC_DIFFUSE) diff |= 4u;
  if (byhi && P.bc_kind[YHI] == BC_DIFFUSE) diff |= 8u;
  double nw[4] = {0.0, 0.0, 0.0, 0.0};
  if (diff) {
    double inc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int j = lane; j < nv; j += 32) {
      const int vi = T.vinfo[j];
      const double2 cxy = T.cxy[j];
      const double g = fc[j].x;
      const int sx = vi_sx(vi), sy = vi_sy(vi);
      if (sx < 0) inc[0] = fma(-cxy.x, g, inc[0]);
      if (sx > 0) inc[1] = fma(cxy.x, g, inc[1]);
      if (sy < 0) inc[2] = fma(-cxy.y, g, inc[2]);
      if (sy > 0) inc[3] = fma(cxy.y, g, inc[3]);
    }
    const double w = warp_reduce4(inc[0], inc[1], inc[2], inc[3]);
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const double tot = __shfl_sync(0xffffffffu, w, 8 * f);
      nw[f] = (diff >> f & 1u) ? tot * P.dv / T.emitted[f] : 0.0;
    }
  }

  double s0 = 0.0, sx = 0.0, sy = 0.0, se = 0.0;
  if (DIM == 2) {
    const ptrdiff_t row = (ptrdiff_t)nx * nv;
    const bool interior = !(bxlo || bxhi || bylo || byhi);
    if (interior && P.nvx == 48) {
      stream_interior_rows<3>(P, T, fc, row, tile, s0, sx, sy, se);
    } else if (interior && P.nvx == 64) {
      stream_interior_rows<4>(P, T, fc, row, tile, s0, sx, sy, se);
    } else if (interior && P.nvx == 32) {
      // 32 columns: lane = jx for every j = lane + 32 k, so sum c_x g =
      // c_x[lane] sum g is taken once after the loop (4 operations per point,
      // as many as the row mapping needs with two columns per lane)
#pragma unroll 4
      for (int j = lane; j < nv; j += 32) {
        const int vi = T.vinfo[j];
        const double2 f0 = fc[j];
        const double2 fx = fc[j - vi_sx(vi) * nv];
        const double2 fy = fc[j - vi_sy(vi) * row];
        const double4_32a co = T.coef[j];
        const double cyj = T.cxy[j].y;
        double2 ft;
        ft.x = fma(co.z, fy.x, fma(co.y, fx.x, co.x * f0.x));
        ft.y = fma(co.z, fy.y, fma(co.y, fx.y, co.x * f0.y));
        tile[j] = ft;
        s0 += ft.x;
        sy = fma(cyj, ft.x, sy);
        se = fma(co.w, ft.x, se) + ft.y;
      }
      sx = T.cx[lane] * s0;
    } else if (interior) {
      // interior cell: every upwind neighbour is a cell of the grid
#pragma unroll 4
      for (int j = lane; j < nv; j += 32) {
        const int vi = T.vinfo[j];
        const double2 f0 = fc[j];
        const double2 fx = fc[j - vi_sx(vi) * nv];
        const double2 fy = fc[j - vi_sy(vi) * row];
        const double4_32a co = T.coef[j];
        const double2 cxy = T.cxy[j];
        double2 ft;
        ft.x = fma(co.z, fy.x, fma(co.y, fx.x, co.x * f0.x));
        ft.y = fma(co.z, fy.y, fma(co.y, fx.y, co.x * f0.y));
        tile[j] = ft;
        s0 += ft.x;
        sx = fma(cxy.x, ft.x, sx);
        sy = fma(cxy.y, ft.x, sy);
        se = fma(co.w, ft.x, se) + ft.y;
      }
    } else {
      for (int j = lane; j < nv; j += 32) {
        const int vi = T.vinfo[j];
        const int jx = vi_jx(vi), jy = vi_jy(vi), sgx = vi_sx(vi), sgy = vi_sy(vi);
        const double2 f0 = fc[j];
        double2 fx = f0, fy = f0;
        if (sgx > 0) fx = bxlo ? ghost_at(P, T, XLO, j, jx, jy, nw[XLO], fc) : fc[j - nv];
        else if (sgx < 0) fx = bxhi ? ghost_at(P, T, XHI, j, jx, jy, nw[XHI], fc) : fc[j + nv];
        if (sgy > 0) fy = bylo ? ghost_at(P, T, YLO, j, jx, jy, nw[YLO], fc) : fc[j - row];
        else if (sgy < 0) fy = byhi ? ghost_at(P, T, YHI, j, jx, jy, nw[YHI], fc) : fc[j + row];
        const double4_32a co = T.coef[j];
        const double2 cxy = T.cxy[j];
        double2 ft;
        ft.x = fma(co.z, fy.x, fma(co.y, fx.x, co.x * f0.x));
        ft.y = fma(co.z, fy.y, fma(co.y, fx.y, co.x * f0.y));
        tile[j] = ft;
        s0 += ft.x;
        sx = fma(cxy.x, ft.x, sx);
        sy = fma(cxy.y, ft.x, sy);
        se = fma(co.w, ft.x, se) + ft.y;
      }
    }
  } else {
    for (int j = lane; j < nv; j += 32) {
      const int vi = T.vinfo[j];
      const int sgx = vi_sx(vi);
      const int s = T.shift[j];
      const int i1 = ix - s, i2 = ix - s - sgx;
      double2 f1, f2;
      if (i1 < 0) f1 = ghost_at(P, T, XLO, j, j, 0, nw[XLO], fc);
      else if (i1 >= nx) f1 = ghost_at(P, T, XHI, j, j, 0, nw[XHI], fc);
      else f1 = fin[(size_t)i1 * nv + j];
      if (i2 < 0) f2 = ghost_at(P, T, XLO, j, j, 0, nw[XLO], fc);
      else if (i2 >= nx) f2 = ghost_at(P, T, XHI, j, j, 0, nw[XHI], fc);
      else f2 = fin[(size_t)i2 * nv + j];
      const double4_32a co = T.coef[j];
      const double cx = T.cxy[j].x;
      double2 ft;
      ft.x = fma(co.y, f2.x, co.x * f1.x);
      ft.y = fma(co.y, f2.y, co.x * f1.y);
      tile[j] = ft;
      s0 += ft.x;
      sx = fma(cx, ft.x, sx);
      se = fma(co.w, ft.x, se) + ft.y;
    }
  }
  const double w = warp_reduce4(s0, sx, sy, se);
  if ((lane & 7) == 0) sums[lane >> 3] = w;
}

// ---- phase 2 ---------------------------------------------------------------
// Sums of five values over the L lanes of a group (sub = 0 .. L-1, L a power
// of two >= 4), returned to every lane of the group.  Recursive halving: the
// first exchange splits the values 3 + 2 between the two halves of the
// group, the second 2 + 1 within each half, the third leaves one value per
// lane, then plain butterflies; 8 FP64 additions at L = 32 (5 at L = 4)
// instead of 5 log2 L.  The lane pattern of each value is fixed, so the
// result does not depend on the data.
template <int L>
__device__ __forceinline__ void group_sum5(double& m0, double& m1, double& m2, double& m3, double& m4,
                                           int sub) {
  static_assert(L >= 4 && (L & (L - 1)) == 0, "group of 4, 8, 16 or 32 lanes");
  constexpr unsigned kAll = 0xffffffffu;
  const int base = (threadIdx.x & 31) - sub;
  // 1: the low half keeps (m0, m1, m2), the high half (m3, m4, 0)
  const bool h1 = sub & (L / 2);
  double a0 = h1 ? m3 : m0, a1 = h1 ? m4 : m1, a2 = h1 ? 0.0 : m2;
  const double t0 = h1 ? m0 : m3, t1 = h1 ? m1 : m4, t2 = h1 ? m2 : 0.0;
  a0 += __shfl_xor_sync(kAll, t0, L / 2);
  a1 += __shfl_xor_sync(kAll, t1, L / 2);
  a2 += __shfl_xor_sync(kAll, t2, L / 2);
  // 2: of (a0, a1, a2) the low quarter keeps (a0, a1), the high one (a2, 0)
  const bool h2 = sub & (L / 4);
  double k0 = h2 ? a2 : a0, k1 = h2 ? 0.0 : a1;
  const double u0 = h2 ? a0 : a2, u1 = h2 ? a1 : 0.0;
  k0 += __shfl_xor_sync(kAll, u0, L / 4);
  k1 += __shfl_xor_sync(kAll, u1, L / 4);
  if (L == 4) {
    // lane 0: (m0, m1), lane 1: (m2, 0), lane 2: (m3, m4), lane 3: (0, 0)
    m0 = __shfl_sync(kAll, k0, base);
    m1 = __shfl_sync(kAll, k1, base);
    m2 = __shfl_sync(kAll, k0, base + 1);
    m3 = __shfl_sync(kAll, k0, base + 2);
    m4 = __shfl_sync(kAll, k1, base + 2);
    return;
  }
  // 3: one value per lane, then the remaining lane bits summed out
  const bool h3 = sub & (L / 8);
  double v = h3 ? k1 : k0;
  v += __shfl_xor_sync(kAll, h3 ? k0 : k1, L / 8);
#pragma unroll
  for (int s = L / 16; s > 0; s >>= 1) v += __shfl_xor_sync(kAll, v, s);
  // m0 at sub 0, m1 at L/8, m2 at L/4, m3 at L/2, m4 at L/2 + L/8
  m0 = __shfl_sync(kAll, v, base);
  m1 = __shfl_sync(kAll, v, base + L / 8);
  m2 = __shfl_sync(kAll, v, base + L / 4);
  m3 = __shfl_sync(kAll, v, base + L / 2);
  m4 = __shfl_sync(kAll, v, base + L / 2 + L / 8);
}

// Exponentials e_j = exp(-(c_j - u)^2 / theta) of one axis for one cell,
// lanes sub, sub + L, ... of the cell's group; stores them when `store`;
// returns the group's central sums M_m = sum d^m e, d = c_j - u, m = 0..4.
// On the uniform grid a lane's points are d_i = d_0 + i D (D = L dc), and a
// Gaussian obeys e_{i+1} = e_i r_i, r_i = exp(-(2 d_i D + D^2) / theta),
// r_{i+1} = r_i exp(-2 D^2 / theta): three exponentials per lane and two
// products per further point instead of one exponential per point (each
// product adds a rounding: after k points the relative error is about k^2
// ulp, 1e-14 at k = 8).  Lanes with fewer than four points, and where e_0
// could underflow or r_0 overflow (theta far below the grid's scale), take
// one exponential per point.
template <int L>
__device__ __forceinline__ void axis_sums(const double* __restrict__ c, int n, double dc, double u,
                                          double inv_th, int sub, bool store, double* __restrict__ out, bool want,
                                          double M[5]) {
  double m0 = 0.0, m1 = 0.0, m2 = 0.0, m3 = 0.0, m4 = 0.0;
  if (sub < n) {
    const double D = L * dc;
    const double d0 = c[sub] - u;
    const double x0 = (d0 * d0) * inv_th, y0 = (2.0 * d0 * D + D * D) * inv_th;
    const bool rec = n >= 4 * L && x0 < 600.0 && -y0 < 600.0;
    double e = exp(-x0);
    double r = rec ? exp(-y0) : 0.0;
    const double q = rec ? exp(-2.0 * D * D * inv_th) : 0.0;
    for (int j = sub;;) {
      const double d = c[j] - u;
      if (store) out[j] = e;
      if (want) {
        double t = e;
        m0 += t;
        t *= d;
        m1 += t;
        t *= d;
        m2 += t;
        t *= d;
        m3 += t;
        t *= d;
        m4 += t;
      }
      j += L;
      if (j >= n) break;
      if (rec) {
        e *= r;
        r *= q;
      } else {
        const double dn = c[j] - u;
        e = exp(-(dn * dn) * inv_th);
      }
    }
  }
  if (want) group_sum5<L>(m0, m1, m2, m3, m4, sub);
  M[0] = m0;
  M[1] = m1;
  M[2] = m2;
  M[3] = m3;
  M[4] = m4;
}

template <int DIM, int G>
__device__ void maxwellian_cells(const Params& P, const Tables& T, int cell0, const double (*sums)[4],
                                 double* __restrict__ phx, double* __restrict__ phy, double* sb,
                                 double* sk, int* sok, double4_32a* __restrict__ mom,
                                 double4_32a* __restrict__ par, int* __restrict__ err) {
  constexpr int L = 32 / G;
  const int lane = threadIdx.x & 31, c = lane / L, sub = lane % L;
  const int cell = cell0 + c;
  const bool live = cell < P.nx * P.ny;
  double qm[4] = {1.0, 0.0, 0.0, 1.0};  // moments of f~ (Eq. macroscopic)
  if (live) moments_from_sums(sums[c][0], sums[c][1], sums[c][2], sums[c][3], P.dv, qm);
  bool ok = live && moments_ok(qm);
  // a failed cell keeps its lanes busy on a harmless stand-in state
  const double q[4] = {ok ? qm[0] : 1.0, ok ? qm[1] : 0.0, ok ? qm[2] : 0.0, ok ? qm[3] : 1.0};
  double a, b;
  relax_weights(P, q, a, b);
  double* px = phx + c * P.nvx;
  double* py = phy + c * P.nvy;
  const bool cons = P.conservative != 0;
  EffState E;
  eff_init(E, q, !(cons && ok));
  double Mx[5], My[5] = {1.0, 0.0, 0.0, 0.0, 0.0};
  for (int round = 0; round <= kEffMaxIt; ++round) {
    const bool need = round == 0 || E.reeval;
    if (!__any_sync(0xffffffffu, need)) break;
    const double inv_th = E.ith;
    double Mt[5];
    axis_sums<L>(T.cx, P.nvx, P.dcx, E.base[1], inv_th, sub, need, px, cons, Mt);
    if (need)
      for (int m = 0; m < 5; ++m) Mx[m] = Mt[m];
    if (DIM == 2) {
      axis_sums<L>(T.cy, P.nvy, P.dcy, E.base[2], inv_th, sub, need, py, cons, Mt);
      if (need)
        for (int m = 0; m < 5; ++m) My[m] = Mt[m];
    }
    E.reeval = false;
    eff_iterate<DIM>(P, q, Mx, My, E);  // A3, linearised about E.base
  }
  if (E.fail) ok = false;
  const double* p = E.p;
  if (ok) {
    // A4 factors: a Phi_g = px[jx] py[jy], moved from E.base to p
    double w1x, w1y, w2;
    eff_lin(E, w1x, w1y, w2);
    const double pref = (DIM == 1) ? p[0] * rsqrt(kPi() * p[3]) : p[0] / (kPi() * p[3]);
    const double ap = a * pref;
    for (int j = sub; j < P.nvx; j += L) {
      const double d = T.cx[j] - E.base[1];
      px[j] = ap * (px[j] * fma(d, fma(d, w2, w1x), 1.0));
    }
    if (DIM == 2) {
      for (int j = sub; j < P.nvy; j += L) {
        const double d = T.cy[j] - E.base[2];
        py[j] = py[j] * fma(d, fma(d, w2, w1y), 1.0);
      }
    }
  }
  if (sub == 0) {
    sb[c] = b;
    sk[c] = (DIM == 1) ? p[3] : 0.5 * p[3];
    sok[c] = ok ? 1 : 0;
    if (live) {
      mom[cell] = make_double4_32a(qm[0], qm[1], qm[2], qm[3]);
      if (par) par[cell] = make_double4_32a(p[0], p[1], p[2], p[3]);
      if (!ok) atomicOr(err, E.fail ? ERR_EFFECTIVE : ERR_MOMENT);
    }
  }
}

// Phase 2 of a 2D CTA on two warps: the y-axis Gaussian sums and factors of
// the G cells run on warp 1 (another SM sub-partition) while warp 0 does the
// x axis and the scalar solve, so the CTA's other warps wait at the barrier
// for about one axis less.  Every value is computed by the same functions in
// the same order as in maxwellian_cells, so the results are the same bit
// for bit.  Warp 0 hands warp 1 the base point of each round and the factor
// update; warp 1 hands back the y central sums (named barrier 1, 64 threads).
template <int G>
struct SolveXchg {
  double ub[G], ith[G];  // y base velocity and 1 / theta_b of the round
  double my[G][5];       // y central sums of the round
  double w1y[G], w2[G];  // factor update (after the last round)
  int need[G], ok[G];
  int go;
};

__device__ __forceinline__ void pair_barrier() { asm volatile("bar.sync 1, 64;" ::: "memory"); }

template <int G>
__device__ void maxwellian_cells_2w(const Params& P, const Tables& T, int cell0, const double (*sums)[4],
                                    double* __restrict__ phx, double* __restrict__ phy, double* sb, double* sk,
                                    int* sok, double4_32a* __restrict__ mom, double4_32a* __restrict__ par,
                                    int* __restrict__ err, SolveXchg<G>& X) {
  constexpr int L = 32 / G;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, c = lane / L, sub = lane % L;
  const bool cons = P.conservative != 0;
  if (warp == 1) {
    double* py = phy + c * P.nvy;
    for (;;) {
      pair_barrier();  // base point of the round published
      if (!X.go) break;
      const bool need = X.need[c] != 0;
      double Mt[5];
      axis_sums<L>(T.cy, P.nvy, P.dcy, X.ub[c], X.ith[c], sub, need, py, cons, Mt);
      if (sub == 0)
        for (int m = 0; m < 5; ++m) X.my[c][m] = Mt[m];
      pair_barrier();  // sums handed over
    }
    pair_barrier();  // factor update published
    if (X.ok[c]) {
      const double ub = X.ub[c], w1y = X.w1y[c], w2 = X.w2[c];
      for (int j = sub; j < P.nvy; j += L) {
        const double d = T.cy[j] - ub;
        py[j] = py[j] * fma(d, fma(d, w2, w1y), 1.0);
      }
    }
    return;
  }
  const int cell = cell0 + c;
  const bool live = cell < P.nx * P.ny;
  double qm[4] = {1.0, 0.0, 0.0, 1.0};  // moments of f~ (Eq. macroscopic)
  if (live) moments_from_sums(sums[c][0], sums[c][1], sums[c][2], sums[c][3], P.dv, qm);
  bool ok = live && moments_ok(qm);
  const double q[4] = {ok ? qm[0] : 1.0, ok ? qm[1] : 0.0, ok ? qm[2] : 0.0, ok ? qm[3] : 1.0};
  double* px = phx + c * P.nvx;
  EffState E;
  eff_init(E, q, !(cons && ok));
  double a = 0.0, b = 0.0;
  double Mx[5], My[5];
  // every exit from this loop goes through a published go = 0 (warp 1
  // leaves its loop on it), so the two warps pass the same barriers
  for (int round = 0;; ++round) {
    const bool need = round <= kEffMaxIt && (round == 0 || E.reeval);
    const bool go = __any_sync(0xffffffffu, need);
    if (sub == 0) {
      X.need[c] = need ? 1 : 0;
      X.ub[c] = E.base[2];
      X.ith[c] = E.ith;
    }
    if (lane == 0) X.go = go ? 1 : 0;
    pair_barrier();
    if (!go) break;
    double Mt[5];
    axis_sums<L>(T.cx, P.nvx, P.dcx, E.base[1], E.ith, sub, need, px, cons, Mt);
    if (need)
      for (int m = 0; m < 5; ++m) Mx[m] = Mt[m];
    if (round == 0) relax_weights(P, q, a, b);
    pair_barrier();
    if (need)
      for (int m = 0; m < 5; ++m) My[m] = X.my[c][m];
    E.reeval = false;
    eff_iterate<2>(P, q, Mx, My, E);  // A3, linearised about E.base
  }
  if (E.fail) ok = false;
  const double* p = E.p;
  double w1x = 0.0, w1y = 0.0, w2 = 0.0;
  if (ok) eff_lin(E, w1x, w1y, w2);
  if (sub == 0) {
    X.ok[c] = ok ? 1 : 0;
    X.ub[c] = E.base[2];
    X.w1y[c] = w1y;
    X.w2[c] = w2;
  }
  pair_barrier();
  if (ok) {
    // A4 factors: a Phi_g = px[jx] py[jy], moved from E.base to p
    const double ap = a * (p[0] / (kPi() * p[3]));
    for (int j = sub; j < P.nvx; j += L) {
      const double d = T.cx[j] - E.base[1];
      px[j] = ap * (px[j] * fma(d, fma(d, w2, w1x), 1.0));
    }
  }
  if (sub == 0) {
    sb[c] = b;
    sk[c] = 0.5 * p[3];
    sok[c] = ok ? 1 : 0;
    if (live) {
      mom[cell] = make_double4_32a(qm[0], qm[1], qm[2], qm[3]);
      if (par) par[cell] = make_double4_32a(p[0], p[1], p[2], p[3]);
      if (!ok) atomicOr(err, E.fail ? ERR_EFFECTIVE : ERR_MOMENT);
    }
  }
}

// ---- phase 3 ---------------------------------------------------------------
// A4 for the warp's cell: f^{n+1} = b f~ + a Phi from the f~ parked in the
// cell's output slots, a Phi_g = px[jx] py[jy], a Phi_h = kappa a Phi_g.
template <int DIM>
__device__ __forceinline__ void relax_cell(const Params& P, const Tables& T, double2* __restrict__ fout, int cell,
                                           const double* __restrict__ px, const double* __restrict__ py, double b,
                                           double kappa, bool ok) {
  const int lane = threadIdx.x & 31;
  const int nv = P.nv;
  double2* __restrict__ fo = fout + (size_t)cell * nv;
  const double2* tile = fo;
  if (DIM == 2 && ok && (P.nvx == 48 || P.nvx == 64)) {
    // rows jy = h, h + 2, ..., columns jx = l + 16 m of lane 16 h + l, as
    // in stream_interior_rows: a Phi = px[jx] py[jy] from shared memory
    const int l = lane & 15;
    for (int jy = lane >> 4; jy < P.nvy; jy += 2) {
      const double pyv = py[jy];
#pragma unroll 4
      for (int jx = l; jx < P.nvx; jx += 16) {
        const int j = jy * P.nvx + jx;
        const double2 ft = tile[j];
        const double aphi = px[jx] * pyv;
        fo[j] = make_double2(fma(b, ft.x, aphi), fma(b, ft.y, kappa * aphi));
      }
    }
    return;
  }
#pragma unroll 4
  for (int j = lane; j < nv; j += 32) {
    const double2 ft = tile[j];
    double2 r = ft;
    if (ok) {
      double aphi;
      if (DIM == 2) {
        const int vi = T.vinfo[j];
        aphi = px[vi_jx(vi)] * py[vi_jy(vi)];
      } else {
        aphi = px[j];
      }
      r.x = fma(b, ft.x, aphi);
      r.y = fma(b, ft.y, kappa * aphi);
    }
    fo[j] = r;
  }
}

}  // namespace

// 4 cells per CTA runs 8 CTAs per SM at 64 registers: spilling a little
// beats 4 CTAs at 124 registers (measured: 204 -> 191 us on 64^2 x 32^2,
// 5.14 -> 4.84 ms on 256^2 x 48^2; 5 and 6 CTAs were slower); 8 cells per
// CTA run 4 CTAs per SM at 64 registers (the choice for large 2D grids).
template <int DIM, int G>
__global__ void __launch_bounds__(32 * G, G == 4 ? 8 : (G == 8 ? 4 : 1))
    step_f64_kernel(const double2* __restrict__ fin, double2* __restrict__ fout,
                    double4_32a* __restrict__ mom, double4_32a* __restrict__ par, const Params P,
                    const Tables T, int* __restrict__ err) {
  extern __shared__ double4_32a smem4[];
  double* phx = reinterpret_cast<double*>(smem4);
  double* phy = phx + G * P.nvx;
  __shared__ double s_sum[G][4];
  __shared__ double s_b[G], s_k[G];
  __shared__ int s_ok[G];

  const int warp = threadIdx.x >> 5;
  const int nv = P.nv;
  const int cell = blockIdx.x * G + warp;
  const bool live = cell < P.nx * P.ny;
  // f~ of the warp's cell is parked in the cell's own output slots between
  // the passes (each lane rereads only what it wrote; the values come back
  // from L2): staging it in shared memory (16 B per velocity) held an SM to
  // 3 CTAs, measured 21 % (64^2 x 32^2) and 40 % (256^2 x 48^2) slower
  double2* tile = fout + (size_t)cell * nv;

  if (live) stream_cell<DIM>(P, T, fin, cell, tile, s_sum[warp]);
  __syncthreads();
  if (DIM == 2 && G >= 2) {
    __shared__ SolveXchg<G> s_x;
    if (warp < 2) maxwellian_cells_2w<G>(P, T, blockIdx.x * G, s_sum, phx, phy, s_b, s_k, s_ok, mom, par, err, s_x);
  } else if (warp == 0) {
    maxwellian_cells<DIM, G>(P, T, blockIdx.x * G, s_sum, phx, phy, s_b, s_k, s_ok, mom, par, err);
  }
  __syncthreads();
  if (!live) return;

  relax_cell<DIM>(P, T, fout, cell, phx + warp * P.nvx, phy + warp * P.nvy, s_b[warp], s_k[warp],
                  s_ok[warp] != 0);
}

namespace {

size_t step_smem(const Params& P, int G) {
  return sizeof(double) * (size_t)G * (P.nvx + P.nvy);
}

template <int DIM, int G>
cudaError_t launch_g(const Params& P, const Tables& T, const double2* fin, double2* fout,
                     double4_32a* mom, double4_32a* par, int* err, cudaStream_t stream) {
  const int ncell = P.nx * P.ny;
  const unsigned grid = (unsigned)((ncell + G - 1) / G);
  step_f64_kernel<DIM, G><<<grid, 32 * G, step_smem(P, G), stream>>>(fin, fout, mom, par, P, T, err);
  return cudaGetLastError();
}

// The attribute belongs to the kernel, not to a solver: set it to the
// largest dynamic shared memory any solver may request (what the device
// allows a CTA beside the kernel's static shared memory) so that solvers
// with different grids sharing an instantiation never shrink it.
template <int DIM, int G>
cudaError_t prepare_g(const Params&) {
  int dev = 0, optin = 0;
  cudaFuncAttributes fa;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, step_f64_kernel<DIM, G>);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(step_f64_kernel<DIM, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              optin - (int)fa.sharedSizeBytes);
}

template <int DIM>
cudaError_t dispatch(const Params& P, const Tables& T, const double2* fin, double2* fout,
                     double4_32a* mom, double4_32a* par, int* err, cudaStream_t stream) {
  switch (P.tile) {
    case 1: return launch_g<DIM, 1>(P, T, fin, fout, mom, par, err, stream);
    case 2: return launch_g<DIM, 2>(P, T, fin, fout, mom, par, err, stream);
    case 4: return launch_g<DIM, 4>(P, T, fin, fout, mom, par, err, stream);
    case 8: return launch_g<DIM, 8>(P, T, fin, fout, mom, par, err, stream);
  }
  return cudaErrorInvalidValue;
}

template <int DIM>
cudaError_t prepare_dim(const Params& P) {
  switch (P.tile) {
    case 1: return prepare_g<DIM, 1>(P);
    case 2: return prepare_g<DIM, 2>(P);
    case 4: return prepare_g<DIM, 4>(P);
    case 8: return prepare_g<DIM, 8>(P);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

size_t step_f64_smem_bytes(const Params& P, int tile) { return step_smem(P, tile); }

cudaError_t prepare_step_f64(const Params& P) {
  return P.dim == 1 ? prepare_dim<1>(P) : prepare_dim<2>(P);
}

cudaError_t launch_step_f64(const Params& P, const Tables& T, const double2* fin, double2* fout,
                            double4_32a* mom, int* err, cudaStream_t stream, double4_32a* par) {
  return P.dim == 1 ? dispatch<1>(P, T, fin, fout, mom, par, err, stream)
                    : dispatch<2>(P, T, fin, fout, mom, par, err, stream);
}

}  // namespace bgk
