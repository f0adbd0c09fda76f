// bgk_step.cu - the fused FP64 BGK phase-space step.
//
// One CTA owns one spatial cell and all of its velocities (threads stride
// over the velocity index v = jy*nvx + jx, 16-byte (g, h) pairs).  Per step
// and cell the CTA
//   A0  computes the diffuse-wall densities n_W of the faces the cell
//       touches from its own f^n (zero net mass flux, below Eq. bc_cavity);
//   A1  streams: f~ = a0 f + ax f_(upwind x) + ay f_(upwind y) (2D unsplit
//       donor cell), or f~ = (1-|r|) f_(i-[C]) + |r| f_(i-[C]-sgn C) (1D,
//       Eq. upwind after the integer shift of Eq. exact), neighbours read
//       from L2 and boundary values from the ghost tables;
//   A2  reduces the moments of f~ (Eq. macroscopic) in FP64;
//   A3  forms nu = n theta^(1-omega) and the (effective) Maxwellian
//       parameters in one warp, writing separable factors to shared memory;
//   A4  relaxes in registers, f^{n+1} = b f~ + a Phi (Eq. relaxation:
//       b = e^{-nu dt}, a = 1 - b; Euler: a = nu dt, b = 1 - a), and stores.
// f^n is read once from HBM and f^{n+1} written once; neighbour re-reads of
// the same f^n hit L2 because CTAs run in raster order.
#include <cstdio>

#include "bgk_device.cuh"

namespace bgk {

template <int DIM, int BLOCK, int NPT>
__global__ void __launch_bounds__(BLOCK)
    step_f64_kernel(const double2* __restrict__ fin, double2* __restrict__ fout,
                    double4_32a* __restrict__ mom, const Params P, const Tables T, int* __restrict__ err) {
  extern __shared__ double sh_dyn[];  // phx[nvx], phy[nvy]
  __shared__ double red[4 * (BLOCK / 32)];
  __shared__ double tot[4];
  __shared__ double sc[8];  // 0..3: n_W per face; 4: b; 5: kappa; 6: ok
  double* phx = sh_dyn;
  double* phy = sh_dyn + P.nvx;

  const int cell = blockIdx.x;
  const int tid = threadIdx.x;
  const int nx = P.nx, nv = P.nv;
  const int ix = cell % nx, iy = cell / nx;
  const double2* __restrict__ fc = fin + (size_t)cell * nv;

  double2 own[NPT];
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    const int j = tid + k * BLOCK;
    own[k] = (j < nv) ? __ldg(fc + j) : make_double2(0.0, 0.0);
  }

  // ---- A0: diffuse-wall densities for the faces this cell touches ---------
  unsigned diff = 0;
  if (ix == 0 && P.bc_kind[XLO] == BC_DIFFUSE) diff |= 1u;
  if (ix == nx - 1 && P.bc_kind[XHI] == BC_DIFFUSE) diff |= 2u;
  if (DIM == 2) {
    if (iy == 0 && P.bc_kind[YLO] == BC_DIFFUSE) diff |= 4u;
    if (iy == P.ny - 1 && P.bc_kind[YHI] == BC_DIFFUSE) diff |= 8u;
  }
  if (diff) {  // uniform over the CTA
    double inc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
      const int j = tid + k * BLOCK;
      if (j < nv) {
        const double cx = T.cx[DIM == 2 ? j % P.nvx : j];
        const double g = own[k].x;
        if (cx < 0.0) inc[0] = fma(-cx, g, inc[0]);
        if (cx > 0.0) inc[1] = fma(cx, g, inc[1]);
        if (DIM == 2) {
          const double cy = T.cy[j / P.nvx];
          if (cy < 0.0) inc[2] = fma(-cy, g, inc[2]);
          if (cy > 0.0) inc[3] = fma(cy, g, inc[3]);
        }
      }
    }
    block_reduce4<BLOCK>(inc[0], inc[1], inc[2], inc[3], red, tot);
    if (tid < 4) sc[tid] = (diff >> tid & 1u) ? tot[tid] * P.dv / T.emitted[tid] : 0.0;
    __syncthreads();
  }

  // ---- A1: free streaming ----------------------------------------------
  double2 ft[NPT];
  double s0 = 0.0, sx = 0.0, sy = 0.0, se = 0.0;
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    const int j = tid + k * BLOCK;
    ft[k] = make_double2(0.0, 0.0);
    if (j < nv) {
      const double4_32a co = T.coef[j];
      if (DIM == 2) {
        const int jx = j % P.nvx, jy = j / P.nvx;
        const double cx = T.cx[jx], cy = T.cy[jy];
        double2 fx = own[k], fy = own[k];
        if (cx > 0.0) {
          fx = (ix > 0) ? fin[(size_t)(cell - 1) * nv + j] : ghost_value(P, T, XLO, j, sc[XLO], fc);
        } else if (cx < 0.0) {
          fx = (ix < nx - 1) ? fin[(size_t)(cell + 1) * nv + j] : ghost_value(P, T, XHI, j, sc[XHI], fc);
        }
        if (cy > 0.0) {
          fy = (iy > 0) ? fin[(size_t)(cell - nx) * nv + j] : ghost_value(P, T, YLO, j, sc[YLO], fc);
        } else if (cy < 0.0) {
          fy = (iy < P.ny - 1) ? fin[(size_t)(cell + nx) * nv + j] : ghost_value(P, T, YHI, j, sc[YHI], fc);
        }
        ft[k].x = fma(co.z, fy.x, fma(co.y, fx.x, co.x * own[k].x));
        ft[k].y = fma(co.z, fy.y, fma(co.y, fx.y, co.x * own[k].y));
        // ---- A2 (partial): velocity sums of f~ -----------------------------
        s0 += ft[k].x;
        sx = fma(cx, ft[k].x, sx);
        sy = fma(cy, ft[k].x, sy);
        se = fma(co.w, ft[k].x, se) + ft[k].y;
      } else {
        const double cx = T.cx[j];
        const int s = T.shift[j];
        const int up = cx > 0.0 ? 1 : -1;
        const int i1 = ix - s, i2 = ix - s - up;
        double2 f1, f2;
        if (s == 0) f1 = own[k];
        else if (i1 < 0) f1 = ghost_value(P, T, XLO, j, sc[XLO], fc);
        else if (i1 >= nx) f1 = ghost_value(P, T, XHI, j, sc[XHI], fc);
        else f1 = fin[(size_t)i1 * nv + j];
        if (i2 < 0) f2 = ghost_value(P, T, XLO, j, sc[XLO], fc);
        else if (i2 >= nx) f2 = ghost_value(P, T, XHI, j, sc[XHI], fc);
        else f2 = fin[(size_t)i2 * nv + j];
        ft[k].x = fma(co.y, f2.x, co.x * f1.x);
        ft[k].y = fma(co.y, f2.y, co.x * f1.y);
        s0 += ft[k].x;
        sx = fma(cx, ft[k].x, sx);
        se = fma(co.w, ft[k].x, se) + ft[k].y;
      }
    }
  }

  // ---- A2: block reduction of the moments --------------------------------
  block_reduce4<BLOCK>(s0, sx, sy, se, red, tot);

  // ---- A3: nu and the Maxwellian, one warp --------------------------------
  if (tid < 32) {
    double q[4];
    moments_from_sums(tot[0], tot[1], tot[2], tot[3], P.dv, q);
    bool ok = moments_ok(q);
    double p[4] = {q[0], q[1], q[2], q[3]};
    double a = 0.0, b = 1.0;
    if (ok) {
      const double nu = q[0] * pow(q[3], 1.0 - P.omega);
      if (P.relax_exact) {
        b = exp(-nu * P.dt);
        a = 1.0 - b;
      } else {
        a = P.dt * nu;
        b = 1.0 - a;
      }
      if (P.conservative && effective_params_warp(P, T.cx, T.cy, q, p) < 0) {
        ok = false;
        if (tid == 0) atomicOr(err, ERR_EFFECTIVE);
      }
    } else if (tid == 0) {
      atomicOr(err, ERR_MOMENT);
    }
    if (ok) maxwell_factors_warp(P, T.cx, T.cy, p, a, phx, phy);
    if (tid == 0) {
      mom[cell] = make_double4_32a(q[0], q[1], q[2], q[3]);
      sc[4] = b;
      sc[5] = (DIM == 1) ? p[3] : 0.5 * p[3];
      sc[6] = ok ? 1.0 : 0.0;
    }
  }
  __syncthreads();

  // ---- A4: relaxation and store --------------------------------------------
  const double b = sc[4], kappa = sc[5];
  const bool ok = sc[6] != 0.0;
  double2* __restrict__ fo = fout + (size_t)cell * nv;
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    const int j = tid + k * BLOCK;
    if (j < nv) {
      double2 r = ft[k];
      if (ok) {
        const double aphi = (DIM == 2) ? phx[j % P.nvx] * phy[j / P.nvx] : phx[j];
        r.x = fma(b, ft[k].x, aphi);
        r.y = fma(b, ft[k].y, kappa * aphi);
      }
      fo[j] = r;
    }
  }
}

namespace {

template <int DIM, int BLOCK, int NPT>
cudaError_t launch_t(const Params& P, const Tables& T, const double2* fin, double2* fout,
                     double4_32a* mom, int* err, cudaStream_t stream) {
  const size_t shmem = sizeof(double) * (P.nvx + (DIM == 2 ? P.nvy : 0));
  step_f64_kernel<DIM, BLOCK, NPT><<<P.nx * P.ny, BLOCK, shmem, stream>>>(fin, fout, mom, P, T, err);
  return cudaGetLastError();
}

template <int DIM, int BLOCK>
cudaError_t dispatch_npt(const Params& P, const Tables& T, const double2* fin, double2* fout,
                         double4_32a* mom, int* err, cudaStream_t stream) {
  const int need = (P.nv + BLOCK - 1) / BLOCK;
  if (need <= 1) return launch_t<DIM, BLOCK, 1>(P, T, fin, fout, mom, err, stream);
  if (need <= 2) return launch_t<DIM, BLOCK, 2>(P, T, fin, fout, mom, err, stream);
  if (need <= 3) return launch_t<DIM, BLOCK, 3>(P, T, fin, fout, mom, err, stream);
  if (need <= 4) return launch_t<DIM, BLOCK, 4>(P, T, fin, fout, mom, err, stream);
  if (need <= 6) return launch_t<DIM, BLOCK, 6>(P, T, fin, fout, mom, err, stream);
  if (need <= 8) return launch_t<DIM, BLOCK, 8>(P, T, fin, fout, mom, err, stream);
  if (need <= 9) return launch_t<DIM, BLOCK, 9>(P, T, fin, fout, mom, err, stream);
  if (need <= 12) return launch_t<DIM, BLOCK, 12>(P, T, fin, fout, mom, err, stream);
  if (need <= 16) return launch_t<DIM, BLOCK, 16>(P, T, fin, fout, mom, err, stream);
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_step_f64(const Params& P, const Tables& T, const double2* fin, double2* fout,
                            double4_32a* mom, int* err, cudaStream_t stream) {
  if (P.dim == 1) {
    if (P.nv <= 64 * 16) return dispatch_npt<1, 64>(P, T, fin, fout, mom, err, stream);
    return dispatch_npt<1, 256>(P, T, fin, fout, mom, err, stream);
  }
  return dispatch_npt<2, 256>(P, T, fin, fout, mom, err, stream);
}

}  // namespace bgk
