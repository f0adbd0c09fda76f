// bgk_step3v.cu - the FP64 BGK step on a full three-dimensional velocity
// grid with one spatial dimension: the normal shock of Sec. 4.1 as the paper
// computed it (the Chu reduction is not made; f lives on N_vx x N_vy x N_vz
// velocity cells per spatial cell; Delta t = 0.05 puts the fast velocities
// several cells per step, so streaming is the integer shift of Eq. (exact)
// followed by the upwind remainder of Eq. (upwind)).
//
// One CTA of 256 threads per spatial cell (4 096 to 27 000 velocities):
//   pass 1  f~ = (1 - r) f_{i-[C]} + r f_{i-[C]-sgn C} per velocity (inflow
//           Maxwellians beyond the ends) and the five sums of Eq.
//           (macroscopic) (n, n U, E), reduced over the CTA;
//   cell    nu = n theta^(1-omega), the relaxation weights, and the
//           effective parameters p (Sec. 2.1 remark) by p <- p + (q - D(p))
//           with the Gaussian factored per axis: warp a of the first three
//           evaluates axis a's 1D factor and its sums, the three warps
//           synchronise on a named barrier;
//   pass 2  f^{n+1} = b f~ + a Phi, Phi = px[jx] py[jy] pz[jz], on the f~
//           values pass 1 parked in the cell's output slots (each thread
//           rereads its own writes, from L2).
#include "bgk_device.cuh"

namespace bgk {

namespace {

constexpr int kT = 256;  // threads per CTA
constexpr int kW = kT / 32;

struct Idx3 {
  int jx, jy, jz;
};
__device__ __forceinline__ Idx3 split3(const Params3v& P, int j) {
  const int jyz = j / P.nvx;
  const int jz = jyz / P.nvy;
  return {j - jyz * P.nvx, jyz - jz * P.nvy, jz};
}

// f~ at velocity j of cell i: Eq. (exact) shift by [C], Eq. (upwind) with
// the remainder |C - [C]| toward the upwind side.
__device__ __forceinline__ double stream3(const Params3v& P, const Tables3v& T, const double* __restrict__ fin,
                                          int i, int j, int jx) {
  const int i1 = i - T.shift[jx];
  const int i2 = i1 - T.upwind[jx];
  const double f1 = i1 < 0 ? T.ghost[j] : i1 >= P.nx ? T.ghost[P.nv + j] : fin[(size_t)i1 * P.nv + j];
  const double f2 = i2 < 0 ? T.ghost[j] : i2 >= P.nx ? T.ghost[P.nv + j] : fin[(size_t)i2 * P.nv + j];
  return fma(T.rem[jx], f2 - f1, f1);
}

// Sums of N values over the CTA in a fixed order, totals in out (all threads).
__device__ __forceinline__ void cta_sum8(const double (&v)[8], double* red, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double x = warp_reduce8(v);  // lane 4k + r holds total k
  if ((lane & 3) == 0) red[warp * 8 + (lane >> 2)] = x;
  __syncthreads();
  if (threadIdx.x < 8) {
    double t = 0.0;
    for (int w = 0; w < kW; ++w) t += red[w * 8 + threadIdx.x];
    out[threadIdx.x] = t;
  }
  __syncthreads();
}

__device__ __forceinline__ int axis_n(const Params3v& P, int a) { return a == 0 ? P.nvx : a == 1 ? P.nvy : P.nvz; }

// The three warps' barrier (warps 0..2, 96 threads).
__device__ __forceinline__ void bar_axes() { asm volatile("bar.sync 1, 96;" ::: "memory"); }

// Warp `a` (0..2): 1D Gaussian e_j = exp(-(c_j - u)^2 / theta) of its axis
// at p; returns the warp totals (sum e, sum d e, sum d^2 e) in every lane and
// leaves e_j in fac (when not null).
__device__ __forceinline__ void axis_sums(const Params3v& P, const Tables3v& T, int a, double u, double inv_th,
                                          double* fac, double (&s)[3]) {
  const int lane = threadIdx.x & 31;
  s[0] = s[1] = s[2] = 0.0;
  for (int j = lane; j < axis_n(P, a); j += 32) {
    const double d = T.c[a][j] - u;
    const double e = exp(-(d * d) * inv_th);
    if (fac) fac[j] = e;
    s[0] += e;
    s[1] = fma(d, e, s[1]);
    s[2] = fma(d * d, e, s[2]);
  }
  for (int k = 0; k < 3; ++k)
    for (int m = 16; m > 0; m >>= 1) s[k] += __shfl_xor_sync(0xffffffffu, s[k], m);
}

}  // namespace

__global__ void __launch_bounds__(kT) step3v_kernel(const Params3v P, const Tables3v T,
                                                    const double* __restrict__ fin, double* __restrict__ fout,
                                                    double* __restrict__ mom, int* __restrict__ err) {
  extern __shared__ double fac[];  // px[nvx], py[nvy], pz[nvz]
  __shared__ double red[kW * 8], tot[8];
  __shared__ double s_ax[3][3];   // per axis: sum e, sum d e, sum d^2 e
  __shared__ double s_ab[2];      // relaxation weights a (on Phi), b (on f~)
  __shared__ int s_ok;
  const int i = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // pass 1: stream (f~ parked in the cell's output slots) and the five sums
  // of Eq. (macroscopic)
  double* fo = fout + (size_t)i * P.nv;
  double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int j = threadIdx.x; j < P.nv; j += kT) {
    const Idx3 k = split3(P, j);
    const double ft = stream3(P, T, fin, i, j, k.jx);
    fo[j] = ft;
    acc[0] += ft;
    acc[1] = fma(T.c[0][k.jx], ft, acc[1]);
    acc[2] = fma(T.c[1][k.jy], ft, acc[2]);
    acc[3] = fma(T.c[2][k.jz], ft, acc[3]);
    acc[4] = fma(T.c2[j], ft, acc[4]);
  }
  cta_sum8(acc, red, tot);

  // per-cell parameters, warps 0..2 (warp a works on axis a)
  if (warp < 3) {
    const double n = tot[0] * P.dv;
    const double q[5] = {n, tot[1] / tot[0], tot[2] / tot[0], tot[3] / tot[0],
                         (2.0 / 3.0) * (tot[4] / tot[0] -
                                        ((tot[1] / tot[0]) * (tot[1] / tot[0]) + (tot[2] / tot[0]) * (tot[2] / tot[0]) +
                                         (tot[3] / tot[0]) * (tot[3] / tot[0])))};
    bool ok = q[0] > 0.0 && q[4] > 0.0 && isfinite(q[0]) && isfinite(q[1]) && isfinite(q[2]) && isfinite(q[3]) &&
              isfinite(q[4]);
    double p[5] = {q[0], q[1], q[2], q[3], q[4]};
    if (!ok) {
      p[0] = 1.0;
      p[1] = p[2] = p[3] = 0.0;
      p[4] = 1.0;
    }
    bool fail_eff = false;
    if (ok && P.conservative) {
      const double vs = sqrt(q[4]);
      for (int it = 1; it <= kEffMaxIt; ++it) {
        double s[3];
        axis_sums(P, T, warp, p[1 + warp], 1.0 / p[4], nullptr, s);
        if (lane == 0)
          for (int m = 0; m < 3; ++m) s_ax[warp][m] = s[m];
        bar_axes();
        double d[5];
        const double S0 = s_ax[0][0] * s_ax[1][0] * s_ax[2][0];
        d[0] = p[0] / (kPi() * p[4] * sqrt(kPi() * p[4])) * P.dv * S0;
        double th = 0.0;
        for (int a = 0; a < 3; ++a) {
          const double mu = s_ax[a][1] / s_ax[a][0];
          d[1 + a] = p[1 + a] + mu;
          th += s_ax[a][2] / s_ax[a][0] - mu * mu;
        }
        d[4] = (2.0 / 3.0) * th;
        bar_axes();  // s_ax is rewritten by the next iteration
        double r = 0.0;
        for (int m = 0; m < 5; ++m) {
          const double delta = q[m] - d[m];
          p[m] += delta;
          r = fmax(r, fabs(delta) / (m == 0 ? q[0] : m == 4 ? q[4] : vs));
        }
        if (!(p[0] > 0.0) || !(p[4] > 0.0) || !isfinite(r)) {
          fail_eff = true;
          break;
        }
        if (r < kEffTol) break;
        if (it == kEffMaxIt && r >= kEffFail) fail_eff = true;
      }
    }
    if (fail_eff) ok = false;
    // factors at the final p: px carries a n (pi theta)^(-3/2)
    const double nu = q[0] * pow(q[4], 1.0 - P.omega);
    const double a = !ok ? 0.0 : P.relax_exact ? 1.0 - exp(-nu * P.dt) : nu * P.dt;
    const double b = !ok ? 1.0 : P.relax_exact ? exp(-nu * P.dt) : 1.0 - a;
    double* fw = fac + (warp == 0 ? 0 : warp == 1 ? P.nvx : P.nvx + P.nvy);
    double s[3];
    axis_sums(P, T, warp, p[1 + warp], 1.0 / p[4], fw, s);
    if (warp == 0) {
      __syncwarp();
      const double scale = a * p[0] / (kPi() * p[4] * sqrt(kPi() * p[4]));
      for (int j = lane; j < P.nvx; j += 32) fw[j] *= scale;
      if (lane == 0) {
        s_ab[0] = a;
        s_ab[1] = b;
        s_ok = ok ? 1 : 0;
        mom[(size_t)i * 5 + 0] = q[0];
        mom[(size_t)i * 5 + 1] = q[1];
        mom[(size_t)i * 5 + 2] = q[2];
        mom[(size_t)i * 5 + 3] = q[3];
        mom[(size_t)i * 5 + 4] = q[4];
        if (!ok) atomicOr(err, fail_eff ? ERR_EFFECTIVE : ERR_MOMENT);
      }
    }
  }
  __syncthreads();

  // pass 2: f^{n+1} = b f~ + a Phi, each thread on the f~ values it parked
  const double b = s_ab[1];
  const double* px = fac;
  const double* py = fac + P.nvx;
  const double* pz = py + P.nvy;
  if (s_ok == 0) return;  // f^{n+1} = f~ (flagged)
  for (int j = threadIdx.x; j < P.nv; j += kT) {
    const Idx3 k = split3(P, j);
    fo[j] = fma(b, fo[j], px[k.jx] * py[k.jy] * pz[k.jz]);
  }
}

// Moments (n, ux, uy, uz, theta) of a state, one CTA per cell.
__global__ void __launch_bounds__(kT) moments3v_kernel(const Params3v P, const Tables3v T,
                                                       const double* __restrict__ f, double* __restrict__ mom) {
  __shared__ double red[kW * 8], tot[8];
  const int i = blockIdx.x;
  double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int j = threadIdx.x; j < P.nv; j += kT) {
    const Idx3 k = split3(P, j);
    const double v = f[(size_t)i * P.nv + j];
    acc[0] += v;
    acc[1] = fma(T.c[0][k.jx], v, acc[1]);
    acc[2] = fma(T.c[1][k.jy], v, acc[2]);
    acc[3] = fma(T.c[2][k.jz], v, acc[3]);
    acc[4] = fma(T.c2[j], v, acc[4]);
  }
  cta_sum8(acc, red, tot);
  if (threadIdx.x == 0) {
    const double ux = tot[1] / tot[0], uy = tot[2] / tot[0], uz = tot[3] / tot[0];
    mom[(size_t)i * 5 + 0] = tot[0] * P.dv;
    mom[(size_t)i * 5 + 1] = ux;
    mom[(size_t)i * 5 + 2] = uy;
    mom[(size_t)i * 5 + 3] = uz;
    mom[(size_t)i * 5 + 4] = (2.0 / 3.0) * (tot[4] / tot[0] - (ux * ux + uy * uy + uz * uz));
  }
}

// 3D Maxwellian n (pi theta)^(-3/2) exp(-|c - U|^2 / theta) at velocity j.
__device__ __forceinline__ double maxwell3(const Params3v& P, const double* c0, const double* c1, const double* c2,
                                           const double s[5], int j) {
  const Idx3 k = split3(P, j);
  const double dx = c0[k.jx] - s[1], dy = c1[k.jy] - s[2], dz = c2[k.jz] - s[3];
  return s[0] / (kPi() * s[4] * sqrt(kPi() * s[4])) * exp(-(dx * dx + dy * dy + dz * dz) / s[4]);
}

// Per-velocity tables: cell centres, |c|^2, Courant shift and remainder,
// inflow Maxwellians of both ends.
__global__ void tables3v_kernel(const Params3v P, double* c0, double* c1, double* c2, double* cc, int* shift,
                                int* upwind, double* rem, double* ghost, Inflow3v inflow) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < P.nvx) {
    const double cx = P.vmin[0] + (j + 0.5) * P.dc[0];
    c0[j] = cx;
    const double C = cx * P.dt / P.dx;
    const int s = (int)C;
    shift[j] = s;
    upwind[j] = C > 0.0 ? 1 : -1;
    rem[j] = fabs(C - s);
  }
  if (j < P.nvy) c1[j] = P.vmin[1] + (j + 0.5) * P.dc[1];
  if (j < P.nvz) c2[j] = P.vmin[2] + (j + 0.5) * P.dc[2];
  if (j < P.nv) {
    const Idx3 k = split3(P, j);
    const double cx = P.vmin[0] + (k.jx + 0.5) * P.dc[0];
    const double cy = P.vmin[1] + (k.jy + 0.5) * P.dc[1];
    const double cz = P.vmin[2] + (k.jz + 0.5) * P.dc[2];
    cc[j] = cx * cx + cy * cy + cz * cz;
  }
}

// Inflow Maxwellians (after the axis tables exist).
__global__ void ghost3v_kernel(const Params3v P, const double* c0, const double* c1, const double* c2,
                               double* ghost, Inflow3v inflow) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= P.nv) return;
  ghost[j] = maxwell3(P, c0, c1, c2, inflow.s[0], j);
  ghost[P.nv + j] = maxwell3(P, c0, c1, c2, inflow.s[1], j);
}

__global__ void init3v_kernel(const Params3v P, const Tables3v T, double x_split, Inflow3v lr, double* f) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)P.nx * P.nv) return;
  const int i = (int)(idx / P.nv), j = (int)(idx % P.nv);
  const double x = P.x0 + (i + 0.5) * P.dx;
  f[idx] = maxwell3(P, T.c[0], T.c[1], T.c[2], lr.s[x < x_split ? 0 : 1], j);
}

cudaError_t launch_tables3v(const Params3v& P, double* c0, double* c1, double* c2, double* cc, int* shift,
                            int* upwind, double* rem, double* ghost, const Inflow3v& inflow, cudaStream_t stream) {
  const int n = P.nv > P.nvx ? P.nv : P.nvx;
  tables3v_kernel<<<(n + 255) / 256, 256, 0, stream>>>(P, c0, c1, c2, cc, shift, upwind, rem, ghost, inflow);
  ghost3v_kernel<<<(P.nv + 255) / 256, 256, 0, stream>>>(P, c0, c1, c2, ghost, inflow);
  return cudaGetLastError();
}

cudaError_t launch_init3v(const Params3v& P, const Tables3v& T, double x_split, const Inflow3v& lr, double* f,
                          cudaStream_t stream) {
  const size_t total = (size_t)P.nx * P.nv;
  init3v_kernel<<<(unsigned)((total + 255) / 256), 256, 0, stream>>>(P, T, x_split, lr, f);
  return cudaGetLastError();
}

cudaError_t launch_step3v(const Params3v& P, const Tables3v& T, const double* fin, double* fout, double* mom,
                          int* err, cudaStream_t stream) {
  const size_t smem = sizeof(double) * (size_t)(P.nvx + P.nvy + P.nvz);
  step3v_kernel<<<P.nx, kT, smem, stream>>>(P, T, fin, fout, mom, err);
  return cudaGetLastError();
}

cudaError_t launch_moments3v(const Params3v& P, const Tables3v& T, const double* f, double* mom,
                             cudaStream_t stream) {
  moments3v_kernel<<<P.nx, kT, 0, stream>>>(P, T, f, mom);
  return cudaGetLastError();
}

}  // namespace bgk
