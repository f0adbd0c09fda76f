// bgk_mixed.cu - the reduced-precision BGK step (2D): the state is stored as
// FP32 (g, h) pairs, or as BF16 deviations (dg, dh) from the absolute
// Maxwellian M_abs (n = 1, U = 0, theta = 1), and streamed and relaxed on the
// FP32 pipe.  Moment sums are carried as float-float pairs by error-free
// transformations (Kahan per lane, TwoSum across lanes: about 48 significant
// bits); the pairs are published per cell, and bgk_moments finishes them in
// FP64 on request, while the step itself rounds each sum once to FP32 and
// forms n, U, theta, nu and the relaxation weight in FP32.  The effective
// Maxwellian parameters are two FP32 updates; its normalisation a n/(pi
// theta) is evaluated in float-float and rounded once to FP32; the Gaussian
// factors are FP32.
//
// Conservation in low precision: streaming uses the flux form
// f~ = f - ax (f - f_upx) - ay (f - f_upy), which telescopes whatever the
// rounded weights, and relaxation uses f^{n+1} = f~ + (a Phi - a f~), whose
// mass change is only the rounding of each term (no systematic drift from
// weights that do not sum to 1).
//
// Each lane handles groups of 4 consecutive velocities (one row, one sign
// of c_x and c_y: the velocity grid has nvx % 8 == 0 and sign changes on
// multiples of 4, checked on the host).  Two kernels: a block of G cells per
// CTA (8 / G warps per cell, f~ kept in registers between streaming and
// relaxation), and for one cell per CTA a pipelined kernel that streams the
// next cell while two extra warps solve the previous cell's parameters (f~
// in shared memory).  Both run the same arithmetic in the same order.
#include <cuda_bf16.h>

#include "bgk_device.cuh"

namespace bgk {

namespace {

__device__ __forceinline__ int vi_jx(int vi) { return vi & 0xfff; }
__device__ __forceinline__ int vi_jy(int vi) { return (vi >> 12) & 0xfff; }
__device__ __forceinline__ int vi_sx(int vi) { return ((vi >> 24) & 3) - 1; }
__device__ __forceinline__ int vi_sy(int vi) { return ((vi >> 26) & 3) - 1; }

// ---- error-free FP32 arithmetic ----------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bp = s - a;
  e = (a - (s - bp)) + (b - bp);
}
// (h, l) += (bh, bl), renormalised
__device__ __forceinline__ void ff_add(float& h, float& l, float bh, float bl) {
  float s, e;
  two_sum(h, bh, s, e);
  e += l + bl;
  h = s + e;
  l = e - (h - s);
}
// Kahan: (s, c) accumulates x; the sum is s - c
__device__ __forceinline__ void kahan(float& s, float& c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}
__device__ __forceinline__ void ff_xor(float& h, float& l, int m) {
  const float oh = __shfl_xor_sync(0xffffffffu, h, m);
  const float ol = __shfl_xor_sync(0xffffffffu, l, m);
  ff_add(h, l, oh, ol);
}
// Four float-float values per lane -> lane L holds the warp total of value
// (L >> 3) & 3 (recursive halving, as warp_reduce4).
__device__ __forceinline__ void warp_reduce4_ff(float (&h)[4], float (&l)[4], float& oh, float& ol) {
  const int lane = threadIdx.x & 31;
  const bool b4 = lane & 16, b3 = lane & 8;
  float ah[2], al[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float sh = __shfl_xor_sync(0xffffffffu, b4 ? h[k] : h[k + 2], 16);
    const float sl = __shfl_xor_sync(0xffffffffu, b4 ? l[k] : l[k + 2], 16);
    ah[k] = b4 ? h[k + 2] : h[k];
    al[k] = b4 ? l[k + 2] : l[k];
    ff_add(ah[k], al[k], sh, sl);
  }
  const float sh = __shfl_xor_sync(0xffffffffu, b3 ? ah[0] : ah[1], 8);
  const float sl = __shfl_xor_sync(0xffffffffu, b3 ? al[0] : al[1], 8);
  oh = b3 ? ah[1] : ah[0];
  ol = b3 ? al[1] : al[0];
  ff_add(oh, ol, sh, sl);
  ff_xor(oh, ol, 4);
  ff_xor(oh, ol, 2);
  ff_xor(oh, ol, 1);
}

// ---- (g, h) pairs on the paired FP32 pipe ------------------------------------
// FFMA2 / FADD2 / FMUL2 apply one FP32 operation to both members of a pair
// with the rounding of the scalar operation, so these give the results of
// the scalar code at half the instructions.
__device__ __forceinline__ float2 splat(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

// ---- storage --------------------------------------------------------------
template <int PREC>
struct Store;

// FP32 storage order inside a cell's block (2D): the velocities come in
// groups of 4 (one row, one sign of c_x and c_y) and the groups in chunks of
// 32; a chunk of cs groups stores the first two velocities of each group
// (16 bytes, group after group), then the last two.  The 32 lanes of a warp
// take the 32 groups of a chunk, so each 16-byte access of the warp covers
// 512 contiguous bytes (4 L1 wavefronts) instead of 1 KB at a 32-byte
// stride.  Offsets are in float2 units from the start of the cell's block.
__host__ __device__ __forceinline__ int f32_half(int g, int ngroups, int half) {
  const int q = g >> 5, cs = min(32, ngroups - 32 * q);
  return 128 * q + 2 * (g & 31) + half * 2 * cs;
}
__host__ __device__ __forceinline__ int f32_pos(int j, int ngroups) {
  return f32_half(j >> 2, ngroups, (j >> 1) & 1) + (j & 1);
}

template <>
struct Store<PREC_F32> {
  static constexpr bool delta = false;
  // the 4 velocities j0..j0+3 (j0 = 4 g) of the cell whose block starts at c0
  __device__ static void load4(const void* base, size_t c0, int j0, int ng, float2 (&v)[4]) {
    const float2* b = static_cast<const float2*>(base) + c0;
    const int g = j0 >> 2;
    const float4 a = __ldg(reinterpret_cast<const float4*>(b + f32_half(g, ng, 0)));
    const float4 c = __ldg(reinterpret_cast<const float4*>(b + f32_half(g, ng, 1)));
    v[0] = make_float2(a.x, a.y);
    v[1] = make_float2(a.z, a.w);
    v[2] = make_float2(c.x, c.y);
    v[3] = make_float2(c.z, c.w);
  }
  __device__ static void store4(void* base, size_t c0, int j0, int ng, const float2 (&v)[4]) {
    float2* b = static_cast<float2*>(base) + c0;
    const int g = j0 >> 2;
    *reinterpret_cast<float4*>(b + f32_half(g, ng, 0)) = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
    *reinterpret_cast<float4*>(b + f32_half(g, ng, 1)) = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
  }
  __device__ static float2 load1(const void* base, size_t c0, int j, int ng) {
    return __ldg(static_cast<const float2*>(base) + c0 + f32_pos(j, ng));
  }
};

template <>
struct Store<PREC_BF16> {
  static constexpr bool delta = true;
  __device__ static float2 unpack(unsigned w) {
    __nv_bfloat162 b;
    memcpy(&b, &w, 4);
    return __bfloat1622float2(b);
  }
  __device__ static unsigned pack(float2 v) {
    const __nv_bfloat162 b = __float22bfloat162_rn(v);
    unsigned w;
    memcpy(&w, &b, 4);
    return w;
  }
  // one 32-bit word per velocity in velocity order (ng unused)
  __device__ static void load4(const void* base, size_t c0, int j0, int, float2 (&v)[4]) {
    const uint4 u = __ldg(reinterpret_cast<const uint4*>(static_cast<const unsigned*>(base) + c0 + j0));
    v[0] = unpack(u.x);
    v[1] = unpack(u.y);
    v[2] = unpack(u.z);
    v[3] = unpack(u.w);
  }
  __device__ static void store4(void* base, size_t c0, int j0, int, const float2 (&v)[4]) {
    *reinterpret_cast<uint4*>(static_cast<unsigned*>(base) + c0 + j0) =
        make_uint4(pack(v[0]), pack(v[1]), pack(v[2]), pack(v[3]));
  }
  __device__ static float2 load1(const void* base, size_t c0, int j, int) {
    return unpack(__ldg(static_cast<const unsigned*>(base) + c0 + j));
  }
};

// Boundary value at velocity j in the stored representation (full value, or
// deviation from M_abs for the BF16 form).
template <int PREC>
__device__ __forceinline__ float2 ghost_m(const Params& P, const MixedTables& M, int face, int j,
                                          float nw, const void* fin, size_t c0) {
  const int kind = P.bc_kind[face];
  if (kind == BC_SPECULAR) {
    const int vi = M.vinfo[j];
    const int jx = vi_jx(vi), jy = vi_jy(vi);
    const int jr = (face == XLO || face == XHI) ? jy * P.nvx + (P.nvx - 1 - jx)
                                                : (P.nvy - 1 - jy) * P.nvx + jx;
    return Store<PREC>::load1(fin, c0, jr, P.nv >> 2);  // M_abs is mirror symmetric
  }
  float2 g = M.ghost[face * P.nv + j];
  if (kind == BC_DIFFUSE) g = make_float2(nw * g.x, nw * g.y);
  if (Store<PREC>::delta) {
    const float2 m = M.mabs[j];
    g = make_float2(g.x - m.x, g.y - m.y);
  }
  return g;
}

// ---- the step --------------------------------------------------------------
// A CTA holds G cells and 8 warps, WPC = 8/G warps per cell.  The velocities
// of a cell come in groups of 4 consecutive indices (one row, one sign of c_x
// and c_y); group k goes to lane k mod (32 WPC) of the cell's warps, at most
// MGL groups per lane, and f~ of those groups stays in that lane's registers
// from streaming (phase 1) to relaxation (phase 3).  Phase 2 runs on the
// cell's first warp, on the FP32 pipe except the normalisation.

// Bytes of the Gaussian factors of G cells in shared memory.
__host__ __device__ __forceinline__ size_t mixed_factor_bytes(const Params& P, int G) {
  return (sizeof(float) * (size_t)G * (P.nvx + P.nvy) + 15) & ~(size_t)15;
}

// Where a cell sits: which faces it touches, and n_W of its diffuse faces.
struct CellCtx {
  size_t c0, row;
  bool bxlo, bxhi, bylo, byhi, interior;
  float nw[4];
};

// The flux form of A1 for the 4 velocities of a group (row jy, columns
// jx0..jx0+3; vi = vinfo of its first velocity) from their own and upwind
// values; the weights come from the per-axis tables (one 16-byte load for
// the 4 columns).
__device__ __forceinline__ void flux_form(const MixedTables& M, int vi, const float2 (&f0)[4],
                                          const float2 (&fx)[4], const float2 (&fy)[4], float2 (&ft)[4]) {
  const float4 a4 = *reinterpret_cast<const float4*>(M.ax + vi_jx(vi));
  const float ax[4] = {a4.x, a4.y, a4.z, a4.w};
  const float ay = M.ay[vi_jy(vi)];
  const float2 m1 = splat(-1.f), nay = splat(-ay);
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const float2 dx = fma2(fx[p], m1, f0[p]);  // f - f_upx, rounded once
    const float2 dy = fma2(fy[p], m1, f0[p]);
    ft[p] = fma2(nay, dy, fma2(splat(-ax[p]), dx, f0[p]));
  }
}

__device__ __forceinline__ void unpack_f32(const float4& lo, const float4& hi, float2 (&v)[4]) {
  v[0] = make_float2(lo.x, lo.y);
  v[1] = make_float2(lo.z, lo.w);
  v[2] = make_float2(hi.x, hi.y);
  v[3] = make_float2(hi.z, hi.w);
}

// A1 for the 4 velocities j0..j0+3 of one cell, flux form
//   f~ = f - ax (f - f_upx) - ay (f - f_upy)
// in the stored representation (deviations for BF16).
template <int PREC>
__device__ __forceinline__ void stream_group(const Params& P, const MixedTables& M, const void* fin,
                                             const CellCtx& C, int j0, int vi, float2 (&ft)[4]) {
  using S = Store<PREC>;
  const int nv = P.nv;
  const int sgx = vi_sx(vi), sgy = vi_sy(vi);
  float2 f0[4], fx[4], fy[4];
  const int ng = nv >> 2;
  S::load4(fin, C.c0, j0, ng, f0);
  if (C.interior) {
    S::load4(fin, C.c0 - (ptrdiff_t)sgx * nv, j0, ng, fx);
    S::load4(fin, C.c0 - (ptrdiff_t)sgy * (ptrdiff_t)C.row, j0, ng, fy);
  } else {
    if (sgx > 0 && !C.bxlo) S::load4(fin, C.c0 - nv, j0, ng, fx);
    else if (sgx < 0 && !C.bxhi) S::load4(fin, C.c0 + nv, j0, ng, fx);
    else if (sgx == 0) {
#pragma unroll
      for (int p = 0; p < 4; ++p) fx[p] = f0[p];
    } else {
      const int face = sgx > 0 ? XLO : XHI;
      const float nw = sgx > 0 ? C.nw[XLO] : C.nw[XHI];
#pragma unroll
      for (int p = 0; p < 4; ++p) fx[p] = ghost_m<PREC>(P, M, face, j0 + p, nw, fin, C.c0);
    }
    if (sgy > 0 && !C.bylo) S::load4(fin, C.c0 - C.row, j0, ng, fy);
    else if (sgy < 0 && !C.byhi) S::load4(fin, C.c0 + C.row, j0, ng, fy);
    else if (sgy == 0) {
#pragma unroll
      for (int p = 0; p < 4; ++p) fy[p] = f0[p];
    } else {
      const int face = sgy > 0 ? YLO : YHI;
      const float nw = sgy > 0 ? C.nw[YLO] : C.nw[YHI];
#pragma unroll
      for (int p = 0; p < 4; ++p) fy[p] = ghost_m<PREC>(P, M, face, j0 + p, nw, fin, C.c0);
    }
  }
  flux_form(M, vi, f0, fx, fy, ft);
}

// A2 for the 4 velocities j0..j0+3: their contributions to the lane's FP32
// partial sums s01 = (sum g, sum c_x g), s23 = (sum c_y g, sum |c|^2 g + h).
// A lane sums at most 4 MGL velocities of a cell this way; the lanes'
// partials are then combined in float-float (warp_reduce4_ff and the tree
// over the cell's warps).
__device__ __forceinline__ void group_sums(const MixedTables& M, int vi, const float2 (&ft)[4], float2& s01,
                                           float2& s23) {
  const float4 c4 = *reinterpret_cast<const float4*>(M.cx + vi_jx(vi));
  const float cx[4] = {c4.x, c4.y, c4.z, c4.w};
  const float cy = M.cy[vi_jy(vi)];
  const float cy2 = cy * cy;
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const float2 gg = splat(ft[p].x);
    s01 = fma2(make_float2(1.f, cx[p]), gg, s01);
    s23 = fma2(make_float2(cy, fmaf(cx[p], cx[p], cy2)), gg, s23);
    s23.y += ft[p].y;
  }
}

// A1 + A2 for the 4 velocities j0..j0+3: f~ into ft, their contributions
// to the lane's Kahan sums.
template <int PREC>
__device__ __forceinline__ void stream_sum_group(const Params& P, const MixedTables& M, const void* fin,
                                                 const CellCtx& C, int j0, float2 (&ft)[4], float2& s01,
                                                 float2& s23) {
  const int vi = M.vinfo[j0];
  stream_group<PREC>(P, M, fin, C, j0, vi, ft);
  group_sums(M, vi, ft, s01, s23);
}

// A4 for the 4 velocities j0..j0+3: r holds f~ (stored representation) and
// becomes f~ + (a Phi - a f~), Phi_g = px[jx] py[jy] (the factors carry
// a n / (pi theta)), Phi_h = kappa Phi_g.
template <int PREC>
__device__ __forceinline__ void relax_group(const MixedTables& M, const float* px, const float* py, int j0,
                                            float a, float kappa, float2 (&r)[4]) {
  const int vi = M.vinfo[j0];
  const float4 xv = *reinterpret_cast<const float4*>(px + vi_jx(vi));
  const float2 yv = splat(py[vi_jy(vi)]);
  const float2 ph01 = mul2(make_float2(xv.x, xv.y), yv), ph23 = mul2(make_float2(xv.z, xv.w), yv);
  const float ph[4] = {ph01.x, ph01.y, ph23.x, ph23.y};
  float2 mb[4];
  if (Store<PREC>::delta) {
    const float4* m4 = reinterpret_cast<const float4*>(M.mabs + j0);
    unpack_f32(m4[0], m4[1], mb);
  }
  const float2 na = splat(-a), k1 = make_float2(1.f, kappa);
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const float2 f = Store<PREC>::delta ? add2(r[p], mb[p]) : r[p];  // full f~ for the a f~ term
    r[p] = add2(r[p], fma2(na, f, mul2(k1, splat(ph[p]))));     // + (a Phi - a f~), Phi_h = kappa Phi_g
  }
}

// Cell context, with A0: n_W of each diffuse face from the incident flux
// sum |c_n| g over c_n < 0 of the cell's own (full) state (every warp of the
// cell computes it for itself).
template <int PREC>
__device__ __forceinline__ CellCtx cell_ctx(const Params& P, const MixedTables& M, const void* fin, int cell,
                                            int ix, int iy) {
  using S = Store<PREC>;
  const int lane = threadIdx.x & 31;
  const int nv = P.nv, nx = P.nx;
  CellCtx C;
  C.c0 = (size_t)cell * nv;
  C.row = (size_t)nx * nv;
  C.bxlo = ix == 0;
  C.bxhi = ix == nx - 1;
  C.bylo = iy == 0;
  C.byhi = iy == P.ny - 1;
  C.interior = !(C.bxlo || C.bxhi || C.bylo || C.byhi);
  for (int f = 0; f < 4; ++f) C.nw[f] = 0.f;
  unsigned diff = 0;
  if (C.bxlo && P.bc_kind[XLO] == BC_DIFFUSE) diff |= 1u;
  if (C.bxhi && P.bc_kind[XHI] == BC_DIFFUSE) diff |= 2u;
  if (C.bylo && P.bc_kind[YLO] == BC_DIFFUSE) diff |= 4u;
  if (C.byhi && P.bc_kind[YHI] == BC_DIFFUSE) diff |= 8u;
  if (diff) {
    float hs[4] = {0.f, 0.f, 0.f, 0.f}, cs[4] = {0.f, 0.f, 0.f, 0.f};
    for (int j0 = 4 * lane; j0 < nv; j0 += 128) {
      float2 v[4];
      S::load4(fin, C.c0, j0, nv >> 2, v);
      const int vi = M.vinfo[j0];
      float ax = 0.f, ay = 0.f;
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        float g = v[p].x;
        if (S::delta) g += M.mabs[j0 + p].x;
        const float4 co = M.coef[j0 + p];
        ax = fmaf(fabsf(co.z), g, ax);
        ay = fmaf(fabsf(co.w), g, ay);
      }
      if (vi_sx(vi) < 0) kahan(hs[0], cs[0], ax);
      if (vi_sx(vi) > 0) kahan(hs[1], cs[1], ax);
      if (vi_sy(vi) < 0) kahan(hs[2], cs[2], ay);
      if (vi_sy(vi) > 0) kahan(hs[3], cs[3], ay);
    }
    float ls[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) ls[k] = -cs[k];
    float oh, ol;
    warp_reduce4_ff(hs, ls, oh, ol);
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const float th = __shfl_sync(0xffffffffu, oh, 8 * f), tl = __shfl_sync(0xffffffffu, ol, 8 * f);
      if (diff >> f & 1u) C.nw[f] = (float)(((double)th + (double)tl) * P.dv / M.emitted[f]);
    }
  }
  return C;
}

__device__ __forceinline__ float warp_sum_f(float x) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) x += __shfl_xor_sync(0xffffffffu, x, m);
  return x;
}

// Phase 2, the per-cell parameters, spread over the cell's WPC warps in
// three parts separated by CTA barriers (every warp of the CTA calls each
// part; cells outside the grid only take part in the barriers):
//   2a  every warp: the cell's moments from the float-float velocity sums
//       (lane-parallel tree over the warps' partials), nu and the relaxation
//       weight; then one FP32 Gaussian exp(-(c - u)^2 / theta) per lane for
//       the x and y factors, stored to shared memory, and the lane's share
//       of the central sums sum d^m e (m = 0..4) reduced over the warp;
//   2b  the cell's first warp: two linearised effective-parameter updates
//       (A3, FP32: the reduced forms only need the correction to FP32
//       resolution) and the normalisation n / (pi theta), evaluated in
//       float-float (at least 44 significant bits) and rounded once;
//   2c  every warp: the Gaussian factors moved from (u, theta) to the
//       effective parameters and scaled by a n/(pi theta).
// The first warp also publishes the float-float sums (msum) from which
// bgk_moments forms FP64 moments on request.

// Per-cell scalars shared between the parts.
struct CellPar {
  float n, ux, uy, th, a;  // moments of f~ and the relaxation weight
  float ap, w1x, w1y, w2;  // factor update: ap e (1 + d (w1 + d w2))
  float kappa;             // H = kappa G
  int ok;
};

// a * p0 / (pi * p3) with float-float intermediates, rounded once to FP32.
__device__ __forceinline__ float ff_norm(float a, float p0, float p3) {
  const float pi_h = 3.14159274101257324f;  // pi rounded to FP32
  const float pi_l = -8.74227766e-08f;      // pi - pi_h
  const float dh = pi_h * p3;
  const float dl = fmaf(pi_h, p3, -dh) + pi_l * p3;  // pi p3 = dh + dl
  const float nh = a * p0;
  const float nl = fmaf(a, p0, -nh);  // a p0 = nh + nl exactly
  const float rd = __frcp_rn(dh);
  const float q1 = nh * rd;
  float r = fmaf(-q1, dh, nh);  // exact residual of q1 dh
  r = fmaf(-q1, dl, r) + nl;
  return fmaf(r, rd, q1);
}

template <int PREC, int WPC>
__device__ __forceinline__ void cell_moments(const Params& P, const MixedTables& M, int cell, int wc,
                                             const float2 (*part)[4], CellPar& cp, float2* __restrict__ msum) {
  const int lane = threadIdx.x & 31;
  // lane = 4 w + k holds partial w of value k; tree over w
  const int k = lane & 3, w = lane >> 2;
  float h = 0.f, l = 0.f;
  if (w < WPC) {
    const float2 v = part[w][k];
    h = v.x;
    l = v.y;
  }
  if (WPC > 1) ff_xor(h, l, 4);
  if (WPC > 2) ff_xor(h, l, 8);
  if (WPC > 4) ff_xor(h, l, 16);
  if (wc == 0 && lane < 4) msum[(size_t)cell * 4 + lane] = make_float2(h, l);
  if (Store<PREC>::delta) ff_add(h, l, M.mabs_ff[k].x, M.mabs_ff[k].y);
  const float sk = h + l;
  const float S0 = __shfl_sync(0xffffffffu, sk, 0), S1 = __shfl_sync(0xffffffffu, sk, 1);
  const float S2 = __shfl_sync(0xffffffffu, sk, 2), S3 = __shfl_sync(0xffffffffu, sk, 3);
  const float r0 = __frcp_rn(S0);
  float n = S0 * (float)P.dv, ux = S1 * r0, uy = S2 * r0;
  float th = (2.0f / 3.0f) * (S3 * r0 - (ux * ux + uy * uy));
  const bool ok = n > 0.f && th > 0.f && isfinite(n) && isfinite(ux) && isfinite(uy) && isfinite(th);
  if (!ok) {
    n = 1.f;
    ux = uy = 0.f;
    th = 1.f;
  }
  const float nu = n * (P.omega == 0.5 ? sqrtf(th) : powf(th, (float)(1.0 - P.omega)));
  cp.n = n;
  cp.ux = ux;
  cp.uy = uy;
  cp.th = th;
  cp.a = P.relax_exact ? 1.0f - expf(-nu * (float)P.dt) : nu * (float)P.dt;
  cp.ok = ok;
}

// 2a: Gaussian factors at (u, theta) for j = wc*32 + lane, ... (x: j < nvx,
// y: the rest) into px (y factors follow in py); returns the lane's central
// sums (x in Mx, y in My).
template <int WPC>
__device__ __forceinline__ void cell_gauss(const Params& P, const MixedTables& M, int wc, const CellPar& cp,
                                           float* __restrict__ px, float* __restrict__ py, float (&Mx)[5],
                                           float (&My)[5]) {
  const int lane = threadIdx.x & 31;
  const float inv = __frcp_rn(cp.th);
  for (int m = 0; m < 5; ++m) Mx[m] = My[m] = 0.f;
  for (int j = wc * 32 + lane; j < P.nvx + P.nvy; j += WPC * 32) {
    const bool isx = j < P.nvx;
    const float d = isx ? M.cx[j] - cp.ux : M.cy[j - P.nvx] - cp.uy;
    const float e = expf(-(d * d) * inv);
    if (isx) px[j] = e;
    else py[j - P.nvx] = e;
    float t[5];
    t[0] = e;
#pragma unroll
    for (int m = 1; m < 5; ++m) t[m] = t[m - 1] * d;
#pragma unroll
    for (int m = 0; m < 5; ++m) {
      Mx[m] += isx ? t[m] : 0.f;
      My[m] += isx ? 0.f : t[m];
    }
  }
}

// 2b (first warp of the cell): effective parameters and normalisation.
__device__ __forceinline__ void cell_effective(const Params& P, CellPar& cp, const float (&Mx)[5],
                                               const float (&My)[5]) {
  const float dv = (float)P.dv;
  const float inv = __frcp_rn(cp.th);
  const float q[4] = {cp.n, cp.ux, cp.uy, cp.th};
  float p[4] = {cp.n, cp.ux, cp.uy, cp.th};
  bool ok = cp.ok != 0;
  if (P.conservative) {
    for (int it = 0; it < 2; ++it) {
      const float w2 = (p[3] - cp.th) * inv * inv;
      const float w1x = 2.f * (p[1] - cp.ux) * inv, w1y = 2.f * (p[2] - cp.uy) * inv;
      float Sx[3], Sy[3];
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        Sx[m] = Mx[m] + w1x * Mx[m + 1] + w2 * Mx[m + 2];
        Sy[m] = My[m] + w1y * My[m + 1] + w2 * My[m + 2];
      }
      const float rx = __frcp_rn(Sx[0]), ry = __frcp_rn(Sy[0]);
      const float mux = Sx[1] * rx, muy = Sy[1] * ry;
      float d[4];
      d[0] = p[0] * __frcp_rn(3.14159265f * p[3]) * dv * Sx[0] * Sy[0];
      d[1] = cp.ux + mux;
      d[2] = cp.uy + muy;
      d[3] = (2.f / 3.f) * ((Sx[2] * rx - mux * mux) + (Sy[2] * ry - muy * muy) + 0.5f * p[3]);
#pragma unroll
      for (int k = 0; k < 4; ++k) p[k] += q[k] - d[k];
    }
    if (!(p[0] > 0.f) || !(p[3] > 0.f) || !isfinite(p[0]) || !isfinite(p[1]) || !isfinite(p[2]) ||
        !isfinite(p[3]))
      ok = false;
  }
  cp.ok = ok;
  cp.ap = ok ? ff_norm(cp.a, p[0], p[3]) : 0.f;
  cp.w2 = (p[3] - cp.th) * inv * inv;
  cp.w1x = 2.f * (p[1] - cp.ux) * inv;
  cp.w1y = 2.f * (p[2] - cp.uy) * inv;
  cp.kappa = 0.5f * p[3];
}

// 2c: move the factors to the effective parameters and scale by ap.
template <int WPC>
__device__ __forceinline__ void cell_factors(const Params& P, const MixedTables& M, int wc, const CellPar& cp,
                                             float* __restrict__ px, float* __restrict__ py) {
  const int lane = threadIdx.x & 31;
  for (int j = wc * 32 + lane; j < P.nvx + P.nvy; j += WPC * 32) {
    if (j < P.nvx) {
      const float d = M.cx[j] - cp.ux;
      px[j] = cp.ap * (px[j] * fmaf(d, fmaf(d, cp.w2, cp.w1x), 1.0f));
    } else {
      const float d = M.cy[j - P.nvx] - cp.uy;
      py[j - P.nvx] = py[j - P.nvx] * fmaf(d, fmaf(d, cp.w2, cp.w1y), 1.0f);
    }
  }
}

// Stochastic rounding of an FP32 pair (g, h) to two BF16 values packed in
// one word: 16 bits of dither are added below the kept bits of each value's
// magnitude and the top halves kept.  Rounding away from zero happens with
// probability equal to the discarded fraction, so the rounding is unbiased
// and per-step updates smaller than half a BF16 ulp of the deviation survive
// on average instead of being rounded away every step.  Both dithers come
// from one 32-bit hash of the pair's bits and its position (a
// multiply-xorshift mix in the style of MurmurHash3's finaliser): the low
// half for g, the high half for h.  The conversion instruction with the
// .rs rounding mode (sm_100 and later) does the add, truncate and pack in
// one; it takes the low 16 random bits for its second operand and the high
// 16 for its first, the same split as adding the halves by hand (checked
// bit for bit against that on the GPU).
__device__ __forceinline__ unsigned bf16x2_sr(float2 v, unsigned salt) {
  const unsigned ug = __float_as_uint(v.x), uh = __float_as_uint(v.y);
  unsigned k = (ug ^ salt) * 0x9E3779B1u + uh;
  k ^= k >> 15;
  k *= 0x85EBCA6Bu;
  k ^= k >> 13;
  k *= 0xC2B2AE35u;
  k ^= k >> 16;
  unsigned w;
  asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(w) : "f"(v.y), "f"(v.x), "r"(k));
  return w;
}

// The dither's salt: the velocity point's position plus the step counter
// times 2^32 / golden ratio, so that a value that recurs step after step
// (a nearly stationary deviation) meets a different dither every step;
// with the position alone it would be rounded the same way every step and
// updates below half an ulp would be lost for good.
template <int PREC>
__device__ __forceinline__ void store_result(void* fout, size_t c0, int j0, int ng, const float2 (&r)[4],
                                             unsigned step) {
  if (PREC == PREC_BF16) {
    const size_t idx = c0 + j0;
    const unsigned salt = (unsigned)idx + step * 0x9E3779B9u;
    unsigned w[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) w[p] = bf16x2_sr(r[p], salt + (unsigned)p);
    *reinterpret_cast<uint4*>(static_cast<unsigned*>(fout) + idx) = make_uint4(w[0], w[1], w[2], w[3]);
  } else {
    Store<PREC>::store4(fout, c0, j0, ng, r);
  }
}

}  // namespace

// Step counter of the BF16 dither: every CTA reads word `parity`, one
// thread writes the next value to the other word for the next step's
// kernel (which reads it with the opposite parity).
template <int PREC>
__device__ __forceinline__ unsigned step_counter(const MixedTables& M, int parity) {
  if (PREC != PREC_BF16 || !M.step_ctr) return 0u;
  const unsigned c = *(volatile const unsigned*)(M.step_ctr + parity);
  if (blockIdx.x == 0 && threadIdx.x == 0) M.step_ctr[parity ^ 1] = c + 1u;
  return c;
}

// Shared scratch of one block of G cells (WPC = 8/G warps per cell).
template <int G>
struct MixedShared {
  float2 part[G][8 / G][4];  // float-float partial moment sums per warp
  float gp[G][8 / G][10];    // central sums of the Gaussian factors per warp
  CellPar cp[G];             // per-cell parameters
};

// One block of G cells of a 2D reduced-precision step (all 256 threads of
// the CTA; phx holds G (nvx + nvy) floats).  Used by the per-instance kernel
// below and by the persistent batch kernel.
template <int PREC, int G, int MGL>
__device__ __forceinline__ void mixed2d_block(const Params& P, const MixedTables& M, const void* __restrict__ fin,
                                              void* __restrict__ fout, float2* __restrict__ msum,
                                              int* __restrict__ err, int blk, float* phx, MixedShared<G>& S,
                                              unsigned step) {
  constexpr int WPC = 8 / G;
  float* phy = phx + G * P.nvx;
  auto& s_part = S.part;
  auto& s_gp = S.gp;
  auto& s_cp = S.cp;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = warp / WPC, wc = warp % WPC;
  const int cell = blk * G + c;
  const bool live = cell < P.nx * P.ny;
  const int ngroups = P.nv >> 2;
  const int lic = wc * 32 + lane;

  float2 ft[MGL][4];
  CellCtx C;
  if (live) {
    C = cell_ctx<PREC>(P, M, fin, cell, cell % P.nx, cell / P.nx);
    // A1 + A2: stream this lane's groups, float-float moment sums
    float2 s01 = make_float2(0.f, 0.f), s23 = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < MGL; ++k) {
      const int g = lic + k * 32 * WPC;
      if (g < ngroups) stream_sum_group<PREC>(P, M, fin, C, 4 * g, ft[k], s01, s23);
    }
    float hs[4] = {s01.x, s01.y, s23.x, s23.y}, ls[4] = {0.f, 0.f, 0.f, 0.f};
    float oh, ol;
    warp_reduce4_ff(hs, ls, oh, ol);
    if ((lane & 7) == 0) s_part[c][wc][lane >> 3] = make_float2(oh, ol);
  }
  __syncthreads();
  // phase 2 (see cell_moments .. cell_factors)
  float* pxc = phx + c * P.nvx;
  float* pyc = phy + c * P.nvy;
  CellPar cp;
  if (live) {
    cell_moments<PREC, WPC>(P, M, cell, wc, s_part[c], cp, msum);
    float Mx[5], My[5];
    cell_gauss<WPC>(P, M, wc, cp, pxc, pyc, Mx, My);
    // warp totals of the 10 central sums: lane 4 m + (0: x, 1: y) picks them up
#pragma unroll
    for (int m = 0; m < 5; ++m) {
      Mx[m] = warp_sum_f(Mx[m]);
      My[m] = warp_sum_f(My[m]);
    }
    if (lane < 10) s_gp[c][wc][lane] = lane < 5 ? Mx[lane] : My[lane - 5];
  }
  __syncthreads();
  if (live && wc == 0) {
    float Mx[5], My[5];
#pragma unroll
    for (int m = 0; m < 5; ++m) {
      Mx[m] = s_gp[c][0][m];
      My[m] = s_gp[c][0][5 + m];
      for (int w = 1; w < WPC; ++w) {
        Mx[m] += s_gp[c][w][m];
        My[m] += s_gp[c][w][5 + m];
      }
    }
    cell_effective(P, cp, Mx, My);
    if (lane == 0) {
      s_cp[c] = cp;
      if (!cp.ok) atomicOr(err, ERR_MOMENT);
    }
  }
  __syncthreads();
  if (live) {
    cp = s_cp[c];
    if (cp.ok) cell_factors<WPC>(P, M, wc, cp, pxc, pyc);
  }
  __syncthreads();
  if (!live) return;

  // A4: f^{n+1} = f~ + (a Phi - a f~)
  const float a = cp.a, kappa = cp.kappa;
  const bool ok = cp.ok != 0;
  const float* px = pxc;
  const float* py = pyc;
#pragma unroll
  for (int k = 0; k < MGL; ++k) {
    const int g = lic + k * 32 * WPC;
    if (g < ngroups) {
      const int j0 = 4 * g;
      float2 r[4] = {ft[k][0], ft[k][1], ft[k][2], ft[k][3]};
      if (ok) relax_group<PREC>(M, px, py, j0, a, kappa, r);
      store_result<PREC>(fout, C.c0, j0, ngroups, r, step);
    }
  }
}

// 768 resident threads per SM at most 80 registers each; FP32 with 6 groups
// per lane gets 128 registers and 2 CTAs per SM instead (measured faster than
// spilling; BF16 keeps 3 CTAs and spills a little, also measured).
template <int PREC, int G, int MGL>
__global__ void __launch_bounds__(256, (PREC == PREC_F32 && MGL >= 6) ? 2 : 3)
    step_mixed_kernel(const void* __restrict__ fin, void* __restrict__ fout, float2* __restrict__ msum,
                      const Params P, const MixedTables M, int* __restrict__ err, int parity) {
  extern __shared__ float4 smemf4[];
  __shared__ MixedShared<G> S;
  const unsigned step = step_counter<PREC>(M, parity);
  mixed2d_block<PREC, G, MGL>(P, M, fin, fout, msum, err, blockIdx.x, reinterpret_cast<float*>(smemf4), S, step);
}

// ---- 2D, one cell at a time, pipelined ----------------------------------------
// A resident CTA of 8 streaming warps and two parameter warps walks over the
// cells blockIdx.x, blockIdx.x + gridDim.x, ...  The streaming warps stream
// cell i+1 (A1 + A2) while a parameter warp solves cell i's parameters
// (phase 2); they then relax cell i (A4) from its buffer.  The two
// parameter warps take the cells in turn, each owning one buffer of each
// kind (f~, partial sums, factors), so each has two cells' time for its
// serial phase.  Named barriers hand the sums over (ids 1, 2: the 256
// streaming threads arrive, the owning parameter warp waits) and the
// factors back (ids 3, 4: that warp arrives, the 256 wait).
//
// Every value is computed as in the one-cell block (same velocity-to-thread
// map, same summation order), so the two give identical states; the
// persistent batch kernel runs the block.
constexpr int kPipeMath = 2;
constexpr size_t kPipeMaxSmem = 72 * 1024;  // dynamic shared memory of one pipelined CTA at most

// Barrier ids and thread counts as immediates (a register id would reserve
// all 16); NT threads take part: the streaming warps and one parameter warp.
template <int NT>
__device__ __forceinline__ void bar_sync_id(int id) {
  switch (id) {
    case 1: asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory"); break;
    case 2: asm volatile("bar.sync 2, %0;" ::"n"(NT) : "memory"); break;
    case 3: asm volatile("bar.sync 3, %0;" ::"n"(NT) : "memory"); break;
    default: asm volatile("bar.sync 4, %0;" ::"n"(NT) : "memory"); break;
  }
}
template <int NT>
__device__ __forceinline__ void bar_arrive_id(int id) {
  switch (id) {
    case 1: asm volatile("bar.arrive 1, %0;" ::"n"(NT) : "memory"); break;
    case 2: asm volatile("bar.arrive 2, %0;" ::"n"(NT) : "memory"); break;
    case 3: asm volatile("bar.arrive 3, %0;" ::"n"(NT) : "memory"); break;
    default: asm volatile("bar.arrive 4, %0;" ::"n"(NT) : "memory"); break;
  }
}

// Dynamic shared memory: float4 f~[2 buffers][2 planes][nv / 4] (plane 0
// holds velocities 0, 1 of a group of 4 and plane 1 velocities 2, 3, so
// consecutive threads touch consecutive words), then float factors[2][nvx + nvy].
__host__ __device__ __forceinline__ size_t pipe_smem_bytes(const Params& P) {
  return sizeof(float4) * 4 * (size_t)(P.nv / 4) + ((sizeof(float) * 2 * (size_t)(P.nvx + P.nvy) + 15) & ~(size_t)15);
}

template <int NSW>
constexpr int pipe_threads() { return 32 * (NSW + kPipeMath); }

// NSW streaming warps (group g of a cell goes to thread g mod 32 NSW, as in
// the block of 8 / NSW cells per CTA) and two parameter warps.
template <int PREC, int MGL, int NSW>
__global__ void __launch_bounds__(pipe_threads<NSW>(), NSW == 8 ? 3 : 4)
    step_mixed_pipe_kernel(const void* __restrict__ fin, void* __restrict__ fout, float2* __restrict__ msum,
                           const Params P, const MixedTables M, int* __restrict__ err, int parity) {
  constexpr int NT = 32 * (NSW + 1);
  constexpr int NST = 32 * NSW;
  extern __shared__ float4 smemf4[];
  __shared__ float2 s_part[2][NSW][4];
  __shared__ CellPar s_cp[2];
  const int ngroups = P.nv >> 2;
  const int nf = P.nvx + P.nvy;
  const int ncell = P.nx * P.ny;
  float* fac = reinterpret_cast<float*>(smemf4 + 4 * ngroups);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (warp >= NSW) {  // phase 2 of every second cell, buffer m
    const int m = warp - NSW;
    float* px = fac + m * nf;
    float* py = px + P.nvx;
    for (int cell = blockIdx.x + m * gridDim.x; cell < ncell; cell += kPipeMath * gridDim.x) {
      bar_sync_id<NT>(1 + m);
      CellPar cp;
      cell_moments<PREC, NSW>(P, M, cell, 0, s_part[m], cp, msum);
      // the Gaussians in chunks of 32 as the block's NSW warps take them,
      // each chunk's central sums totalled over the warp, chunks in order
      float Mx[5], My[5];
      for (int w = 0; w < NSW && 32 * w < nf; ++w) {
        float ax[5], ay[5];
        cell_gauss<NSW>(P, M, w, cp, px, py, ax, ay);
#pragma unroll
        for (int k = 0; k < 5; ++k) {
          ax[k] = warp_sum_f(ax[k]);
          ay[k] = warp_sum_f(ay[k]);
          Mx[k] = w == 0 ? ax[k] : Mx[k] + ax[k];
          My[k] = w == 0 ? ay[k] : My[k] + ay[k];
        }
      }
      cell_effective(P, cp, Mx, My);
      if (cp.ok) cell_factors<1>(P, M, 0, cp, px, py);
      if (lane == 0) {
        s_cp[m] = cp;
        if (!cp.ok) atomicOr(err, ERR_MOMENT);
      }
      __syncwarp();
      bar_arrive_id<NT>(3 + m);
    }
    return;
  }

  const int tid = threadIdx.x;
  const unsigned step = step_counter<PREC>(M, parity);
  int b = 0;
  size_t prev_c0 = 0;
  bool have_prev = false;
  // coordinates of the cell, advanced by gridDim.x cells per iteration
  const int dix = gridDim.x % P.nx, diy = gridDim.x / P.nx;
  int ix = blockIdx.x % P.nx, iy = blockIdx.x / P.nx;
  for (int cell = blockIdx.x;; cell += gridDim.x) {
    const bool live = cell < ncell;
    if (live) {  // A1 + A2 of this cell into buffer b
      const CellCtx C = cell_ctx<PREC>(P, M, fin, cell, ix, iy);
      float4* flo = smemf4 + (size_t)(2 * b) * ngroups;
      float4* fhi = flo + ngroups;
      float2 s01 = make_float2(0.f, 0.f), s23 = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < MGL; ++k) {
        const int g = tid + NST * k;
        if (g < ngroups) {
          float2 ft[4];
          stream_sum_group<PREC>(P, M, fin, C, 4 * g, ft, s01, s23);
          flo[g] = make_float4(ft[0].x, ft[0].y, ft[1].x, ft[1].y);
          fhi[g] = make_float4(ft[2].x, ft[2].y, ft[3].x, ft[3].y);
        }
      }
      float hs[4] = {s01.x, s01.y, s23.x, s23.y}, ls[4] = {0.f, 0.f, 0.f, 0.f};
      float oh, ol;
      warp_reduce4_ff(hs, ls, oh, ol);
      if ((lane & 7) == 0) s_part[b][warp][lane >> 3] = make_float2(oh, ol);
      bar_arrive_id<NT>(1 + b);
    }
    if (have_prev) {  // A4 of the previous cell from buffer b ^ 1
      const int pb = b ^ 1;
      bar_sync_id<NT>(3 + pb);
      const CellPar cp = s_cp[pb];
      const float* px = fac + pb * nf;
      const float* py = px + P.nvx;
      const float4* flo = smemf4 + (size_t)(2 * pb) * ngroups;
      const float4* fhi = flo + ngroups;
#pragma unroll
      for (int k = 0; k < MGL; ++k) {
        const int g = tid + NST * k;
        if (g < ngroups) {
          float2 r[4];
          unpack_f32(flo[g], fhi[g], r);
          if (cp.ok) relax_group<PREC>(M, px, py, 4 * g, cp.a, cp.kappa, r);
          store_result<PREC>(fout, prev_c0, 4 * g, ngroups, r, step);
        }
      }
    }
    if (!live) break;
    have_prev = true;
    prev_c0 = (size_t)cell * P.nv;
    b ^= 1;
    ix += dix;
    iy += diy;
    if (ix >= P.nx) {
      ix -= P.nx;
      ++iy;
    }
  }
}

// ---- 1D, FP32 state ---------------------------------------------------------
// One warp per cell (8 cells per CTA), no CTA barrier: the warp streams its
// cell's velocities j = lane + 32 k (Eq. exact shift by [C], Eq. upwind on
// the remainder r, f~ = f1 - r (f1 - f2) in flux form), sums the moments in
// float-float, solves the cell's parameters (two linearised FP32
// effective-parameter updates, normalisation n (pi theta)^(-1/2) in
// float-float) and relaxes f^{n+1} = f~ + (a Phi - a f~), with
// G = Phi_g, H = theta G (Chu, 1D).  Ends are inflow Maxwellians.

// a * p0 / sqrt(pi * p3) with float-float intermediates, rounded once.
__device__ __forceinline__ float ff_norm1d(float a, float p0, float p3) {
  const float pi_h = 3.14159274101257324f, pi_l = -8.74227766e-08f;
  const float xh = pi_h * p3;
  const float xl = fmaf(pi_h, p3, -xh) + pi_l * p3;  // pi p3 = xh + xl
  const float sh = sqrtf(xh);
  const float sl = (fmaf(-sh, sh, xh) + xl) * (0.5f * __frcp_rn(sh));  // sqrt(pi p3) = sh + sl
  const float nh = a * p0;
  const float nl = fmaf(a, p0, -nh);
  const float rd = __frcp_rn(sh);
  const float q1 = nh * rd;
  float r = fmaf(-q1, sh, nh);
  r = fmaf(-q1, sl, r) + nl;
  return fmaf(r, rd, q1);
}

template <int KV>
__device__ __forceinline__ void mixed1d_cell(const Params& P, const MixedTables& M, const float2* __restrict__ fin,
                                             float2* __restrict__ fout, float2* __restrict__ msum,
                                             int* __restrict__ err, int cell) {
  const int lane = threadIdx.x & 31;
  const int nv = P.nvx;
  float2 ft[KV];
  float hs[4] = {0.f, 0.f, 0.f, 0.f}, cs[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < KV; ++k) {
    const int j = lane + 32 * k;
    ft[k] = make_float2(0.f, 0.f);
    if (j < nv) {
      const float4 co = M.coef[j];  // (r, 0, c_x, 0)
      const int i1 = cell - M.shift[j];
      const int i2 = i1 - (vi_sx(M.vinfo[j]) > 0 ? 1 : -1);
      const float2 f1 = i1 < 0 ? M.ghost[XLO * nv + j] : i1 >= P.nx ? M.ghost[XHI * nv + j]
                                                                     : fin[(size_t)i1 * nv + j];
      const float2 f2 = i2 < 0 ? M.ghost[XLO * nv + j] : i2 >= P.nx ? M.ghost[XHI * nv + j]
                                                                     : fin[(size_t)i2 * nv + j];
      ft[k].x = fmaf(-co.x, f1.x - f2.x, f1.x);
      ft[k].y = fmaf(-co.x, f1.y - f2.y, f1.y);
      kahan(hs[0], cs[0], ft[k].x);
      kahan(hs[1], cs[1], co.z * ft[k].x);
      kahan(hs[3], cs[3], fmaf(co.z * co.z, ft[k].x, ft[k].y));
    }
  }
  float ls[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) ls[k] = -cs[k];
  float oh, ol;
  warp_reduce4_ff(hs, ls, oh, ol);  // lane 8 m holds value m
  if ((lane & 7) == 0) msum[(size_t)cell * 4 + (lane >> 3)] = make_float2(oh, ol);
  const float sk = oh + ol;
  const float S0 = __shfl_sync(0xffffffffu, sk, 0), S1 = __shfl_sync(0xffffffffu, sk, 8);
  const float S3 = __shfl_sync(0xffffffffu, sk, 24);
  const float r0 = __frcp_rn(S0);
  float n = S0 * (float)P.dv, u = S1 * r0;
  float th = (2.0f / 3.0f) * (S3 * r0 - u * u);
  bool ok = n > 0.f && th > 0.f && isfinite(n) && isfinite(u) && isfinite(th);
  if (!ok) {
    n = 1.f;
    u = 0.f;
    th = 1.f;
  }
  const float nu = n * (P.omega == 0.5 ? sqrtf(th) : powf(th, (float)(1.0 - P.omega)));
  const float a = P.relax_exact ? 1.0f - expf(-nu * (float)P.dt) : nu * (float)P.dt;
  // Gaussian at (u, theta) and its central sums
  const float inv = __frcp_rn(th);
  float e[KV], Mm[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < KV; ++k) {
    const int j = lane + 32 * k;
    e[k] = 0.f;
    if (j < nv) {
      const float d = M.cx[j] - u;
      e[k] = expf(-(d * d) * inv);
      float t = e[k];
#pragma unroll
      for (int m = 0; m < 5; ++m) {
        Mm[m] += t;
        t *= d;
      }
    }
  }
  float p[3] = {n, u, th};
  if (P.conservative) {
#pragma unroll
    for (int m = 0; m < 5; ++m) Mm[m] = warp_sum_f(Mm[m]);
    const float q[3] = {n, u, th};
    for (int it = 0; it < 2; ++it) {
      const float w2 = (p[2] - th) * inv * inv, w1 = 2.f * (p[1] - u) * inv;
      float S[3];
#pragma unroll
      for (int m = 0; m < 3; ++m) S[m] = Mm[m] + w1 * Mm[m + 1] + w2 * Mm[m + 2];
      const float rs = __frcp_rn(S[0]);
      const float mu = S[1] * rs;
      const float d0 = p[0] * __frsqrt_rn(3.14159265f * p[2]) * (float)P.dv * S[0];
      const float d1 = u + mu;
      const float d2 = (2.f / 3.f) * (S[2] * rs - mu * mu + p[2]);
      p[0] += q[0] - d0;
      p[1] += q[1] - d1;
      p[2] += q[2] - d2;
    }
    if (!(p[0] > 0.f) || !(p[2] > 0.f) || !isfinite(p[0]) || !isfinite(p[1]) || !isfinite(p[2])) ok = false;
  }
  if (!ok && lane == 0) atomicOr(err, ERR_MOMENT);
  const float ap = ok ? ff_norm1d(a, p[0], p[2]) : 0.f;
  const float w2 = (p[2] - th) * inv * inv, w1 = 2.f * (p[1] - u) * inv;
  const float kappa = p[2];
#pragma unroll
  for (int k = 0; k < KV; ++k) {
    const int j = lane + 32 * k;
    if (j < nv) {
      float2 r = ft[k];
      if (ok) {
        const float d = M.cx[j] - u;
        const float ph = ap * (e[k] * fmaf(d, fmaf(d, w2, w1), 1.0f));
        r.x += fmaf(-a, ft[k].x, ph);
        r.y += fmaf(-a, ft[k].y, kappa * ph);
      }
      fout[(size_t)cell * nv + j] = r;
    }
  }
}

template <int KV>
__global__ void __launch_bounds__(256) step_mixed1d_kernel(const float2* __restrict__ fin, float2* __restrict__ fout,
                                                           float2* __restrict__ msum, const Params P,
                                                           const MixedTables M, int* __restrict__ err) {
  const int cell = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (cell < P.nx) mixed1d_cell<KV>(P, M, fin, fout, msum, err, cell);
}

// ---- persistent batch ----------------------------------------------------------
// One cooperative launch advances every instance of a batch (FP32, 2D and
// 1D) by nsteps.  Work units are blocks of cells (G cells of a 2D instance,
// 8 cells of a 1D one), numbered instance after instance; CTA b takes the
// units b, b + gridDim.x, ... (so that at any moment the grid works on a
// window of neighbouring units, whose upwind sources are then on chip); the
// instance descriptors sit in constant memory.  Between steps a grid
// barrier: each CTA announces
// its arrival and waits for the generation count to move, for at most
// spin_limit polls, after which it records ERR_TIMEOUT and returns (every
// other CTA then gives up at its own limit), so the launch always ends.

__device__ __forceinline__ void mixed1d_unit(const PInstance& I, const void* fin, void* fout, int blk) {
  const int cell = blk * 8 + (threadIdx.x >> 5);
  if (cell >= I.P.nx) return;
  const float2* fi = static_cast<const float2*>(fin);
  float2* fo = static_cast<float2*>(fout);
  switch (I.kind) {
    case PK_1D_K1: mixed1d_cell<1>(I.P, I.M, fi, fo, I.msum, I.err, cell); break;
    case PK_1D_K2: mixed1d_cell<2>(I.P, I.M, fi, fo, I.msum, I.err, cell); break;
    default: mixed1d_cell<4>(I.P, I.M, fi, fo, I.msum, I.err, cell); break;
  }
}

// One work unit of each kind, inlined (with the descriptor in shared memory,
// measured 5 % faster than calling each kind's code apart; 3 CTAs per SM).
constexpr int kPersistMinBlocks = 3;
template <int G, int MGL>
__device__ __forceinline__ void unit2d(const PInstance& I, const void* fin, void* fout, int blk, float* phx,
                                       char* raw) {
  mixed2d_block<PREC_F32, G, MGL>(I.P, I.M, fin, fout, I.msum, I.err, blk, phx,
                                  *reinterpret_cast<MixedShared<G>*>(raw), 0u);
}
__device__ __forceinline__ void unit1d(const PInstance& I, const void* fin, void* fout, int blk) {
  mixed1d_unit(I, fin, fout, blk);
}

// Returns false when the wait ran out (or another CTA already failed).
__device__ bool grid_barrier(GridBarrier* bar, int* gerr, long long spin_limit) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned int* vgen = &bar->gen;
    const unsigned int g = *vgen;
    __threadfence();
    if (atomicAdd(&bar->count, 1u) + 1u == gridDim.x) {
      bar->count = 0;
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      long long spins = 0;
      while (*vgen == g) {
        if (++spins > spin_limit || *(volatile int*)gerr) {
          atomicOr(gerr, ERR_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(128);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Instance descriptors of the launch, copied in by the graph before the
// kernel (read-only memory: the step's shared-memory stores cannot alias it).
__constant__ PInstance c_pinst[kMaxPersistInstances];

__global__ void __launch_bounds__(256, kPersistMinBlocks)
    batch_persistent_kernel(int ninst, int total_units, int nsteps, GridBarrier* bar, int* gerr,
                            long long spin_limit) {
  extern __shared__ float4 dynf4[];
  float* phx = reinterpret_cast<float*>(dynf4);
  __shared__ __align__(16) char s_raw[sizeof(MixedShared<8>) > sizeof(MixedShared<1>) ? sizeof(MixedShared<8>)
                                                                                       : sizeof(MixedShared<1>)];
  // the descriptor of the instance being worked on, copied from constant
  // memory once per instance and step: the unit code reads its parameters
  // from shared memory instead of through a generic pointer
  __shared__ PInstance s_inst;
  for (int step = 0; step < nsteps; ++step) {
    const bool even = (step & 1) == 0;
    int i = 0, cur = -1;
    for (int u = blockIdx.x; u < total_units; u += gridDim.x) {
      while (c_pinst[i].unit0 + c_pinst[i].units <= u) ++i;  // u grows: scan forward
      if (i != cur) {
        __syncthreads();  // the previous unit has finished reading s_inst
        const unsigned* src = reinterpret_cast<const unsigned*>(&c_pinst[i]);
        unsigned* dst = reinterpret_cast<unsigned*>(&s_inst);
        for (int k = threadIdx.x; k < (int)(sizeof(PInstance) / 4); k += blockDim.x) dst[k] = src[k];
        __syncthreads();
        cur = i;
      }
      const PInstance& I = s_inst;
      const void* fin = even ? I.f_even : I.f_odd;
      void* fout = even ? I.f_odd : const_cast<void*>(I.f_even);
      const int blk = u - I.unit0;
      switch (I.kind) {
        case PK_2D_G1_M2: unit2d<1, 2>(I, fin, fout, blk, phx, s_raw); break;
        case PK_2D_G1_M4: unit2d<1, 4>(I, fin, fout, blk, phx, s_raw); break;
        case PK_2D_G2_M2: unit2d<2, 2>(I, fin, fout, blk, phx, s_raw); break;
        case PK_2D_G2_M4: unit2d<2, 4>(I, fin, fout, blk, phx, s_raw); break;
        case PK_2D_G4_M2: unit2d<4, 2>(I, fin, fout, blk, phx, s_raw); break;
        case PK_2D_G4_M4: unit2d<4, 4>(I, fin, fout, blk, phx, s_raw); break;
        case PK_2D_G8_M2: unit2d<8, 2>(I, fin, fout, blk, phx, s_raw); break;
        default: unit1d(I, fin, fout, blk); break;
      }
    }
    if (!grid_barrier(bar, gerr, spin_limit)) return;
  }
}

cudaError_t upload_persistent(const PInstance* d_inst, int ninst, cudaStream_t stream) {
  if (ninst > kMaxPersistInstances) return cudaErrorInvalidValue;
  return cudaMemcpyToSymbolAsync(c_pinst, d_inst, sizeof(PInstance) * (size_t)ninst, 0, cudaMemcpyDeviceToDevice,
                                 stream);
}

int persistent_kind(const Params& P) {
  if (P.dim == 1) {
    if (P.nvx > 128) return -1;
    return P.nvx <= 32 ? PK_1D_K1 : P.nvx <= 64 ? PK_1D_K2 : PK_1D_K4;
  }
  // the persistent kernel carries kinds of 2 and 4 groups per lane
  const int m = mixed_groups_per_lane(P, P.tile);
  const bool m4 = m == 3 || m == 4;
  switch (P.tile) {
    case 1: return m == 2 ? PK_2D_G1_M2 : m4 ? PK_2D_G1_M4 : -1;
    case 2: return m == 2 ? PK_2D_G2_M2 : m4 ? PK_2D_G2_M4 : -1;
    case 4: return m == 2 ? PK_2D_G4_M2 : m4 ? PK_2D_G4_M4 : -1;
    case 8: return m == 2 ? PK_2D_G8_M2 : -1;
  }
  return -1;
}

int persistent_units(const Params& P, int kind) {
  if (kind >= PK_1D_K1) return (P.nx + 7) / 8;
  return (P.nx * P.ny + P.tile - 1) / P.tile;
}

size_t persistent_smem(const Params& P) { return P.dim == 1 ? 0 : mixed_factor_bytes(P, P.tile); }

cudaError_t persistent_grid(size_t smem, int* grid) {
  int dev = 0, per_sm = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_persistent_kernel, 256, smem);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  *grid = per_sm * sms;
  return e;
}

cudaError_t launch_persistent(int ninst, int total_units, int nsteps, GridBarrier* bar, int* gerr,
                              long long spin_limit, int grid, size_t smem, cudaStream_t stream) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // all CTAs resident: the grid barrier needs it
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, batch_persistent_kernel, ninst, total_units, nsteps, bar, gerr, spin_limit);
}

// FP64 moments (n, ux, uy, theta) from the float-float velocity sums a step
// published (bgk_moments, which = 1, reduced precisions).
__global__ void msum_moments_kernel(const Params P, const MixedTables M, int prec, const float2* msum,
                                    double4_32a* mom) {
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= P.nx * P.ny) return;
  double s[4];
  for (int k = 0; k < 4; ++k) {
    const float2 v = msum[(size_t)cell * 4 + k];
    s[k] = (double)v.x + (double)v.y + (prec == PREC_BF16 ? M.mabs_sums[k] : 0.0);
  }
  double q[4];
  moments_from_sums(s[0], s[1], s[2], s[3], P.dv, q);
  mom[cell] = make_double4_32a(q[0], q[1], q[2], q[3]);
}

cudaError_t launch_msum_moments(const Params& P, int prec, const MixedTables& M, const float2* msum,
                                double4_32a* mom, cudaStream_t stream) {
  const int ncell = P.nx * P.ny;
  msum_moments_kernel<<<(ncell + 255) / 256, 256, 0, stream>>>(P, M, prec, msum, mom);
  return cudaGetLastError();
}

// ---- tables -------------------------------------------------------------------
// FP32 copies of the per-velocity tables, the FP32 absolute Maxwellian and
// the FP64 sums that pin the mixed form's moments and wall fluxes to the
// values actually stored.
__global__ void mixed_tables_kernel(const Params P, const Tables T, float4* coef, float* cx, float* cy,
                                    float* ax, float* ay, float2* ghost, float2* mabs) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= P.nv) return;
  const int jx = j % P.nvx, jy = j / P.nvx;
  const double4_32a c = T.coef[j];
  const double2 v = T.cxy[j];
  coef[j] = make_float4((float)c.y, (float)c.z, (float)v.x, (float)v.y);
  if (jy == 0) cx[jx] = (float)v.x;
  if (jx == 0) cy[jy] = (float)v.y;
  if (jy == 0) ax[jx] = (float)c.y;  // 2D: |c_x| dt / dx depends on jx alone
  if (jx == 0) ay[jy] = (float)c.z;  //     |c_y| dt / dy on jy alone
  for (int face = 0; face < kFaces; ++face) {
    const double2 g = T.ghost[face * P.nv + j];
    ghost[face * P.nv + j] = make_float2((float)g.x, (float)g.y);
  }
  const double unit[4] = {1.0, 0.0, 0.0, 1.0};
  const double2 m = maxwell_point(P.dim, unit, v.x, v.y);
  mabs[j] = make_float2((float)m.x, (float)m.y);
}

__global__ void __launch_bounds__(256) mixed_sums_kernel(const Params P, const MixedTables M,
                                                         double* mabs_sums, float2* mabs_ff, double* emitted) {
  __shared__ double red[4 * 8];
  __shared__ double tot[4];
  double s[4] = {0.0, 0.0, 0.0, 0.0}, e[4] = {0.0, 0.0, 0.0, 0.0};
  for (int j = threadIdx.x; j < P.nv; j += 256) {
    const float4 co = M.coef[j];
    const double cx = co.z, cy = co.w;
    const double c2 = (double)fmaf(co.z, co.z, co.w * co.w);
    const float2 m = M.mabs[j];
    s[0] += m.x;
    s[1] = fma(cx, (double)m.x, s[1]);
    s[2] = fma(cy, (double)m.x, s[2]);
    s[3] = fma(c2, (double)m.x, s[3]) + (double)m.y;
    const double cn[4] = {cx, -cx, cy, -cy};
    for (int f = 0; f < 4; ++f)
      if (P.bc_kind[f] == BC_DIFFUSE && cn[f] > 0.0) e[f] = fma(cn[f], (double)M.ghost[f * P.nv + j].x, e[f]);
  }
  block_reduce4<256>(s[0], s[1], s[2], s[3], red, tot);
  if (threadIdx.x < 4) {
    const double v = tot[threadIdx.x];
    mabs_sums[threadIdx.x] = v;
    const float hi = (float)v;
    mabs_ff[threadIdx.x] = make_float2(hi, (float)(v - (double)hi));
  }
  block_reduce4<256>(e[0], e[1], e[2], e[3], red, tot);
  if (threadIdx.x < 4) emitted[threadIdx.x] = tot[threadIdx.x] * P.dv;
}

cudaError_t launch_build_mixed_tables(const Params& P, const Tables& T, const MixedTables& M,
                                      cudaStream_t stream) {
  mixed_tables_kernel<<<(P.nv + 255) / 256, 256, 0, stream>>>(
      P, T, const_cast<float4*>(M.coef), const_cast<float*>(M.cx), const_cast<float*>(M.cy),
      const_cast<float*>(M.ax), const_cast<float*>(M.ay), const_cast<float2*>(M.ghost),
      const_cast<float2*>(M.mabs));
  mixed_sums_kernel<<<1, 256, 0, stream>>>(P, M, const_cast<double*>(M.mabs_sums),
                                           const_cast<float2*>(M.mabs_ff), const_cast<double*>(M.emitted));
  return cudaGetLastError();
}

// ---- conversions between the FP64 layout of the ABI and the storage ------------
template <int PREC>
__global__ void to_f64_kernel(const Params P, const MixedTables M, const void* f, double2* out) {
  const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  const size_t total = (size_t)P.nx * P.ny * P.nv;
  if (idx >= total) return;
  const size_t c0 = idx - idx % P.nv;
  const int j = (int)(idx % P.nv);
  const float2 v = (PREC == PREC_F32 && P.dim == 1) ? static_cast<const float2*>(f)[idx]
                                                    : Store<PREC>::load1(f, c0, j, P.nv >> 2);
  double2 r = make_double2((double)v.x, (double)v.y);
  if (Store<PREC>::delta) {
    const float2 m = M.mabs[idx % P.nv];
    r.x += (double)m.x;
    r.y += (double)m.y;
  }
  out[idx] = r;
}

template <int PREC>
__global__ void from_f64_kernel(const Params P, const MixedTables M, const double2* in, void* f) {
  const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  const size_t total = (size_t)P.nx * P.ny * P.nv;
  if (idx >= total) return;
  double2 v = in[idx];
  if (PREC == PREC_F32) {
    const size_t at = P.dim == 1 ? idx : idx - idx % P.nv + f32_pos((int)(idx % P.nv), P.nv >> 2);
    static_cast<float2*>(f)[at] = make_float2((float)v.x, (float)v.y);
  } else {
    const float2 m = M.mabs[idx % P.nv];
    v.x -= (double)m.x;
    v.y -= (double)m.y;
    static_cast<unsigned*>(f)[idx] = Store<PREC_BF16>::pack(make_float2((float)v.x, (float)v.y));
  }
}

cudaError_t launch_to_f64(const Params& P, int prec, const MixedTables& M, const void* f, double2* out,
                          cudaStream_t stream) {
  const size_t total = (size_t)P.nx * P.ny * P.nv;
  const unsigned grid = (unsigned)((total + 255) / 256);
  if (prec == PREC_F32) to_f64_kernel<PREC_F32><<<grid, 256, 0, stream>>>(P, M, f, out);
  else to_f64_kernel<PREC_BF16><<<grid, 256, 0, stream>>>(P, M, f, out);
  return cudaGetLastError();
}

cudaError_t launch_from_f64(const Params& P, int prec, const MixedTables& M, const double2* in, void* f,
                            cudaStream_t stream) {
  const size_t total = (size_t)P.nx * P.ny * P.nv;
  const unsigned grid = (unsigned)((total + 255) / 256);
  if (prec == PREC_F32) from_f64_kernel<PREC_F32><<<grid, 256, 0, stream>>>(P, M, in, f);
  else from_f64_kernel<PREC_BF16><<<grid, 256, 0, stream>>>(P, M, in, f);
  return cudaGetLastError();
}

// ---- launch ------------------------------------------------------------------
namespace {

// The Gaussian factors of G cells.
size_t mixed_smem(const Params& P, int G, int) { return mixed_factor_bytes(P, G); }

template <int PREC, int G, int MGL>
cudaError_t launch_mg(const Params& P, const MixedTables& M, const void* fin, void* fout, float2* msum,
                      int* err, cudaStream_t stream, int parity) {
  const int ncell = P.nx * P.ny;
  const unsigned grid = (unsigned)((ncell + G - 1) / G);
  const size_t smem = mixed_smem(P, G, PREC);
  step_mixed_kernel<PREC, G, MGL><<<grid, 256, smem, stream>>>(fin, fout, msum, P, M, err, parity);
  return cudaGetLastError();
}

template <int PREC, int G>
cudaError_t dispatch_mgl(const Params& P, const MixedTables& M, const void* fin, void* fout, float2* msum,
                         int* err, cudaStream_t stream, int parity) {
  switch (P.mgl) {
    case 2: return launch_mg<PREC, G, 2>(P, M, fin, fout, msum, err, stream, parity);
    case 3: return launch_mg<PREC, G, 3>(P, M, fin, fout, msum, err, stream, parity);
    case 4: return launch_mg<PREC, G, 4>(P, M, fin, fout, msum, err, stream, parity);
    case 5: return launch_mg<PREC, G, 5>(P, M, fin, fout, msum, err, stream, parity);
    case 6: return launch_mg<PREC, G, 6>(P, M, fin, fout, msum, err, stream, parity);
  }
  return cudaErrorInvalidValue;
}

// Groups of 4 velocities per streaming thread of the pipelined kernel with
// nsw streaming warps (a cell has at most 4096 velocities); 0 if more than 4.
int pipe_groups(const Params& P, int nsw) {
  const int need = (P.nv / 4 + 32 * nsw - 1) / (32 * nsw);
  return need <= 4 ? need : 0;
}

template <int PREC, int MGL, int NSW>
cudaError_t launch_pipe(const Params& P, const MixedTables& M, const void* fin, void* fout, float2* msum,
                        int* err, cudaStream_t stream, int parity) {
  const size_t smem = pipe_smem_bytes(P);
  int dev = 0, per_sm = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(step_mixed_pipe_kernel<PREC, MGL, NSW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kPipeMaxSmem);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_mixed_pipe_kernel<PREC, MGL, NSW>,
                                                      pipe_threads<NSW>(), smem);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int ncell = P.nx * P.ny;
  const int grid = per_sm * sms < ncell ? per_sm * sms : ncell;
  step_mixed_pipe_kernel<PREC, MGL, NSW><<<grid, pipe_threads<NSW>(), smem, stream>>>(fin, fout, msum, P, M, err,
                                                                                       parity);
  return cudaGetLastError();
}

// Tile 1: the pipelined kernel when its buffers fit, else the one-cell block
// (the same arithmetic).
template <int PREC>
cudaError_t dispatch_tile1(const Params& P, const MixedTables& M, const void* fin, void* fout, float2* msum,
                           int* err, cudaStream_t stream, int parity) {
  if (pipe_smem_bytes(P) <= kPipeMaxSmem) switch (pipe_groups(P, 8)) {
      case 1: return launch_pipe<PREC, 1, 8>(P, M, fin, fout, msum, err, stream, parity);
      case 2: return launch_pipe<PREC, 2, 8>(P, M, fin, fout, msum, err, stream, parity);
      case 3: return launch_pipe<PREC, 3, 8>(P, M, fin, fout, msum, err, stream, parity);
      case 4: return launch_pipe<PREC, 4, 8>(P, M, fin, fout, msum, err, stream, parity);
    }
  return dispatch_mgl<PREC, 1>(P, M, fin, fout, msum, err, stream, parity);
}

template <int PREC>
cudaError_t dispatch_m(const Params& P, const MixedTables& M, const void* fin, void* fout, float2* msum,
                       int* err, cudaStream_t stream, int parity) {
  switch (P.tile) {
    case 1: return dispatch_tile1<PREC>(P, M, fin, fout, msum, err, stream, parity);
    case 2: return dispatch_mgl<PREC, 2>(P, M, fin, fout, msum, err, stream, parity);
    case 4: return dispatch_mgl<PREC, 4>(P, M, fin, fout, msum, err, stream, parity);
    case 8: return dispatch_mgl<PREC, 8>(P, M, fin, fout, msum, err, stream, parity);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

bool mixed_pipe_preferred(const Params& P) {
  return P.dim == 2 && pipe_smem_bytes(P) <= kPipeMaxSmem && pipe_groups(P, 8) >= 3;
}

size_t step_mixed_smem_bytes(const Params& P, int tile, int prec) { return mixed_smem(P, tile, prec); }

// Groups of 4 velocities per lane when a cell has 256/tile lanes (at least
// 2); 0 if more than 6 would be needed.  Every count from 2 to 6 is
// instantiated: the f~ a lane keeps in registers is sized by it, and one
// group too many cost registers (BF16 at 4.5 groups per lane: 64 bytes of
// spills and 0.798 ms per 256^2 x 48^2 step at 6, 16 bytes and 0.771 ms at
// 5).  The count does not change the arithmetic (a lane's groups and their
// order are the same), only which registers hold them.
int mixed_groups_per_lane(const Params& P, int tile) {
  const int lanes = 256 / tile;
  const int need = (P.nv / 4 + lanes - 1) / lanes;
  if (need <= 2) return 2;
  if (need <= 6) return need;
  return 0;
}

// The pipelined kernels raise their dynamic shared-memory limit at launch.
cudaError_t prepare_step_mixed(const Params&, int) { return cudaSuccess; }

cudaError_t launch_step_mixed(const Params& P, int prec, const MixedTables& M, const void* fin, void* fout,
                              double4_32a* mom, int* err, cudaStream_t stream, int parity) {
  float2* msum = reinterpret_cast<float2*>(mom);  // 32 bytes per cell either way
  if (P.dim == 1) {
    const unsigned grid = (unsigned)((P.nx + 7) / 8);
    const float2* fi = static_cast<const float2*>(fin);
    float2* fo = static_cast<float2*>(fout);
    if (P.nvx <= 32) step_mixed1d_kernel<1><<<grid, 256, 0, stream>>>(fi, fo, msum, P, M, err);
    else if (P.nvx <= 64) step_mixed1d_kernel<2><<<grid, 256, 0, stream>>>(fi, fo, msum, P, M, err);
    else step_mixed1d_kernel<4><<<grid, 256, 0, stream>>>(fi, fo, msum, P, M, err);
    return cudaGetLastError();
  }
  return prec == PREC_F32 ? dispatch_m<PREC_F32>(P, M, fin, fout, msum, err, stream, parity)
                          : dispatch_m<PREC_BF16>(P, M, fin, fout, msum, err, stream, parity);
}

}  // namespace bgk
