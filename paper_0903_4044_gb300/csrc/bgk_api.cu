// bgk_api.cu - host runtime and C ABI of libbgk.so (declared in bgk.h).
//
// A solver holds two device state buffers (ping-pong), per-cell moment
// storage, the per-velocity tables and a device error flag.  bgk_step
// enqueues one fused kernel per time step; runs of kChunk steps replay a
// CUDA graph captured once per starting buffer.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "bgk.h"
#include "bgk_internal.h"

namespace {

thread_local std::string g_last_error;

bgk_status fail(bgk_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

bgk_status cuda_fail(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation)
    return fail(BGK_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  return fail(BGK_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

constexpr int kChunk = 64;  // steps per captured graph (even: ends on the same buffer)
constexpr size_t kMaxSmem = 224 * 1024;   // dynamic shared memory one CTA may use (227 KB minus static, at most 3 KB)
constexpr size_t kAutoSmem = 113 * 1024;  // automatic tiles leave room for two CTAs per SM

}  // namespace

struct bgk_solver {
  bgk_config cfg;
  bgk::Params P;
  int device = 0;
  cudaStream_t stream = nullptr;      // caller's stream (may be the legacy default)
  cudaStream_t cap_stream = nullptr;  // private stream used only for graph capture
  int prec = bgk::PREC_F64;
  void* f[2] = {nullptr, nullptr};  // state ping-pong, storage type by precision
  int cur = 0;
  double2* stage = nullptr;  // FP64 view of the state (reduced precisions only)
  double4_32a* mom_step = nullptr;  // moments of the last post-streaming state
  double4_32a* mom_tmp = nullptr;   // scratch for bgk_moments(which = 0)
  double4_32a* flux_tmp = nullptr;  // scratch for bgk_wall_fluxes
  double* cx = nullptr;
  double* cy = nullptr;  // [2 nvy]: centres, then their squares
  double4_32a* coef = nullptr;
  int* shift = nullptr;
  double2* cxy = nullptr;
  int* vinfo = nullptr;
  double2* ghost = nullptr;
  double* emitted = nullptr;
  // FP32 tables of the reduced-precision step
  float4* m_coef = nullptr;
  float* m_cx = nullptr;
  float* m_cy = nullptr;
  float* m_ax = nullptr;
  float* m_ay = nullptr;
  float2* m_ghost = nullptr;
  float2* m_mabs = nullptr;
  double* m_sums = nullptr;  // [12]: mabs sums, emitted, mabs sums as float-float pairs
  unsigned* m_ctr = nullptr;  // [2] step counter of the BF16 dither (see MixedTables::step_ctr)
  int* err = nullptr;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int64_t gen = 0;  // bumped whenever captured launches become stale (tile change)
  int64_t steps_done = 0;
  int64_t device_bytes = 0;
  double max_courant = 0.0;

  bgk::Tables tables() const {
    bgk::Tables T;
    T.cx = cx;
    T.cy = cy;
    T.cy2 = cy + P.nvy;
    T.coef = coef;
    T.shift = shift;
    T.cxy = cxy;
    T.vinfo = vinfo;
    T.ghost = ghost;
    T.emitted = emitted;
    return T;
  }
  bgk::MixedTables mtables() const {
    bgk::MixedTables M;
    M.coef = m_coef;
    M.vinfo = vinfo;
    M.cx = m_cx;
    M.cy = m_cy;
    M.ax = m_ax;
    M.ay = m_ay;
    M.ghost = m_ghost;
    M.mabs = m_mabs;
    M.mabs_sums = m_sums;
    M.emitted = m_sums + 4;
    M.mabs_ff = reinterpret_cast<const float2*>(m_sums + 8);
    M.shift = shift;
    M.step_ctr = m_ctr;
    return M;
  }
  size_t state_elems() const { return (size_t)P.nx * P.ny * P.nv; }  // (g,h) pairs
  size_t point_bytes() const { return prec == bgk::PREC_F64 ? 16 : prec == bgk::PREC_F32 ? 8 : 4; }
  // FP64 (g, h) view of the current state: the state itself in FP64, else
  // converted into the staging buffer
  cudaError_t f64_view(const double2** out) {
    if (prec == bgk::PREC_F64) {
      *out = (const double2*)f[cur];
      return cudaSuccess;
    }
    *out = stage;
    return bgk::launch_to_f64(P, prec, mtables(), f[cur], stage, stream);
  }
};

namespace {

bool finite_all(std::initializer_list<double> v) {
  for (double x : v)
    if (!std::isfinite(x)) return false;
  return true;
}

double max_abs_centre(double vmin, double vmax, int n) {
  const double dc = (vmax - vmin) / n;
  double m = 0.0;
  for (int j = 0; j < n; ++j) m = std::fmax(m, std::fabs(vmin + (j + 0.5) * dc));
  return m;
}

size_t step_smem(const bgk::Params& P, int prec, int tile) {
  return prec == BGK_F64 ? bgk::step_f64_smem_bytes(P, tile) : bgk::step_mixed_smem_bytes(P, tile, prec == BGK_BF16_DEV ? bgk::PREC_BF16 : bgk::PREC_F32);
}

// All configuration checks, before any CUDA call.  Fills P and max_courant.
bgk_status validate(const bgk_config* c, bgk::Params* P, double* max_courant) {
  if (c->dim != 1 && c->dim != 2) return fail(BGK_ERR_INVALID_ARG, "dim must be 1 or 2 (got %d)", c->dim);
  if (c->nx < 1) return fail(BGK_ERR_INVALID_ARG, "nx must be >= 1 (got %d)", c->nx);
  if (c->dim == 1 && c->ny != 1) return fail(BGK_ERR_INVALID_ARG, "ny must be 1 when dim = 1 (got %d)", c->ny);
  if (c->dim == 2 && c->ny < 1) return fail(BGK_ERR_INVALID_ARG, "ny must be >= 1 (got %d)", c->ny);
  if (c->nvx < 2) return fail(BGK_ERR_INVALID_ARG, "nvx must be >= 2 (got %d)", c->nvx);
  if (c->dim == 1 && c->nvy != 1) return fail(BGK_ERR_INVALID_ARG, "nvy must be 1 when dim = 1 (got %d)", c->nvy);
  if (c->dim == 2 && c->nvy < 2) return fail(BGK_ERR_INVALID_ARG, "nvy must be >= 2 (got %d)", c->nvy);
  const int64_t nv = (int64_t)c->nvx * c->nvy;
  if (nv > bgk::kMaxNv)
    return fail(BGK_ERR_UNSUPPORTED, "nvx*nvy = %lld exceeds the %d velocities one CTA handles",
                (long long)nv, bgk::kMaxNv);
  if ((int64_t)c->nx * c->ny > (int64_t)0x7fffffff)
    return fail(BGK_ERR_UNSUPPORTED, "more than 2^31-1 spatial cells");
  if (!finite_all({c->x0, c->lx, c->vx_min, c->vx_max, c->omega, c->dt, c->cfl}))
    return fail(BGK_ERR_INVALID_ARG, "non-finite configuration value");
  if (!(c->lx > 0.0)) return fail(BGK_ERR_INVALID_ARG, "lx must be > 0");
  if (!(c->vx_max > c->vx_min)) return fail(BGK_ERR_INVALID_ARG, "vx_max must exceed vx_min");
  if (c->dim == 2) {
    if (!finite_all({c->y0, c->ly, c->vy_min, c->vy_max}))
      return fail(BGK_ERR_INVALID_ARG, "non-finite configuration value");
    if (!(c->ly > 0.0)) return fail(BGK_ERR_INVALID_ARG, "ly must be > 0");
    if (!(c->vy_max > c->vy_min)) return fail(BGK_ERR_INVALID_ARG, "vy_max must exceed vy_min");
  }
  if (c->dt < 0.0) return fail(BGK_ERR_INVALID_ARG, "dt must be >= 0");
  if (c->dt == 0.0 && !(c->cfl > 0.0)) return fail(BGK_ERR_INVALID_ARG, "dt = 0 needs cfl > 0");
  if (c->conservative != 0 && c->conservative != 1) return fail(BGK_ERR_INVALID_ARG, "conservative must be 0 or 1");
  if (c->relax_exact != 0 && c->relax_exact != 1) return fail(BGK_ERR_INVALID_ARG, "relax_exact must be 0 or 1");
  if (c->reserved0 != 0) return fail(BGK_ERR_INVALID_ARG, "reserved0 must be 0");
  if (c->tile_cells != 0 && c->tile_cells != 1 && c->tile_cells != 2 && c->tile_cells != 4 &&
      c->tile_cells != 8)
    return fail(BGK_ERR_INVALID_ARG, "tile_cells must be 0, 1, 2, 4 or 8 (got %d)", c->tile_cells);
  if (c->precision != BGK_F64 && c->precision != BGK_F32 && c->precision != BGK_BF16_DEV)
    return fail(BGK_ERR_INVALID_ARG, "unknown precision %d", c->precision);
  if (c->precision != BGK_F64 && c->dim == 1) {
    // 1D reduced precision: FP32 state, one warp per cell, inflow ends
    if (c->precision != BGK_F32) return fail(BGK_ERR_UNSUPPORTED, "dim 1 reduced precision is FP32 only");
    if (c->nvx > 128) return fail(BGK_ERR_UNSUPPORTED, "dim 1 FP32 needs nvx <= 128 (got %d)", c->nvx);
    if (c->bc[0].kind != BGK_BC_INFLOW || c->bc[1].kind != BGK_BC_INFLOW)
      return fail(BGK_ERR_UNSUPPORTED, "dim 1 FP32 needs inflow boundaries");
  } else if (c->precision != BGK_F64) {
    // the reduced-precision kernel streams 4 consecutive velocities of one
    // row per lane: rows of a multiple of 8 with c_x changing sign only on
    // multiples of 4
    if (c->nvx % 8 != 0)
      return fail(BGK_ERR_UNSUPPORTED, "reduced precision needs nvx a multiple of 8 (got %d)", c->nvx);
    const double dc = (c->vx_max - c->vx_min) / c->nvx;
    for (int j = 0; j < c->nvx; ++j) {
      const double a = c->vx_min + (j + 0.5) * dc, b0 = c->vx_min + ((j & ~3) + 0.5) * dc;
      if ((a > 0.0) != (b0 > 0.0) || (a < 0.0) != (b0 < 0.0))
        return fail(BGK_ERR_UNSUPPORTED,
                    "reduced precision needs c_x to change sign on a multiple of 4 velocities");
    }
  }

  bgk::Params& p = *P;
  std::memset(&p, 0, sizeof(p));
  p.dim = c->dim;
  p.nx = c->nx;
  p.ny = c->dim == 2 ? c->ny : 1;
  p.nvx = c->nvx;
  p.nvy = c->dim == 2 ? c->nvy : 1;
  p.nv = (int)nv;
  p.conservative = c->conservative;
  p.relax_exact = c->relax_exact;
  p.dx = c->lx / c->nx;
  p.dy = c->dim == 2 ? c->ly / c->ny : 1.0;
  p.dcx = (c->vx_max - c->vx_min) / c->nvx;
  p.dcy = c->dim == 2 ? (c->vy_max - c->vy_min) / c->nvy : 1.0;
  p.dv = c->dim == 2 ? p.dcx * p.dcy : p.dcx;
  p.x0 = c->x0;
  p.vx_min = c->vx_min;
  p.vy_min = c->dim == 2 ? c->vy_min : 0.0;
  p.omega = c->omega;
  const double mx = max_abs_centre(c->vx_min, c->vx_max, c->nvx);
  const double my = c->dim == 2 ? max_abs_centre(c->vy_min, c->vy_max, c->nvy) : 0.0;
  if (c->dt > 0.0) {
    p.dt = c->dt;
  } else if (c->dim == 1) {
    p.dt = c->cfl * p.dx / mx;
  } else {
    p.dt = c->cfl / (mx / p.dx + my / p.dy);
  }
  *max_courant = c->dim == 1 ? mx * p.dt / p.dx : mx * p.dt / p.dx + my * p.dt / p.dy;

  // cells per CTA: the caller's choice (checked here), else chosen in
  // bgk_create once the device's SM count is known
  p.tile = c->tile_cells;
  if (c->tile_cells && c->precision != BGK_F64 && bgk::mixed_groups_per_lane(p, p.tile) == 0)
    return fail(BGK_ERR_UNSUPPORTED, "tile_cells = %d leaves more than 24 velocities per lane", p.tile);
  if (c->tile_cells && c->precision != BGK_F64) p.mgl = bgk::mixed_groups_per_lane(p, p.tile);
  if (c->tile_cells && step_smem(p, c->precision, p.tile) > kMaxSmem)
    return fail(BGK_ERR_UNSUPPORTED, "tile_cells = %d needs %zu bytes of shared memory (max %zu)",
                p.tile, step_smem(p, c->precision, p.tile), kMaxSmem);
  if (!c->tile_cells && step_smem(p, c->precision, 1) > kMaxSmem)
    return fail(BGK_ERR_UNSUPPORTED, "one cell's state needs %zu bytes of shared memory (max %zu)",
                step_smem(p, c->precision, 1), kMaxSmem);

  const int nfaces = c->dim == 2 ? 4 : 2;
  bool walls = false;
  for (int face = 0; face < bgk::kFaces; ++face) {
    const bgk_bc& b = c->bc[face];
    p.bc_kind[face] = b.kind;
    p.bc_state[face][0] = b.n;
    p.bc_state[face][1] = b.ux;
    p.bc_state[face][2] = b.uy;
    p.bc_state[face][3] = b.theta;
    if (face >= nfaces) continue;
    const bool xface = face < 2;
    if (!finite_all({b.n, b.ux, b.uy, b.theta}))
      return fail(BGK_ERR_INVALID_ARG, "face %d: non-finite boundary state", face);
    if (c->dim == 1 && b.uy != 0.0)
      return fail(BGK_ERR_INVALID_ARG, "face %d: uy must be 0 in 1D", face);
    switch (b.kind) {
      case BGK_BC_INFLOW:
        if (!(b.n > 0.0) || !(b.theta > 0.0))
          return fail(BGK_ERR_INVALID_ARG, "face %d: inflow needs n > 0 and theta > 0", face);
        break;
      case BGK_BC_DIFFUSE:
        walls = true;
        if (!(b.theta > 0.0)) return fail(BGK_ERR_INVALID_ARG, "face %d: wall theta must be > 0", face);
        if ((xface && b.ux != 0.0) || (!xface && b.uy != 0.0))
          return fail(BGK_ERR_INVALID_ARG, "face %d: wall velocity must be tangential", face);
        break;
      case BGK_BC_SPECULAR: {
        walls = true;
        const double lo = xface ? c->vx_min : c->vy_min, hi = xface ? c->vx_max : c->vy_max;
        if (std::fabs(lo + hi) > 1e-12 * std::fabs(hi))
          return fail(BGK_ERR_INVALID_ARG,
                      "face %d: specular walls need a velocity grid symmetric about 0", face);
        break;
      }
      default:
        return fail(BGK_ERR_INVALID_ARG, "face %d: unknown boundary kind %d", face, b.kind);
    }
  }
  if (c->dim == 2 && *max_courant > 1.0 + 1e-12)
    return fail(BGK_ERR_UNSUPPORTED, "2D donor cell needs (max|cx|/dx + max|cy|/dy) dt <= 1 (got %.6g)",
                *max_courant);
  if (walls && *max_courant > 1.0 + 1e-12)
    return fail(BGK_ERR_UNSUPPORTED, "walls need a Courant number <= 1 (got %.6g)", *max_courant);
  return BGK_OK;
}

// Largest tile (cells per CTA) that keeps two CTAs' shared memory within an
// SM and still gives every SM at least two CTAs.  FP64 takes 8 cells per CTA
// (4 CTAs per SM) only in 2D with at least three full waves of them: the
// per-cell solve then serves 8 cells per warp instruction (measured 2.6 %
// faster on 256^2 x 48^2, and 2.8 % on the gradient of the 128^2 x 32^2
// cavity); on fewer cells the last wave leaves SMs idle (7 % slower on
// 64^2 x 32^2), and 4 cells per CTA are kept.
int auto_tile(const bgk::Params& P, int prec, int sms) {
  const long long ncell = (long long)P.nx * P.ny;
  if (prec == BGK_F64 && P.dim == 2 && ncell >= 8LL * 4 * 3 * sms && step_smem(P, prec, 8) <= kAutoSmem) return 8;
  // FP32, 2D, at least 3 groups of 4 velocities per streaming thread: the
  // pipelined one-cell kernel (measured 9 % faster than 2 cells per CTA on
  // 256^2 x 48^2; slower on 64^2 x 32^2 and in BF16)
  if (prec == BGK_F32 && P.dim == 2 && bgk::mixed_pipe_preferred(P) && ncell >= 2LL * sms) return 1;
  for (int t : {8, 4, 2}) {
    if (prec == BGK_F64 && t > 4) continue;
    // reduced precisions: at most 24 velocities per lane (instantiated)
    if (prec != BGK_F64 && bgk::mixed_groups_per_lane(P, t) == 0) continue;
    if (step_smem(P, prec, t) <= kAutoSmem && (ncell + t - 1) / t >= 2LL * sms) return t;
  }
  return 1;
}

template <typename T>
cudaError_t dev_alloc(bgk_solver* s, T** p, size_t count) {
  const size_t bytes = sizeof(T) * (count ? count : 1);
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e == cudaSuccess) s->device_bytes += (int64_t)bytes;
  return e;
}

void release(bgk_solver* s) {
  if (!s) return;
  for (auto& g : s->graph)
    if (g) cudaGraphExecDestroy(g);
  void* bufs[] = {s->f[0], s->f[1], s->stage, s->mom_step, s->mom_tmp, s->flux_tmp, s->cx, s->cy,
                  s->coef, s->shift, s->cxy, s->vinfo, s->ghost, s->emitted, s->m_coef, s->m_cx,
                  s->m_cy, s->m_ax, s->m_ay, s->m_ghost, s->m_mabs, s->m_sums, s->m_ctr, s->err};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
  delete s;
}

cudaError_t enqueue_step(bgk_solver* s, int from, cudaStream_t st) {
  if (s->prec == bgk::PREC_F64)
    return bgk::launch_step_f64(s->P, s->tables(), (const double2*)s->f[from], (double2*)s->f[1 - from],
                                s->mom_step, s->err, st);
  return bgk::launch_step_mixed(s->P, s->prec, s->mtables(), s->f[from], s->f[1 - from], s->mom_step,
                                s->err, st, from);
}

// Write an FP64 state (device pointer, ABI layout) into the current buffer.
cudaError_t store_f64(bgk_solver* s, const double2* src) {
  if (s->prec == bgk::PREC_F64)
    return cudaMemcpyAsync(s->f[s->cur], src, sizeof(double2) * s->state_elems(), cudaMemcpyDeviceToDevice,
                           s->stream);
  return bgk::launch_from_f64(s->P, s->prec, s->mtables(), src, s->f[s->cur], s->stream);
}

bgk_status ensure_graph(bgk_solver* s, int start) {
  if (s->graph[start]) return BGK_OK;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(e, "graph capture begin");
  int b = start;
  cudaError_t le = cudaSuccess;
  for (int i = 0; i < kChunk && le == cudaSuccess; ++i) {
    le = enqueue_step(s, b, s->cap_stream);
    b ^= 1;
  }
  e = cudaStreamEndCapture(s->cap_stream, &g);
  if (le != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(le, "step launch during capture");
  }
  if (e != cudaSuccess) return cuda_fail(e, "graph capture end");
  e = cudaGraphInstantiate(&s->graph[start], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    s->graph[start] = nullptr;
    return cuda_fail(e, "graph instantiate");
  }
  return BGK_OK;
}

bgk_status check_flag(bgk_solver* s) {
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, s->err, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
  if (h & bgk::ERR_MOMENT)
    return fail(BGK_ERR_NUMERIC, "a cell reached n <= 0, theta <= 0 or a non-finite moment");
  if (h & bgk::ERR_EFFECTIVE)
    return fail(BGK_ERR_NUMERIC, "the effective-parameter iteration did not converge in a cell");
  return BGK_OK;
}

#define BGK_GUARD_BEGIN try {
#define BGK_GUARD_END                                                     \
  }                                                                       \
  catch (const std::bad_alloc&) {                                         \
    return fail(BGK_ERR_OOM, "host allocation failed");                   \
  }                                                                       \
  catch (...) {                                                           \
    return fail(BGK_ERR_INVALID_ARG, "unexpected host exception");        \
  }

bgk_status select_device(const bgk_solver* s) {
  cudaError_t e = cudaSetDevice(s->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  return BGK_OK;
}

}  // namespace

extern "C" {

int bgk_abi_version(void) { return BGK_ABI_VERSION; }

const char* bgk_last_error(void) { return g_last_error.c_str(); }

const char* bgk_status_string(bgk_status st) {
  switch (st) {
    case BGK_OK: return "BGK_OK";
    case BGK_ERR_INVALID_ARG: return "BGK_ERR_INVALID_ARG";
    case BGK_ERR_UNSUPPORTED: return "BGK_ERR_UNSUPPORTED";
    case BGK_ERR_OOM: return "BGK_ERR_OOM";
    case BGK_ERR_CUDA: return "BGK_ERR_CUDA";
    case BGK_ERR_NUMERIC: return "BGK_ERR_NUMERIC";
    case BGK_ERR_TIMEOUT: return "BGK_ERR_TIMEOUT";
  }
  return "BGK_ERR_UNKNOWN";
}

bgk_status bgk_rankine_hugoniot(double mach, double gamma, double up[4], double down[4]) {
  if (!up || !down) return fail(BGK_ERR_INVALID_ARG, "null output");
  if (!(mach >= 1.0) || !(gamma > 1.0) || !std::isfinite(mach) || !std::isfinite(gamma))
    return fail(BGK_ERR_INVALID_ARG, "need mach >= 1 and gamma > 1");
  // Eq. (RH) with n- = 1, T- = 1 and u- = M sqrt(gamma/2) (units of sqrt(2RT-)).
  const double m2 = mach * mach;
  const double dens = 4.0 * m2 / (m2 + 3.0);
  const double temp = (5.0 * m2 - 1.0) * (m2 + 3.0) / (16.0 * m2);
  up[0] = 1.0;
  up[1] = mach * std::sqrt(0.5 * gamma);
  up[2] = 0.0;
  up[3] = 1.0;
  down[0] = dens;
  down[1] = up[1] / dens;
  down[2] = 0.0;
  down[3] = temp;
  return BGK_OK;
}

bgk_status bgk_create(const bgk_config* cfg, bgk_solver** out) {
  BGK_GUARD_BEGIN
  if (!out) return fail(BGK_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!cfg) return fail(BGK_ERR_INVALID_ARG, "cfg is NULL");
  bgk::Params P;
  double maxc = 0.0;
  bgk_status st = validate(cfg, &P, &maxc);
  if (st != BGK_OK) return st;

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "no usable CUDA device");
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
  if (prop.major != 10 || prop.minor != 3)
    return fail(BGK_ERR_UNSUPPORTED, "libbgk is built for sm_103a only (device %s is sm_%d%d)",
                prop.name, prop.major, prop.minor);

  if (P.tile == 0) P.tile = auto_tile(P, cfg->precision, prop.multiProcessorCount);
  if (cfg->precision != BGK_F64) P.mgl = bgk::mixed_groups_per_lane(P, P.tile);

  bgk_solver* s = new bgk_solver();
  s->prec = cfg->precision;
  s->cfg = *cfg;
  s->P = P;
  s->device = dev;
  s->stream = (cudaStream_t)cfg->cuda_stream;
  s->max_courant = maxc;
  const size_t elems = s->state_elems();
  const size_t ncell = (size_t)P.nx * P.ny;
  const int nfc = P.nx > P.ny ? P.nx : P.ny;
#define ALLOC(ptr, n)                                  \
  do {                                                 \
    cudaError_t ae = dev_alloc(s, &s->ptr, (n));       \
    if (ae != cudaSuccess) {                           \
      bgk_status rs = cuda_fail(ae, "allocate " #ptr); \
      release(s);                                      \
      return rs;                                       \
    }                                                  \
  } while (0)
  {
    const size_t bytes = s->point_bytes() * elems;
    unsigned char *f0 = nullptr, *f1 = nullptr;
    cudaError_t ae = dev_alloc(s, &f0, bytes);
    if (ae == cudaSuccess) {
      s->f[0] = f0;
      ae = dev_alloc(s, &f1, bytes);
      if (ae == cudaSuccess) s->f[1] = f1;
    }
    if (ae != cudaSuccess) {
      bgk_status rs = cuda_fail(ae, "allocate state");
      release(s);
      return rs;
    }
  }
  if (s->prec != bgk::PREC_F64) {
    ALLOC(stage, elems);
    ALLOC(m_coef, P.nv);
    ALLOC(m_cx, P.nvx);
    ALLOC(m_cy, P.nvy);
    ALLOC(m_ax, P.nvx);
    ALLOC(m_ay, P.nvy);
    ALLOC(m_ghost, (size_t)bgk::kFaces * P.nv);
    ALLOC(m_mabs, P.nv);
    ALLOC(m_sums, 12);
    ALLOC(m_ctr, 2);
  }
  ALLOC(mom_step, ncell);
  ALLOC(mom_tmp, ncell);
  ALLOC(flux_tmp, nfc);
  ALLOC(cx, P.nvx);
  ALLOC(cy, 2 * (size_t)P.nvy);
  ALLOC(coef, P.nv);
  ALLOC(shift, P.nv);
  ALLOC(cxy, P.nv);
  ALLOC(vinfo, P.nv);
  ALLOC(ghost, (size_t)bgk::kFaces * P.nv);
  ALLOC(emitted, bgk::kFaces);
  ALLOC(err, 1);
#undef ALLOC
  e = cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->f[0], 0, s->point_bytes() * elems, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->f[1], 0, s->point_bytes() * elems, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->mom_step, 0, sizeof(double4_32a) * ncell, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->err, 0, sizeof(int), s->stream);
  if (e == cudaSuccess && s->m_ctr) e = cudaMemsetAsync(s->m_ctr, 0, 2 * sizeof(unsigned), s->stream);
  if (e == cudaSuccess)
    e = bgk::launch_build_tables(P, s->cx, s->cy, s->coef, s->shift, s->cxy, s->vinfo, s->ghost,
                                 s->emitted, s->stream);
  if (e == cudaSuccess && s->prec != bgk::PREC_F64) e = bgk::launch_build_mixed_tables(P, s->tables(), s->mtables(), s->stream);
  if (e == cudaSuccess) e = s->prec == bgk::PREC_F64 ? bgk::prepare_step_f64(P) : bgk::prepare_step_mixed(P, s->prec);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) {
    bgk_status rs = cuda_fail(e, "solver set-up");
    release(s);
    return rs;
  }
  *out = s;
  return BGK_OK;
  BGK_GUARD_END
}

bgk_status bgk_destroy(bgk_solver* s) {
  if (!s) return BGK_OK;
  BGK_GUARD_BEGIN
  cudaSetDevice(s->device);
  cudaStreamSynchronize(s->stream);
  release(s);
  return BGK_OK;
  BGK_GUARD_END
}

bgk_status bgk_get_info(const bgk_solver* s, bgk_info* out) {
  if (!s || !out) return fail(BGK_ERR_INVALID_ARG, "null argument");
  std::memset(out, 0, sizeof(*out));
  out->dt = s->P.dt;
  out->dx = s->P.dx;
  out->dy = s->P.dy;
  out->dcx = s->P.dcx;
  out->dcy = s->P.dcy;
  out->dv = s->P.dv;
  out->max_courant = s->max_courant;
  out->ncell = (int64_t)s->P.nx * s->P.ny;
  out->nv = s->P.nv;
  out->state_doubles = (int64_t)s->state_elems() * 2;
  out->steps_done = s->steps_done;
  out->device_bytes = s->device_bytes;
  out->precision = s->cfg.precision;
  out->tile_cells = s->P.tile;
  return BGK_OK;
}

bgk_status bgk_init_maxwellian_step(bgk_solver* s, double x_split, const double left[4],
                                    const double right[4]) {
  BGK_GUARD_BEGIN
  if (!s || !left || !right) return fail(BGK_ERR_INVALID_ARG, "null argument");
  for (const double* st : {left, right}) {
    if (!(st[0] > 0.0) || !(st[3] > 0.0) || !finite_all({st[0], st[1], st[2], st[3]}))
      return fail(BGK_ERR_INVALID_ARG, "states need finite values, n > 0 and theta > 0");
    if (s->P.dim == 1 && st[2] != 0.0) return fail(BGK_ERR_INVALID_ARG, "uy must be 0 in 1D");
  }
  if (!std::isfinite(x_split)) return fail(BGK_ERR_INVALID_ARG, "x_split must be finite");
  bgk_status st = select_device(s);
  if (st != BGK_OK) return st;
  cudaError_t e = cudaMemsetAsync(s->err, 0, sizeof(int), s->stream);
  double2* out = s->prec == bgk::PREC_F64 ? (double2*)s->f[s->cur] : s->stage;
  if (e == cudaSuccess) e = bgk::launch_init_step(s->P, out, x_split, left, right, s->stream);
  if (e == cudaSuccess && s->prec != bgk::PREC_F64) e = store_f64(s, s->stage);
  if (e != cudaSuccess) return cuda_fail(e, "init step profile");
  s->steps_done = 0;
  return BGK_OK;
  BGK_GUARD_END
}

bgk_status bgk_init_uniform(bgk_solver* s, const double state[4], const double* xi, int xi_on_device,
                            double amplitude) {
  BGK_GUARD_BEGIN
  if (!s || !state) return fail(BGK_ERR_INVALID_ARG, "null argument");
  if (!(state[0] > 0.0) || !(state[3] > 0.0) || !finite_all({state[0], state[1], state[2], state[3], amplitude}))
    return fail(BGK_ERR_INVALID_ARG, "state needs finite values, n > 0 and theta > 0");
  if (s->P.dim == 1 && state[2] != 0.0) return fail(BGK_ERR_INVALID_ARG, "uy must be 0 in 1D");
  bgk_status st = select_device(s);
  if (st != BGK_OK) return st;
  const size_t bytes = sizeof(double2) * s->state_elems();
  const bool f64 = s->prec == bgk::PREC_F64;
  double2* out = f64 ? (double2*)s->f[s->cur] : s->stage;
  const double2* dxi = nullptr;
  cudaError_t e = cudaMemsetAsync(s->err, 0, sizeof(int), s->stream);
  if (e == cudaSuccess && xi) {
    if (xi_on_device) {
      dxi = (const double2*)xi;
    } else {
      // stage the host perturbation on the device: in the idle FP64 state
      // buffer, or in the FP64 view that the kernel then overwrites in place
      double2* buf = f64 ? (double2*)s->f[1 - s->cur] : s->stage;
      e = cudaMemcpyAsync(buf, xi, bytes, cudaMemcpyHostToDevice, s->stream);
      dxi = buf;
    }
  }
  if (e == cudaSuccess) e = bgk::launch_init_uniform(s->P, out, state, dxi, amplitude, s->stream);
  if (e == cudaSuccess && !f64) e = store_f64(s, s->stage);
  if (e == cudaSuccess && xi && !xi_on_device) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "init uniform state");
  s->steps_done = 0;
  return BGK_OK;
  BGK_GUARD_END
}

bgk_status bgk_set_state(bgk_solver* s, const double* f, int on_device) {
  BGK_GUARD_BEGIN
  if (!s || !f) return fail(BGK_ERR_INVALID_ARG, "null argument");
  bgk_status st = select_device(s);
  if (st != BGK_OK) return st;
  const size_t bytes = sizeof(double2) * s->state_elems();
  cudaError_t e = cudaMemsetAsync(s->err, 0, sizeof(int), s->stream);
  if (e == cudaSuccess) {
    if (s->prec == bgk::PREC_F64) {
      e = cudaMemcpyAsync(s->f[s->cur], f, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                          s->stream);
    } else if (on_device) {
      e = store_f64(s, (const double2*)f);
    } else {
      e = cudaMemcpyAsync(s->stage, f, bytes, cudaMemcpyHostToDevice, s->stream);
      if (e == cudaSuccess) e = store_f64(s, s->stage);
    }
  }
  // a host source may be reused as soon as the call returns
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "set_state copy");
  s->steps_done = 0;
  return BGK_OK;
  BGK_GUARD_END
}

bgk_status bgk_get_state(bgk_solver* s, double* f, int on_device) {
  BGK_GUARD_BEGIN
  if (!s || !f) return fail(BGK_ERR_INVALID_ARG, "null argument");
  bgk_status st = select_device(s);
  if (st != BGK_OK) return st;
  const size_t bytes = sizeof(double2) * s->state_elems();
  cudaError_t e;
  if (s->prec != bgk::PREC_F64 && on_device) {
    e = bgk::launch_to_f64(s->P, s->prec, s->mtables(), s->f[s->cur], (double2*)f, s->stream);
  } else {
    const double2* view = nullptr;
    e = s->f64_view(&view);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(f, view, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          s->stream);
  }
  if (e != cudaSuccess) return cuda_fail(e, "get_state copy");
  return check_flag(s);
  BGK_GUARD_END
}

bgk_status bgk_step(bgk_solver* s, int64_t nsteps) {
  BGK_GUARD_BEGIN
  if (!s) return fail(BGK_ERR_INVALID_ARG, "null solver");
  if (nsteps < 0) return fail(BGK_ERR_INVALID_ARG, "nsteps must be >= 0");
  if (nsteps == 0) return BGK_OK;
  bgk_status st = select_device(s);
  if (st != BGK_OK) return st;
  while (nsteps >= kChunk) {
    st = ensure_graph(s, s->cur);
    if (st != BGK_OK) return st;
    cudaError_t e = cudaGraphLaunch(s->graph[s->cur], s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "graph launch");
    nsteps -= kChunk;
    s->steps_done += kChunk;
  }
  while (nsteps > 0) {
    cudaError_t e = enqueue_step(s, s->cur, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "step launch");
    s->cur ^= 1;
    --nsteps;
    ++s->steps_done;
  }
  return BGK_OK;
  BGK_GUARD_END
}

bgk_status bgk_moments(bgk_solver* s, int which, double* mom, int on_device) {
  BGK_GUARD_BEGIN
  if (!s || !mom) return fail(BGK_ERR_INVALID_ARG, "null argument");
  if (which != 0 && which != 1) return fail(BGK_ERR_INVALID_ARG, "which must be 0 or 1");
  bgk_status st = select_device(s);
  if (st != BGK_OK) return st;
  const size_t ncell = (size_t)s->P.nx * s->P.ny;
  cudaError_t e = cudaSuccess;
  const double4_32a* src = s->mom_step;
  if (which == 1 && s->prec != bgk::PREC_F64) {
    // the reduced-precision step publishes float-float velocity sums
    e = bgk::launch_msum_moments(s->P, s->prec, s->mtables(), (const float2*)s->mom_step, s->mom_tmp,
                                 s->stream);
    src = s->mom_tmp;
  }
  if (which == 0) {
    const double2* view = nullptr;
    e = s->f64_view(&view);
    if (e == cudaSuccess) e = bgk::launch_moments(s->P, s->tables(), view, s->mom_tmp, s->stream);
    src = s->mom_tmp;
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(mom, src, sizeof(double4_32a) * ncell,
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "moments");
  return check_flag(s);
  BGK_GUARD_END
}

bgk_status bgk_wall_fluxes(bgk_solver* s, int face, double* out, int on_device) {
  BGK_GUARD_BEGIN
  if (!s || !out) return fail(BGK_ERR_INVALID_ARG, "null argument");
  const int nfaces = s->P.dim == 2 ? 4 : 2;
  if (face < 0 || face >= nfaces) return fail(BGK_ERR_INVALID_ARG, "face %d does not exist for dim %d", face, s->P.dim);
  bgk_status st = select_device(s);
  if (st != BGK_OK) return st;
  const int ncells = (face < 2) ? s->P.ny : s->P.nx;
  const double2* view = nullptr;
  cudaError_t e = s->f64_view(&view);
  if (e == cudaSuccess) e = bgk::launch_wall_fluxes(s->P, s->tables(), view, face, s->flux_tmp, s->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, s->flux_tmp, sizeof(double4_32a) * ncells,
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "wall fluxes");
  return check_flag(s);
  BGK_GUARD_END
}

bgk_status bgk_lid_shear(bgk_solver* s, double* J) {
  BGK_GUARD_BEGIN
  if (!s || !J) return fail(BGK_ERR_INVALID_ARG, "null argument");
  if (s->P.dim != 2) return fail(BGK_ERR_UNSUPPORTED, "the lid shear needs a 2D solver");
  bgk_status st = select_device(s);
  if (st != BGK_OK) return st;
  std::vector<double4_32a> fl((size_t)s->P.nx);
  const double2* view = nullptr;
  cudaError_t e = s->f64_view(&view);
  if (e == cudaSuccess) e = bgk::launch_wall_fluxes(s->P, s->tables(), view, bgk::YHI, s->flux_tmp, s->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(fl.data(), s->flux_tmp, sizeof(double4_32a) * fl.size(), cudaMemcpyDeviceToHost, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "lid shear");
  st = check_flag(s);  // synchronises the stream
  if (st != BGK_OK) return st;
  double sum = 0.0;
  for (const double4_32a& f : fl) sum += s->P.dx * f.y;
  *J = sum;
  return BGK_OK;
  BGK_GUARD_END
}

bgk_status bgk_sync(bgk_solver* s) {
  BGK_GUARD_BEGIN
  if (!s) return fail(BGK_ERR_INVALID_ARG, "null solver");
  bgk_status st = select_device(s);
  if (st != BGK_OK) return st;
  return check_flag(s);
  BGK_GUARD_END
}

}  // extern "C"

// ---------------------------------------------------------------------------
// bgk_step_noalloc: one step for callers that cannot allocate device memory.
// Its scratch (per-velocity tables, boundary tables, error flag) lives in this
// file-scope device array instead of cudaMalloc'ed buffers; host code reaches
// it through the address cudaGetSymbolAddress returns for the current device.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocScratchBytes = 384 * 1024;  // about 120 bytes per velocity
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Device address of the scratch array on the current device (looked up once
// per device, on the first call made with that device current).
bgk_status noalloc_scratch(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(BGK_ERR_UNSUPPORTED, "device ordinal %d too large", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
    g_noalloc_ptr[dev] = ptr;
  }
  *out = (unsigned char*)g_noalloc_ptr[dev];
  return BGK_OK;
}

}  // namespace

extern "C" bgk_status bgk_step_noalloc(const bgk_config* cfg, const double* f_in, double* f_out,
                                       double* mom_out) {
  BGK_GUARD_BEGIN
  if (!cfg || !f_in || !f_out || !mom_out) return fail(BGK_ERR_INVALID_ARG, "null argument");
  bgk::Params P;
  double maxc = 0.0;
  bgk_status st = validate(cfg, &P, &maxc);
  if (st != BGK_OK) return st;
  if (cfg->precision != BGK_F64)
    return fail(BGK_ERR_UNSUPPORTED, "bgk_step_noalloc takes BGK_F64 states only");
  // the step kernel moves (g, h) pairs as 16-byte vectors and writes each
  // cell's moments with one 32-byte store
  if ((uintptr_t)f_in % 16 || (uintptr_t)f_out % 16 || (uintptr_t)mom_out % 32)
    return fail(BGK_ERR_INVALID_ARG, "bgk_step_noalloc: f_in and f_out must be 16-byte aligned, "
                "mom_out 32-byte aligned");
  const size_t elems = (size_t)P.nx * P.ny * P.nv;
  const char *a = (const char*)f_in, *b = (const char*)f_out;
  if (a < b + elems * sizeof(double2) && b < a + elems * sizeof(double2))
    return fail(BGK_ERR_INVALID_ARG, "f_in and f_out overlap");

  // scratch layout: tables then the error flag, each 256-byte aligned
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align256(off + bytes);
    return at;
  };
  const size_t o_cx = take(sizeof(double) * P.nvx), o_cy = take(sizeof(double) * 2 * P.nvy);
  const size_t o_coef = take(sizeof(double4_32a) * P.nv), o_shift = take(sizeof(int) * P.nv);
  const size_t o_cxy = take(sizeof(double2) * P.nv), o_vinfo = take(sizeof(int) * P.nv);
  const size_t o_ghost = take(sizeof(double2) * bgk::kFaces * P.nv);
  const size_t o_emit = take(sizeof(double) * bgk::kFaces), o_err = take(sizeof(int));
  if (off > kNoAllocScratchBytes)
    return fail(BGK_ERR_UNSUPPORTED, "bgk_step_noalloc: tables need %zu bytes, the scratch holds %zu",
                off, kNoAllocScratchBytes);

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "no usable CUDA device");
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
  if (prop.major != 10 || prop.minor != 3)
    return fail(BGK_ERR_UNSUPPORTED, "libbgk is built for sm_103a only (device %s is sm_%d%d)",
                prop.name, prop.major, prop.minor);
  if (P.tile == 0) P.tile = auto_tile(P, BGK_F64, prop.multiProcessorCount);
  unsigned char* base = nullptr;
  st = noalloc_scratch(dev, &base);
  if (st != BGK_OK) return st;

  bgk::Tables T;
  double* cx = (double*)(base + o_cx);
  double* cy = (double*)(base + o_cy);
  double4_32a* coef = (double4_32a*)(base + o_coef);
  int* shift = (int*)(base + o_shift);
  double2* cxy = (double2*)(base + o_cxy);
  int* vinfo = (int*)(base + o_vinfo);
  double2* ghost = (double2*)(base + o_ghost);
  double* emitted = (double*)(base + o_emit);
  int* err = (int*)(base + o_err);
  T.cx = cx;
  T.cy = cy;
  T.cy2 = cy + P.nvy;
  T.coef = coef;
  T.shift = shift;
  T.cxy = cxy;
  T.vinfo = vinfo;
  T.ghost = ghost;
  T.emitted = emitted;

  cudaStream_t stream = (cudaStream_t)cfg->cuda_stream;
  e = cudaMemsetAsync(err, 0, sizeof(int), stream);
  if (e == cudaSuccess) e = bgk::launch_build_tables(P, cx, cy, coef, shift, cxy, vinfo, ghost, emitted, stream);
  if (e == cudaSuccess) e = bgk::prepare_step_f64(P);
  if (e == cudaSuccess)
    e = bgk::launch_step_f64(P, T, (const double2*)f_in, (double2*)f_out, (double4_32a*)mom_out, err, stream);
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cuda_fail(e, "bgk_step_noalloc");
  if (h & bgk::ERR_MOMENT) return fail(BGK_ERR_NUMERIC, "a cell reached n <= 0, theta <= 0 or a non-finite moment");
  if (h & bgk::ERR_EFFECTIVE) return fail(BGK_ERR_NUMERIC, "the effective-parameter iteration did not converge in a cell");
  return BGK_OK;
  BGK_GUARD_END
}

// ---------------------------------------------------------------------------
// Autotuner and batches.
// ---------------------------------------------------------------------------
namespace {

bool tile_admissible(const bgk_solver* s, int t) {
  bgk::Params P = s->P;
  P.tile = t;
  if (s->prec != bgk::PREC_F64 && bgk::mixed_groups_per_lane(P, t) == 0) return false;
  return step_smem(P, s->prec, t) <= kMaxSmem;
}

cudaError_t set_tile(bgk_solver* s, int t) {
  s->P.tile = t;
  if (s->prec != bgk::PREC_F64) s->P.mgl = bgk::mixed_groups_per_lane(s->P, t);
  s->cfg.tile_cells = t;
  for (auto& g : s->graph)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  ++s->gen;
  return s->prec == bgk::PREC_F64 ? bgk::prepare_step_f64(s->P) : bgk::prepare_step_mixed(s->P, s->prec);
}

}  // namespace

struct bgk_batch {
  std::vector<bgk_solver*> inst;
  cudaStream_t stream = nullptr;
  cudaStream_t origin = nullptr;
  std::vector<cudaStream_t> branch;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  struct Graph {
    std::vector<int64_t> key;  // per instance: parity and generation; then steps
    cudaGraphExec_t exec = nullptr;
  };
  std::vector<Graph> graphs;
  // persistent mode: one cooperative kernel per bgk_batch_step call
  int persistent = 0;
  double timeout_s = 5.0;
  bgk::GridBarrier* bar = nullptr;
  int* gerr = nullptr;
  struct PGraph {
    std::vector<int64_t> key;  // per instance: parity and generation; then steps
    cudaGraphExec_t exec = nullptr;
    bgk::PInstance* d_inst = nullptr;
  };
  std::vector<PGraph> pgraphs;
};

namespace {

void batch_release(bgk_batch* b) {
  if (!b) return;
  for (auto& g : b->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  for (auto& g : b->pgraphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.d_inst) cudaFree(g.d_inst);
  }
  if (b->bar) cudaFree(b->bar);
  if (b->gerr) cudaFree(b->gerr);
  for (auto* s : b->inst) release(s);
  for (auto st : b->branch)
    if (st) cudaStreamDestroy(st);
  for (auto ev : b->join)
    if (ev) cudaEventDestroy(ev);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->origin) cudaStreamDestroy(b->origin);
  delete b;
}

// The captured graph for `steps` steps from the instances' current buffers.
bgk_status batch_graph(bgk_batch* b, int steps, cudaGraphExec_t* out) {
  std::vector<int64_t> key;
  for (auto* s : b->inst) {
    key.push_back(s->cur);
    key.push_back(s->gen);
  }
  key.push_back(steps);
  for (auto& g : b->graphs)
    if (g.key == key) {
      *out = g.exec;
      return BGK_OK;
    }
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaGetLastError();  // a stale error would be blamed on a launch below
  if (e != cudaSuccess) return cuda_fail(e, "pending CUDA error before batch capture");
  e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(e, "batch capture begin");
  cudaError_t le = cudaEventRecord(b->fork, b->origin);
  size_t bad = b->inst.size();
  for (size_t i = 0; i < b->inst.size() && le == cudaSuccess; ++i) {
    bad = i;
    bgk_solver* s = b->inst[i];
    le = cudaStreamWaitEvent(b->branch[i], b->fork, 0);
    int buf = s->cur;
    for (int t = 0; t < steps && le == cudaSuccess; ++t) {
      le = enqueue_step(s, buf, b->branch[i]);
      buf ^= 1;
    }
    if (le == cudaSuccess) le = cudaEventRecord(b->join[i], b->branch[i]);
    if (le == cudaSuccess) le = cudaStreamWaitEvent(b->origin, b->join[i], 0);
  }
  e = cudaStreamEndCapture(b->origin, &graph);
  if (le != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    const bgk_solver* s = b->inst[bad < b->inst.size() ? bad : 0];
    return fail(BGK_ERR_CUDA, "batch capture, instance %zu (dim %d, %dx%d cells, %d velocities, precision %d, "
                "tile %d, groups %d): %s", bad, s->P.dim, s->P.nx, s->P.ny, s->P.nv, s->prec, s->P.tile,
                s->P.mgl, cudaGetErrorString(le));
  }
  if (e != cudaSuccess) return cuda_fail(e, "batch capture end");
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e, "batch graph instantiate");
  if (b->graphs.size() >= 4) {
    cudaGraphExecDestroy(b->graphs.front().exec);
    b->graphs.erase(b->graphs.begin());
  }
  b->graphs.push_back({key, exec});
  *out = exec;
  return BGK_OK;
}

// The captured persistent launch for `steps` steps from the instances'
// current buffers: a reset of the grid barrier, then the cooperative kernel.
bgk_status batch_pgraph(bgk_batch* b, int steps, cudaGraphExec_t* out) {
  std::vector<int64_t> key;
  for (auto* s : b->inst) {
    key.push_back(s->cur);
    key.push_back(s->gen);
  }
  key.push_back(steps);
  for (auto& g : b->pgraphs)
    if (g.key == key) {
      *out = g.exec;
      return BGK_OK;
    }
  std::vector<bgk::PInstance> h(b->inst.size());
  int units = 0;
  size_t smem = 0;
  for (size_t i = 0; i < b->inst.size(); ++i) {
    bgk_solver* s = b->inst[i];
    bgk::PInstance& I = h[i];
    std::memset(&I, 0, sizeof(I));
    I.P = s->P;
    I.M = s->mtables();
    I.f_even = s->f[s->cur];
    I.f_odd = s->f[s->cur ^ 1];
    I.msum = reinterpret_cast<float2*>(s->mom_step);
    I.err = s->err;
    I.kind = bgk::persistent_kind(s->P);
    I.unit0 = units;
    I.units = bgk::persistent_units(s->P, I.kind);
    units += I.units;
    smem = std::max(smem, bgk::persistent_smem(s->P));
  }
  int grid = 0;
  cudaError_t e = bgk::persistent_grid(smem, &grid);
  if (e != cudaSuccess) return cuda_fail(e, "persistent occupancy");
  if (grid < 1) return fail(BGK_ERR_UNSUPPORTED, "the persistent kernel does not fit on an SM");
  grid = std::min(grid, units);
  bgk::PInstance* d_inst = nullptr;
  e = cudaMalloc(&d_inst, sizeof(bgk::PInstance) * h.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(d_inst, h.data(), sizeof(bgk::PInstance) * h.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    if (d_inst) cudaFree(d_inst);
    return cuda_fail(e, "persistent descriptors");
  }
  const long long spins = (long long)std::max(1.0, std::min(9.0e18, b->timeout_s / 2.0e-7));
  cudaGraph_t graph = nullptr;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal);
  cudaError_t le = e;
  if (le == cudaSuccess) le = cudaMemsetAsync(b->bar, 0, sizeof(bgk::GridBarrier), b->origin);
  if (le == cudaSuccess) le = bgk::upload_persistent(d_inst, (int)h.size(), b->origin);
  if (le == cudaSuccess)
    le = bgk::launch_persistent((int)h.size(), units, steps, b->bar, b->gerr, spins, grid, smem, b->origin);
  if (e == cudaSuccess) e = cudaStreamEndCapture(b->origin, &graph);
  if (le != cudaSuccess || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaFree(d_inst);
    return cuda_fail(le != cudaSuccess ? le : e, "persistent batch capture");
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    cudaFree(d_inst);
    return cuda_fail(e, "persistent graph instantiate");
  }
  if (b->pgraphs.size() >= 4) {
    cudaGraphExecDestroy(b->pgraphs.front().exec);
    cudaFree(b->pgraphs.front().d_inst);
    b->pgraphs.erase(b->pgraphs.begin());
  }
  b->pgraphs.push_back({key, exec, d_inst});
  *out = exec;
  return BGK_OK;
}

void drop_pgraphs(bgk_batch* b) {
  for (auto& g : b->pgraphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.d_inst) cudaFree(g.d_inst);
  }
  b->pgraphs.clear();
}

}  // namespace

extern "C" {

bgk_status bgk_batch_set_persistent(bgk_batch* b, int enable, double timeout_s) {
  BGK_GUARD_BEGIN
  if (!b) return fail(BGK_ERR_INVALID_ARG, "null batch");
  if (enable != 0 && enable != 1) return fail(BGK_ERR_INVALID_ARG, "enable must be 0 or 1");
  if (!(timeout_s > 0.0) || !std::isfinite(timeout_s)) return fail(BGK_ERR_INVALID_ARG, "timeout must be > 0");
  bgk_status st = select_device(b->inst[0]);
  if (st != BGK_OK) return st;
  if (enable) {
    for (size_t i = 0; i < b->inst.size(); ++i) {
      bgk_solver* s = b->inst[i];
      if (s->prec != bgk::PREC_F32)
        return fail(BGK_ERR_UNSUPPORTED, "instance %zu: the persistent kernel runs FP32 instances only", i);
      if (b->inst.size() > (size_t)bgk::kMaxPersistInstances)
        return fail(BGK_ERR_UNSUPPORTED, "the persistent kernel takes at most %d instances", bgk::kMaxPersistInstances);
      if (bgk::persistent_kind(s->P) < 0) {
        // 2D: the largest admissible tile with at most 4 groups per lane
        int chosen = 0;
        for (int t : {8, 4, 2, 1}) {
          if (!tile_admissible(s, t)) continue;
          bgk::Params q = s->P;
          q.tile = t;
          if (bgk::persistent_kind(q) >= 0) {
            chosen = t;
            break;
          }
        }
        if (!chosen) return fail(BGK_ERR_UNSUPPORTED, "instance %zu: no tile the persistent kernel supports", i);
        cudaError_t e = set_tile(s, chosen);
        if (e != cudaSuccess) return cuda_fail(e, "persistent tile");
      }
    }
    cudaError_t e = cudaSuccess;
    if (!b->bar) e = cudaMalloc(&b->bar, sizeof(bgk::GridBarrier));
    if (e == cudaSuccess && !b->gerr) {
      e = cudaMalloc(&b->gerr, sizeof(int));
      if (e == cudaSuccess) e = cudaMemset(b->gerr, 0, sizeof(int));
    }
    if (e != cudaSuccess) return cuda_fail(e, "persistent barrier");
  }
  drop_pgraphs(b);
  b->persistent = enable;
  b->timeout_s = timeout_s;
  return BGK_OK;
  BGK_GUARD_END
}

bgk_status bgk_autotune(bgk_solver* s, int trial_steps, int* tile_out) {
  BGK_GUARD_BEGIN
  if (!s) return fail(BGK_ERR_INVALID_ARG, "null solver");
  if (trial_steps < 1) return fail(BGK_ERR_INVALID_ARG, "trial_steps must be >= 1");
  bgk_status st = select_device(s);
  if (st != BGK_OK) return st;
  const size_t bytes = s->point_bytes() * s->state_elems();
  void* saved = nullptr;
  cudaError_t e = cudaMalloc(&saved, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "autotune state copy");
  const int cur0 = s->cur;
  const int64_t done0 = s->steps_done;
  const int tile0 = s->P.tile;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  e = cudaMemcpyAsync(saved, s->f[cur0], bytes, cudaMemcpyDeviceToDevice, s->stream);
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  int best = tile0;
  float best_ms = 0.f;
  for (int t : {1, 2, 4, 8}) {
    if (e != cudaSuccess) break;
    if (!tile_admissible(s, t)) continue;
    e = set_tile(s, t);
    int buf = cur0;
    if (e == cudaSuccess) {  // one warm-up step, then the timed trial
      e = enqueue_step(s, buf, s->stream);
      buf ^= 1;
    }
    if (e == cudaSuccess) e = cudaEventRecord(t0, s->stream);
    for (int k = 0; k < trial_steps && e == cudaSuccess; ++k) {
      e = enqueue_step(s, buf, s->stream);
      buf ^= 1;
    }
    if (e == cudaSuccess) e = cudaEventRecord(t1, s->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    if (e == cudaSuccess && (best_ms == 0.f || ms < best_ms)) {
      best_ms = ms;
      best = t;
    }
    // put the saved state back
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->f[cur0], saved, bytes, cudaMemcpyDeviceToDevice, s->stream);
  }
  if (e == cudaSuccess) e = set_tile(s, best);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->err, 0, sizeof(int), s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  s->cur = cur0;
  s->steps_done = done0;
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  cudaFree(saved);
  if (e != cudaSuccess) return cuda_fail(e, "autotune");
  if (tile_out) *tile_out = best;
  return BGK_OK;
  BGK_GUARD_END
}

bgk_status bgk_batch_create(const bgk_config* cfgs, int count, void* cuda_stream, bgk_batch** out) {
  BGK_GUARD_BEGIN
  if (!out) return fail(BGK_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!cfgs || count < 1) return fail(BGK_ERR_INVALID_ARG, "need at least one configuration");
  bgk_batch* b = new bgk_batch();
  b->stream = (cudaStream_t)cuda_stream;
  for (int i = 0; i < count; ++i) {
    bgk_config c = cfgs[i];
    c.cuda_stream = cuda_stream;
    bgk_solver* s = nullptr;
    bgk_status st = bgk_create(&c, &s);
    if (st != BGK_OK) {
      const std::string msg = g_last_error;
      batch_release(b);
      return fail(st, "instance %d: %s", i, msg.c_str());
    }
    b->inst.push_back(s);
  }
  cudaError_t e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  for (int i = 0; i < count && e == cudaSuccess; ++i) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) b->branch.push_back(st);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) b->join.push_back(ev);
  }
  if (e != cudaSuccess) {
    bgk_status rs = cuda_fail(e, "batch streams");
    batch_release(b);
    return rs;
  }
  *out = b;
  return BGK_OK;
  BGK_GUARD_END
}

bgk_status bgk_batch_solver(bgk_batch* b, int index, bgk_solver** out) {
  if (!b || !out) return fail(BGK_ERR_INVALID_ARG, "null argument");
  if (index < 0 || index >= (int)b->inst.size())
    return fail(BGK_ERR_INVALID_ARG, "instance %d out of range (batch of %zu)", index, b->inst.size());
  *out = b->inst[index];
  return BGK_OK;
}

bgk_status bgk_batch_step(bgk_batch* b, int64_t nsteps) {
  BGK_GUARD_BEGIN
  if (!b) return fail(BGK_ERR_INVALID_ARG, "null batch");
  if (nsteps < 0) return fail(BGK_ERR_INVALID_ARG, "nsteps must be >= 0");
  if (nsteps == 0) return BGK_OK;
  bgk_status st = select_device(b->inst[0]);
  if (st != BGK_OK) return st;
  if (b->persistent) {
    const int k = (int)std::min<int64_t>(nsteps, 1 << 30);
    cudaGraphExec_t exec = nullptr;
    st = batch_pgraph(b, k, &exec);
    if (st != BGK_OK) return st;
    cudaError_t e = cudaGraphLaunch(exec, b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "persistent batch launch");
    for (auto* s : b->inst) {
      s->steps_done += k;
      if (k & 1) s->cur ^= 1;
    }
    nsteps -= k;
  }
  while (nsteps > 0) {
    const int k = (int)std::min<int64_t>(nsteps, kChunk);
    cudaGraphExec_t exec = nullptr;
    st = batch_graph(b, k, &exec);
    if (st != BGK_OK) return st;
    cudaError_t e = cudaGraphLaunch(exec, b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch graph launch");
    for (auto* s : b->inst) {
      s->steps_done += k;
      if (k & 1) s->cur ^= 1;
    }
    nsteps -= k;
  }
  return BGK_OK;
  BGK_GUARD_END
}

bgk_status bgk_batch_sync(bgk_batch* b) {
  BGK_GUARD_BEGIN
  if (!b) return fail(BGK_ERR_INVALID_ARG, "null batch");
  if (b->gerr) {
    int h = 0;
    cudaError_t e = cudaSetDevice(b->inst[0]->device);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, b->gerr, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess && h) e = cudaMemsetAsync(b->gerr, 0, sizeof(int), b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch synchronize");
    if (h & bgk::ERR_TIMEOUT)
      return fail(BGK_ERR_TIMEOUT, "a grid barrier of the persistent batch kernel timed out; the steps did not complete");
  }
  for (size_t i = 0; i < b->inst.size(); ++i) {
    bgk_status st = bgk_sync(b->inst[i]);
    if (st != BGK_OK) {
      const std::string msg = g_last_error;
      return fail(st, "instance %zu: %s", i, msg.c_str());
    }
  }
  return BGK_OK;
  BGK_GUARD_END
}

bgk_status bgk_batch_destroy(bgk_batch* b) {
  if (!b) return BGK_OK;
  BGK_GUARD_BEGIN
  cudaSetDevice(b->inst[0]->device);
  cudaStreamSynchronize(b->stream);
  batch_release(b);
  return BGK_OK;
  BGK_GUARD_END
}

bgk_status bgk_batch_autotune(bgk_batch* b, int trial_steps) {
  BGK_GUARD_BEGIN
  if (!b) return fail(BGK_ERR_INVALID_ARG, "null batch");
  std::map<std::tuple<int, int, int, int, int, int>, int> known;
  for (size_t i = 0; i < b->inst.size(); ++i) {
    bgk_solver* s = b->inst[i];
    const auto key = std::make_tuple(s->P.dim, s->P.nx, s->P.ny, s->P.nvx, s->P.nvy, s->prec);
    auto it = known.find(key);
    if (it != known.end()) {
      cudaError_t e = set_tile(s, it->second);
      if (e != cudaSuccess) return cuda_fail(e, "batch autotune");
      continue;
    }
    int best = 0;
    bgk_status st = bgk_autotune(s, trial_steps, &best);
    if (st != BGK_OK) {
      const std::string msg = g_last_error;
      return fail(st, "instance %zu: %s", i, msg.c_str());
    }
    known[key] = best;
  }
  return BGK_OK;
  BGK_GUARD_END
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Adjoint host loop (kernels in bgk_adjoint.cu).
//   forward:   f^0 .. f^N, saving f^{mK} (M checkpoints);
//   seed:      lambda^N = dJ/df^N, J per lid cell, explicit dJ/dU_W;
//   reverse:   per segment m = M-1 .. 0, recompute f^{mK} .. f^{mK+len}
//              (with the moments and effective parameters of each step),
//              then one adj_step launch per step n (streaming adjoint of
//              step n+1 fused with the collision adjoint of step n; both
//              read only f^{n+1});
//   finish:    the streaming adjoint of step 0 gives lambda^0 = dJ/df^0.
// ---------------------------------------------------------------------------
extern "C" bgk_status bgk_adjoint_lid_shear(bgk_solver* s, int64_t nsteps, int checkpoint_every, double* dJ_df0,
                                            int on_device, double out[3]) {
  BGK_GUARD_BEGIN
  if (!s || !out) return fail(BGK_ERR_INVALID_ARG, "null argument");
  if (nsteps < 1 || checkpoint_every < 0)
    return fail(BGK_ERR_INVALID_ARG, "nsteps must be >= 1 and checkpoint_every >= 0");
  if (s->P.dim != 2 || s->prec != bgk::PREC_F64 || !s->P.relax_exact)
    return fail(BGK_ERR_UNSUPPORTED, "the adjoint needs dim 2, BGK_F64 and exact relaxation");
  if (s->P.bc_kind[bgk::YHI] != BGK_BC_DIFFUSE) return fail(BGK_ERR_UNSUPPORTED, "the adjoint needs a diffuse lid (YHI)");
  if (s->cfg.dt != 0.0) return fail(BGK_ERR_UNSUPPORTED, "the adjoint needs dt derived from cfl (dt = 0)");
  bgk_status st = select_device(s);
  if (st != BGK_OK) return st;
  const bgk::Params& P = s->P;
  const bgk::Tables T = s->tables();
  const size_t elems = s->state_elems(), sbytes = sizeof(double2) * elems;
  // checkpoint_every = 0: K = ceil(sqrt(nsteps)), which minimises the
  // nsteps / K checkpoints plus the K + 1 states of a segment
  int64_t k0 = checkpoint_every;
  if (k0 == 0) {
    k0 = (int64_t)std::ceil(std::sqrt((double)nsteps));
    while (k0 * k0 < nsteps) ++k0;
    while (k0 > 1 && (k0 - 1) * (k0 - 1) >= nsteps) --k0;
  }
  const int K = (int)std::min<int64_t>(k0, nsteps);
  const int64_t M = (nsteps + K - 1) / K;
  const int ncell = P.nx * P.ny;
  std::vector<void*> bufs;
  auto alloc = [&](size_t bytes, void** p) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) bufs.push_back(*p);
    return e;
  };
  auto cleanup = [&]() {
    for (void* b : bufs) cudaFree(b);
  };
  double2 *ckpt = nullptr, *seg = nullptr, *lamA = nullptr, *lamB = nullptr, *dghost = nullptr;
  double4_32a *qbuf = nullptr, *pbuf = nullptr;
  double *dlnl = nullptr, *duw = nullptr, *Jk = nullptr, *duw0 = nullptr, *demit = nullptr;
  cudaError_t e = alloc(sbytes * M, (void**)&ckpt);
  if (e == cudaSuccess) e = alloc(sbytes * (K + 1), (void**)&seg);
  if (e == cudaSuccess) e = alloc(sizeof(double4_32a) * ncell * K, (void**)&qbuf);
  if (e == cudaSuccess) e = alloc(sizeof(double4_32a) * ncell * K, (void**)&pbuf);
  if (e == cudaSuccess) e = alloc(sbytes, (void**)&lamA);
  if (e == cudaSuccess) e = alloc(sbytes, (void**)&lamB);
  if (e == cudaSuccess) e = alloc(sizeof(double2) * P.nv, (void**)&dghost);
  if (e == cudaSuccess) e = alloc(sizeof(double) * ncell, (void**)&dlnl);
  if (e == cudaSuccess) e = alloc(sizeof(double) * P.nx, (void**)&duw);
  if (e == cudaSuccess) e = alloc(sizeof(double) * P.nx, (void**)&Jk);
  if (e == cudaSuccess) e = alloc(sizeof(double) * P.nx, (void**)&duw0);
  if (e == cudaSuccess) e = alloc(sizeof(double), (void**)&demit);
  if (e != cudaSuccess) {
    cleanup();
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? fail(BGK_ERR_OOM, "adjoint buffers (%lld checkpoints, %d segment states)",
                                                 (long long)M, K + 1)
                                          : cuda_fail(e, "adjoint buffers");
  }
  cudaStream_t stream = s->stream;
  // forward with checkpoints f^{mK}
  for (int64_t m = 0; m < M && e == cudaSuccess; ++m) {
    e = cudaMemcpyAsync(ckpt + (size_t)m * elems, s->f[s->cur], sbytes, cudaMemcpyDeviceToDevice, stream);
    const int64_t len = std::min<int64_t>(K, nsteps - m * K);
    for (int64_t t = 0; t < len && e == cudaSuccess; ++t) {
      e = enqueue_step(s, s->cur, stream);
      s->cur ^= 1;
      ++s->steps_done;
    }
  }
  double demit_h = 0.0;
  if (e == cudaSuccess) e = bgk::launch_adj_lid_table(P, T, dghost, demit, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&demit_h, demit, sizeof(double), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(lamA, 0, sbytes, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(dlnl, 0, sizeof(double) * ncell, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(duw, 0, sizeof(double) * P.nx, stream);
  if (e == cudaSuccess)
    e = bgk::launch_adj_seed(P, T, (const double2*)s->f[s->cur], lamA, dghost, demit_h, Jk, duw0, stream);
  // reverse, segment by segment
  double2* lam = lamA;
  double2* other = lamB;
  int tilde = 0;
  for (int64_t m = M - 1; m >= 0 && e == cudaSuccess; --m) {
    const int64_t len = std::min<int64_t>(K, nsteps - m * K);
    e = cudaMemcpyAsync(seg, ckpt + (size_t)m * elems, sbytes, cudaMemcpyDeviceToDevice, stream);
    for (int64_t t = 0; t < len && e == cudaSuccess; ++t)
      e = bgk::launch_step_f64(P, T, seg + (size_t)t * elems, seg + (size_t)(t + 1) * elems, qbuf + (size_t)t * ncell,
                               s->err, stream, pbuf + (size_t)t * ncell);
    for (int64_t t = len - 1; t >= 0 && e == cudaSuccess; --t) {
      e = bgk::launch_adj_step(P, T, seg + (size_t)(t + 1) * elems, qbuf + (size_t)t * ncell,
                               pbuf + (size_t)t * ncell, lam, tilde, 1, other, dghost, demit_h, dlnl, duw, stream);
      std::swap(lam, other);
      tilde = 1;
    }
  }
  // streaming adjoint of step 0 (seg holds f^0 .. of segment 0)
  if (e == cudaSuccess)
    e = bgk::launch_adj_step(P, T, seg, nullptr, nullptr, lam, 1, 0, other, dghost, demit_h, dlnl, duw,
                             stream);
  std::swap(lam, other);
  // gather: J, the scalar derivatives (host sums in a fixed order), dJ/df0
  std::vector<double> h_jk(P.nx), h_duw0(P.nx), h_duw(P.nx), h_dlnl(ncell);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_jk.data(), Jk, sizeof(double) * P.nx, cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_duw0.data(), duw0, sizeof(double) * P.nx, cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_duw.data(), duw, sizeof(double) * P.nx, cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_dlnl.data(), dlnl, sizeof(double) * ncell, cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess && dJ_df0)
    e = cudaMemcpyAsync(dJ_df0, lam, sbytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  cleanup();
  if (e != cudaSuccess) return cuda_fail(e, "adjoint");
  double J = 0.0, duw_t = 0.0, dlnl_t = 0.0;
  for (int k = 0; k < P.nx; ++k) {
    J += h_jk[k];
    duw_t += h_duw0[k] + h_duw[k];
  }
  for (int c = 0; c < ncell; ++c) dlnl_t += h_dlnl[c];
  out[0] = J;
  out[1] = J + dlnl_t;  // J itself scales with dx
  out[2] = duw_t;
  return check_flag(s);
  BGK_GUARD_END
}

// ---------------------------------------------------------------------------
// Full 3D velocity grid, one spatial dimension (kernels in bgk_step3v.cu).
// ---------------------------------------------------------------------------
struct bgk3v_solver {
  bgk3v_config cfg;
  bgk::Params3v P;
  bgk::Inflow3v inflow;
  int device = 0;
  cudaStream_t stream = nullptr;
  double* f[2] = {nullptr, nullptr};
  int cur = 0;
  double* mom_step = nullptr;  // [ncell][5] of the last post-streaming state
  double* mom_tmp = nullptr;
  double* c[3] = {nullptr, nullptr, nullptr};
  double* cc = nullptr;
  int* shift = nullptr;
  int* upwind = nullptr;
  double* rem = nullptr;
  double* ghost = nullptr;
  int* err = nullptr;
  int64_t steps_done = 0;
  int64_t device_bytes = 0;
  double max_courant = 0.0;
  bgk::Tables3v tables() const {
    bgk::Tables3v T;
    T.c[0] = c[0];
    T.c[1] = c[1];
    T.c[2] = c[2];
    T.c2 = cc;
    T.shift = shift;
    T.upwind = upwind;
    T.rem = rem;
    T.ghost = ghost;
    return T;
  }
  size_t state_elems() const { return (size_t)P.nx * P.nv; }
};

namespace {

void release3v(bgk3v_solver* s) {
  if (!s) return;
  void* bufs[] = {s->f[0], s->f[1], s->mom_step, s->mom_tmp, s->c[0], s->c[1], s->c[2], s->cc,
                  s->shift, s->upwind, s->rem, s->ghost, s->err};
  for (void* b : bufs)
    if (b) cudaFree(b);
  delete s;
}

bgk_status validate3v(const bgk3v_config* c, bgk::Params3v& p, double* max_courant) {
  if (c->nx < 1) return fail(BGK_ERR_INVALID_ARG, "nx must be >= 1");
  const int n3[3] = {c->nvx, c->nvy, c->nvz};
  for (int a = 0; a < 3; ++a) {
    if (n3[a] < 1) return fail(BGK_ERR_INVALID_ARG, "velocity cell counts must be >= 1");
    if (n3[a] > 256) return fail(BGK_ERR_UNSUPPORTED, "at most 256 velocity cells per component (got %d)", n3[a]);
    if (!std::isfinite(c->vmin[a]) || !std::isfinite(c->vmax[a]) || !(c->vmax[a] > c->vmin[a]))
      return fail(BGK_ERR_INVALID_ARG, "velocity box component %d must have vmax > vmin", a);
  }
  const long long nv = (long long)c->nvx * c->nvy * c->nvz;
  if (nv > (1LL << 24)) return fail(BGK_ERR_UNSUPPORTED, "%lld velocities per cell (max 2^24)", nv);
  if (!std::isfinite(c->x0) || !std::isfinite(c->lx) || !(c->lx > 0.0))
    return fail(BGK_ERR_INVALID_ARG, "lx must be finite and > 0");
  if (!std::isfinite(c->omega)) return fail(BGK_ERR_INVALID_ARG, "omega must be finite");
  if (c->conservative != 0 && c->conservative != 1) return fail(BGK_ERR_INVALID_ARG, "conservative must be 0 or 1");
  if (c->relax_exact != 0 && c->relax_exact != 1) return fail(BGK_ERR_INVALID_ARG, "relax_exact must be 0 or 1");
  if (c->reserved0 != 0 || c->reserved1 != 0) return fail(BGK_ERR_INVALID_ARG, "reserved fields must be 0");
  for (int e = 0; e < 2; ++e) {
    const double* st = c->inflow[e];
    for (int k = 0; k < 5; ++k)
      if (!std::isfinite(st[k])) return fail(BGK_ERR_INVALID_ARG, "inflow state %d is not finite", e);
    if (!(st[0] > 0.0) || !(st[4] > 0.0)) return fail(BGK_ERR_INVALID_ARG, "inflow state %d needs n > 0 and theta > 0", e);
  }
  p.nx = c->nx;
  p.nvx = c->nvx;
  p.nvy = c->nvy;
  p.nvz = c->nvz;
  p.nv = (int)nv;
  p.conservative = c->conservative;
  p.relax_exact = c->relax_exact;
  p.x0 = c->x0;
  p.dx = c->lx / c->nx;
  p.omega = c->omega;
  double mx = 0.0;
  for (int a = 0; a < 3; ++a) {
    p.dc[a] = (c->vmax[a] - c->vmin[a]) / n3[a];
    p.vmin[a] = c->vmin[a];
  }
  for (int j = 0; j < c->nvx; ++j) mx = std::max(mx, std::fabs(c->vmin[0] + (j + 0.5) * p.dc[0]));
  p.dv = p.dc[0] * p.dc[1] * p.dc[2];
  if (c->dt > 0.0 && std::isfinite(c->dt)) {
    p.dt = c->dt;
  } else if (c->dt == 0.0 && c->cfl > 0.0 && std::isfinite(c->cfl) && mx > 0.0) {
    p.dt = c->cfl * p.dx / mx;
  } else {
    return fail(BGK_ERR_INVALID_ARG, "need dt > 0, or dt = 0 and cfl > 0");
  }
  *max_courant = mx * p.dt / p.dx;
  if (*max_courant > 1e6) return fail(BGK_ERR_UNSUPPORTED, "Courant number %.3g is too large", *max_courant);
  return BGK_OK;
}

template <typename T>
cudaError_t dev_alloc3(bgk3v_solver* s, T** p, size_t count) {
  const size_t bytes = sizeof(T) * (count ? count : 1);
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e == cudaSuccess) s->device_bytes += (int64_t)bytes;
  return e;
}

bgk_status check_flag3v(bgk3v_solver* s) {
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, s->err, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
  if (h & bgk::ERR_MOMENT) return fail(BGK_ERR_NUMERIC, "a cell reached n <= 0, theta <= 0 or a non-finite moment");
  if (h & bgk::ERR_EFFECTIVE)
    return fail(BGK_ERR_NUMERIC, "the effective-parameter iteration did not converge in a cell");
  return BGK_OK;
}

}  // namespace

extern "C" {

bgk_status bgk3v_create(const bgk3v_config* cfg, bgk3v_solver** out) {
  BGK_GUARD_BEGIN
  if (!out) return fail(BGK_ERR_INVALID_ARG, "null output");
  *out = nullptr;
  if (!cfg) return fail(BGK_ERR_INVALID_ARG, "null config");
  bgk::Params3v P{};
  double mc = 0.0;
  bgk_status st = validate3v(cfg, P, &mc);
  if (st != BGK_OK) return st;
  bgk3v_solver* s = new bgk3v_solver();
  s->cfg = *cfg;
  s->P = P;
  s->max_courant = mc;
  s->stream = static_cast<cudaStream_t>(cfg->cuda_stream);
  for (int e = 0; e < 2; ++e)
    for (int k = 0; k < 5; ++k) s->inflow.s[e][k] = cfg->inflow[e][k];
  cudaError_t e = cudaGetDevice(&s->device);
  const size_t n = s->state_elems();
  if (e == cudaSuccess) e = dev_alloc3(s, &s->f[0], n);
  if (e == cudaSuccess) e = dev_alloc3(s, &s->f[1], n);
  if (e == cudaSuccess) e = dev_alloc3(s, &s->mom_step, (size_t)P.nx * 5);
  if (e == cudaSuccess) e = dev_alloc3(s, &s->mom_tmp, (size_t)P.nx * 5);
  if (e == cudaSuccess) e = dev_alloc3(s, &s->c[0], (size_t)P.nvx);
  if (e == cudaSuccess) e = dev_alloc3(s, &s->c[1], (size_t)P.nvy);
  if (e == cudaSuccess) e = dev_alloc3(s, &s->c[2], (size_t)P.nvz);
  if (e == cudaSuccess) e = dev_alloc3(s, &s->cc, (size_t)P.nv);
  if (e == cudaSuccess) e = dev_alloc3(s, &s->shift, (size_t)P.nvx);
  if (e == cudaSuccess) e = dev_alloc3(s, &s->upwind, (size_t)P.nvx);
  if (e == cudaSuccess) e = dev_alloc3(s, &s->rem, (size_t)P.nvx);
  if (e == cudaSuccess) e = dev_alloc3(s, &s->ghost, 2 * (size_t)P.nv);
  if (e == cudaSuccess) e = dev_alloc3(s, &s->err, 1);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->f[0], 0, sizeof(double) * n, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->mom_step, 0, sizeof(double) * P.nx * 5, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->err, 0, sizeof(int), s->stream);
  if (e == cudaSuccess)
    e = bgk::launch_tables3v(P, s->c[0], s->c[1], s->c[2], s->cc, s->shift, s->upwind, s->rem, s->ghost, s->inflow,
                             s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) {
    release3v(s);
    return cuda_fail(e, "bgk3v_create");
  }
  *out = s;
  return BGK_OK;
  BGK_GUARD_END
}

bgk_status bgk3v_destroy(bgk3v_solver* s) {
  if (!s) return BGK_OK;
  cudaSetDevice(s->device);
  cudaStreamSynchronize(s->stream);
  release3v(s);
  return BGK_OK;
}

bgk_status bgk3v_get_info(const bgk3v_solver* s, bgk3v_info* out) {
  if (!s || !out) return fail(BGK_ERR_INVALID_ARG, "null argument");
  out->dt = s->P.dt;
  out->dx = s->P.dx;
  out->dv = s->P.dv;
  out->max_courant = s->max_courant;
  out->ncell = s->P.nx;
  out->nv = s->P.nv;
  out->steps_done = s->steps_done;
  out->device_bytes = s->device_bytes;
  return BGK_OK;
}

bgk_status bgk3v_init_step(bgk3v_solver* s, double x_split, const double left[5], const double right[5]) {
  BGK_GUARD_BEGIN
  if (!s || !left || !right) return fail(BGK_ERR_INVALID_ARG, "null argument");
  for (int k = 0; k < 5; ++k)
    if (!std::isfinite(left[k]) || !std::isfinite(right[k])) return fail(BGK_ERR_INVALID_ARG, "non-finite state");
  if (!(left[0] > 0.0) || !(left[4] > 0.0) || !(right[0] > 0.0) || !(right[4] > 0.0))
    return fail(BGK_ERR_INVALID_ARG, "states need n > 0 and theta > 0");
  if (cudaSetDevice(s->device) != cudaSuccess) return fail(BGK_ERR_CUDA, "cudaSetDevice");
  bgk::Inflow3v lr;
  for (int k = 0; k < 5; ++k) {
    lr.s[0][k] = left[k];
    lr.s[1][k] = right[k];
  }
  s->cur = 0;
  s->steps_done = 0;
  cudaError_t e = cudaMemsetAsync(s->err, 0, sizeof(int), s->stream);
  if (e == cudaSuccess) e = bgk::launch_init3v(s->P, s->tables(), x_split, lr, s->f[0], s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "bgk3v_init_step");
  return BGK_OK;
  BGK_GUARD_END
}

bgk_status bgk3v_set_state(bgk3v_solver* s, const double* f, int on_device) {
  if (!s || !f) return fail(BGK_ERR_INVALID_ARG, "null argument");
  if (cudaSetDevice(s->device) != cudaSuccess) return fail(BGK_ERR_CUDA, "cudaSetDevice");
  s->cur = 0;
  s->steps_done = 0;
  cudaError_t e = cudaMemsetAsync(s->err, 0, sizeof(int), s->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->f[0], f, sizeof(double) * s->state_elems(),
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "bgk3v_set_state");
  return BGK_OK;
}

bgk_status bgk3v_get_state(bgk3v_solver* s, double* f, int on_device) {
  if (!s || !f) return fail(BGK_ERR_INVALID_ARG, "null argument");
  if (cudaSetDevice(s->device) != cudaSuccess) return fail(BGK_ERR_CUDA, "cudaSetDevice");
  cudaError_t e = cudaMemcpyAsync(f, s->f[s->cur], sizeof(double) * s->state_elems(),
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "bgk3v_get_state");
  return BGK_OK;
}

bgk_status bgk3v_step(bgk3v_solver* s, int64_t nsteps) {
  if (!s) return fail(BGK_ERR_INVALID_ARG, "null solver");
  if (nsteps < 0) return fail(BGK_ERR_INVALID_ARG, "nsteps must be >= 0");
  if (nsteps == 0) return BGK_OK;
  if (cudaSetDevice(s->device) != cudaSuccess) return fail(BGK_ERR_CUDA, "cudaSetDevice");
  const bgk::Tables3v T = s->tables();
  for (int64_t k = 0; k < nsteps; ++k) {
    const cudaError_t e = bgk::launch_step3v(s->P, T, s->f[s->cur], s->f[s->cur ^ 1], s->mom_step, s->err, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "bgk3v_step");
    s->cur ^= 1;
    ++s->steps_done;
  }
  return BGK_OK;
}

bgk_status bgk3v_moments(bgk3v_solver* s, int which, double* mom, int on_device) {
  if (!s || !mom) return fail(BGK_ERR_INVALID_ARG, "null argument");
  if (which != 0 && which != 1) return fail(BGK_ERR_INVALID_ARG, "which must be 0 or 1");
  if (cudaSetDevice(s->device) != cudaSuccess) return fail(BGK_ERR_CUDA, "cudaSetDevice");
  cudaError_t e = cudaSuccess;
  const double* src = s->mom_step;
  if (which == 0) {
    e = bgk::launch_moments3v(s->P, s->tables(), s->f[s->cur], s->mom_tmp, s->stream);
    src = s->mom_tmp;
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(mom, src, sizeof(double) * s->P.nx * 5,
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "bgk3v_moments");
  return BGK_OK;
}

bgk_status bgk3v_sync(bgk3v_solver* s) {
  if (!s) return fail(BGK_ERR_INVALID_ARG, "null solver");
  if (cudaSetDevice(s->device) != cudaSuccess) return fail(BGK_ERR_CUDA, "cudaSetDevice");
  return check_flag3v(s);
}

}  // extern "C"
