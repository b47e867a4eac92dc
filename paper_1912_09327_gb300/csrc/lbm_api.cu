// C ABI of the LBMTau1 library: context, workspace layout, host transfers and
// the time loop (Algorithm 1 of arXiv:1912.09327, repeated with the two grid
// copies of Section 2.1 swapped after every step).
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "../../include/lbmtau1.h"
#include "lbm_ctx.h"
#include "lbm_step.cuh"

using lbmtau1::Fields;
using lbmtau1::Layout;

namespace {

constexpr int64_t kPitchAlign = 32;           // nodes; rows start 128-B aligned
constexpr size_t kAlign = 256;                // bytes; every workspace region
constexpr int64_t kStagingNodes = 1 << 20;    // host-transfer chunk (nodes)
constexpr int64_t kMaxExtent = (int64_t(1) << 30) - 1;  // rows index in 32 bits

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

bool params_ok(const lbm_params *p) {
  return p && p->nx >= 1 && p->ny >= 1 && p->nx <= kMaxExtent &&
         p->ny <= kMaxExtent &&
         (p->storage == LBM_STORAGE_F32 || p->storage == LBM_STORAGE_F16 ||
          p->storage == LBM_STORAGE_BF16) &&
         (p->rounding == LBM_ROUND_DEFAULT ||
          p->rounding == LBM_ROUND_NEAREST ||
          p->rounding == LBM_ROUND_STOCHASTIC) &&
         isfinite(p->fx) && isfinite(p->fy) && isfinite(p->sc_g) &&
         (p->sc_g == 0.0 || p->storage == LBM_STORAGE_F32);
}

Layout make_layout(const lbm_params *p) {
  Layout L;
  L.pitch = (p->nx + kPitchAlign - 1) / kPitchAlign * kPitchAlign;
  const size_t plane = static_cast<size_t>(L.pitch) * p->ny;
  L.field_bytes =
      align_up(plane * lbmtau1::storage_bytes(p->storage), kAlign);
  L.nblocks = lbmtau1::step_blocks(p->nx, p->ny);
  int64_t rows = kStagingNodes / p->nx;
  if (rows < 1) rows = 1;
  if (rows > p->ny) rows = p->ny;
  L.staging_rows = rows;
  size_t off = 0;
  L.off_fields = off;
  off += 6 * L.field_bytes;
  L.off_mask = off;
  // bulk row copies may read up to 16 bytes past a row's end; pad the plane
  off += align_up(plane + kAlign, kAlign);
  L.off_partials = off;
  off += align_up(static_cast<size_t>(L.nblocks) * lbmtau1::kTileWarps * 3 *
                      sizeof(double),
                  kAlign);
  L.off_clean = off;
  off += align_up(static_cast<size_t>(L.nblocks) * lbmtau1::kTileWarps, kAlign);
  L.off_result = off;
  off += kAlign;
  L.off_staging = off;
  off += align_up(static_cast<size_t>(rows) * p->nx * 3 * sizeof(double),
                  kAlign);
  L.total = off;
  return L;
}

}  // namespace


namespace {

int fail(lbm_ctx *c, int status, const char *fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof c->err, fmt, ap);
    va_end(ap);
  }
  return status;
}

int cuda_fail(lbm_ctx *c, cudaError_t e, const char *what) {
  return fail(c, LBM_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Makes the workspace's device current (callers may run several GPUs).
int bind_device(lbm_ctx *c) {
  cudaPointerAttributes attr;
  cudaError_t e = cudaPointerGetAttributes(&attr, c->base);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaPointerGetAttributes");
  if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
    return fail(c, LBM_E_WORKSPACE, "workspace is not device memory");
  int cur = -1;
  e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaGetDevice");
  if (cur != attr.device) {
    e = cudaSetDevice(attr.device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  }
  return LBM_OK;
}

int apply_solid_storage(lbm_ctx *c, int copy) {
  const int64_t n = c->L.pitch * c->p.ny;
  cudaError_t e = lbmtau1::launch_solid_storage(
      c->p.storage, c->f[copy], c->mask, n, static_cast<float>(c->p.fx),
      static_cast<float>(c->p.fy), c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "solid storage kernel");
  return LBM_OK;
}

int reset_flags(lbm_ctx *c) {
  cudaError_t e = cudaMemsetAsync(c->result, 0, kAlign, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemsetAsync(result)");
  c->has_residual = false;
  return LBM_OK;
}

}  // namespace

extern "C" {

size_t lbm_workspace_bytes(const lbm_params *p) {
  if (!params_ok(p)) return 0;
  return make_layout(p).total;
}

int lbm_create(const lbm_params *p, void *dev_workspace, size_t workspace_bytes,
               void *cuda_stream, lbm_ctx **out) {
  if (!out) return LBM_E_INVAL;
  *out = nullptr;
  if (!params_ok(p)) return LBM_E_INVAL;
  const Layout L = make_layout(p);
  if (!dev_workspace || reinterpret_cast<uintptr_t>(dev_workspace) % kAlign ||
      workspace_bytes < L.total)
    return LBM_E_WORKSPACE;
  lbm_ctx *c = new (std::nothrow) lbm_ctx();
  if (!c) return LBM_E_INVAL;
  c->p = *p;
  c->L = L;
  c->base = static_cast<char *>(dev_workspace);
  for (int k = 0; k < 2; ++k) {
    char *q = c->base + L.off_fields + 3 * k * L.field_bytes;
    c->f[k].d = reinterpret_cast<float *>(q);
    c->f[k].jx = reinterpret_cast<float *>(q + L.field_bytes);
    c->f[k].jy = reinterpret_cast<float *>(q + 2 * L.field_bytes);
  }
  c->mask = reinterpret_cast<uint8_t *>(c->base + L.off_mask);
  c->partials = reinterpret_cast<double *>(c->base + L.off_partials);
  c->result = reinterpret_cast<double *>(c->base + L.off_result);
  c->clean = reinterpret_cast<uint8_t *>(c->base + L.off_clean);
  c->clean_variant = -1;
  c->flag = reinterpret_cast<unsigned *>(c->result + 3);
  c->staging = reinterpret_cast<double *>(c->base + L.off_staging);
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  c->cur = 0;
  c->variant = -1;
  c->steps = 0;
  c->graph[0] = c->graph[1] = nullptr;
  c->graph_variant[0] = c->graph_variant[1] = -1;
  c->graphs_off = cuda_stream == nullptr || c->stream == cudaStreamLegacy ||
                  c->stream == cudaStreamPerThread;
  c->wait_ns = 1000000000ull;
  c->has_geometry = false;
  c->has_residual = false;
  c->n_fluid = 0;
  c->err[0] = '\0';
  *out = c;
  return LBM_OK;
}

int lbm_set_geometry(lbm_ctx *c, const uint8_t *host_mask) {
  if (!c) return LBM_E_INVAL;
  if (!host_mask) return fail(c, LBM_E_INVAL, "host_mask is NULL");
  const int64_t n = c->p.nx * c->p.ny;
  int64_t fluid = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (host_mask[i] > LBM_FIXED)
      return fail(c, LBM_E_INVAL, "node %lld has type %d (allowed 0, 1, 2)",
                  static_cast<long long>(i), host_mask[i]);
    fluid += host_mask[i] == LBM_FLUID;
  }
  int st = bind_device(c);
  if (st) return st;
  const size_t plane = static_cast<size_t>(c->L.pitch) * c->p.ny;
  cudaError_t e = cudaMemsetAsync(c->mask, LBM_SOLID, plane, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemsetAsync(mask)");
  e = cudaMemcpy2DAsync(c->mask, c->L.pitch, host_mask, c->p.nx, c->p.nx,
                        c->p.ny, cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpy2DAsync(mask)");
  // rest state rho = 1 (delta = 0), j = 0 in both copies
  e = cudaMemsetAsync(c->base + c->L.off_fields, 0, 6 * c->L.field_bytes,
                      c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemsetAsync(fields)");
  for (int k = 0; k < 2; ++k) {
    st = apply_solid_storage(c, k);
    if (st) return st;
  }
  st = reset_flags(c);
  if (st) return st;
  // the host mask may be released as soon as this call returns
  e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize");
  c->cur = 0;
  c->n_fluid = fluid;
  c->clean_variant = -1;  // new node types: flags computed again
  c->has_geometry = true;
  c->err[0] = '\0';
  return LBM_OK;
}

int lbm_set_moments(lbm_ctx *c, const double *rho, const double *jx,
                    const double *jy) {
  if (!c) return LBM_E_INVAL;
  if (!rho || !jx || !jy) return fail(c, LBM_E_INVAL, "null moment array");
  if (!c->has_geometry)
    return fail(c, LBM_E_STATE, "lbm_set_geometry has not been called");
  int st = bind_device(c);
  if (st) return st;
  const int64_t nx = c->p.nx;
  for (int64_t y0 = 0; y0 < c->p.ny; y0 += c->L.staging_rows) {
    const int64_t rows =
        y0 + c->L.staging_rows <= c->p.ny ? c->L.staging_rows : c->p.ny - y0;
    const size_t n = static_cast<size_t>(rows) * nx;
    const double *src[3] = {rho, jx, jy};
    for (int k = 0; k < 3; ++k) {
      cudaError_t e = cudaMemcpyAsync(c->staging + k * n, src[k] + y0 * nx,
                                      n * sizeof(double),
                                      cudaMemcpyHostToDevice, c->stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpyAsync(H2D)");
    }
    cudaError_t e = lbmtau1::launch_pack(c->p.storage, c->staging,
                                         c->f[c->cur], nx, c->L.pitch, y0,
                                         rows, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "pack kernel");
  }
  st = apply_solid_storage(c, c->cur);
  if (st) return st;
  st = reset_flags(c);
  if (st) return st;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize");
  c->err[0] = '\0';
  return LBM_OK;
}

int lbm_set_state(lbm_ctx *c, const void *drho, const void *jx,
                  const void *jy) {
  if (!c) return LBM_E_INVAL;
  if (!drho || !jx || !jy) return fail(c, LBM_E_INVAL, "null state array");
  if (!c->has_geometry)
    return fail(c, LBM_E_STATE, "lbm_set_geometry has not been called");
  int st = bind_device(c);
  if (st) return st;
  const void *src[3] = {drho, jx, jy};
  void *dst[3] = {c->f[c->cur].d, c->f[c->cur].jx, c->f[c->cur].jy};
  const size_t es = lbmtau1::storage_bytes(c->p.storage);
  const size_t row = static_cast<size_t>(c->p.nx) * es;
  for (int k = 0; k < 3; ++k) {
    cudaError_t e = cudaMemcpy2DAsync(dst[k], c->L.pitch * es,
                                      src[k], row, row, c->p.ny,
                                      cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpy2DAsync(H2D)");
  }
  st = apply_solid_storage(c, c->cur);
  if (st) return st;
  st = reset_flags(c);
  if (st) return st;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize");
  c->err[0] = '\0';
  return LBM_OK;
}

int lbm_get_state(lbm_ctx *c, void *drho, void *jx, void *jy) {
  if (!c) return LBM_E_INVAL;
  if (!drho || !jx || !jy) return fail(c, LBM_E_INVAL, "null state array");
  if (!c->has_geometry)
    return fail(c, LBM_E_STATE, "lbm_set_geometry has not been called");
  int st = bind_device(c);
  if (st) return st;
  void *dst[3] = {drho, jx, jy};
  const void *src[3] = {c->f[c->cur].d, c->f[c->cur].jx, c->f[c->cur].jy};
  const size_t es = lbmtau1::storage_bytes(c->p.storage);
  const size_t row = static_cast<size_t>(c->p.nx) * es;
  for (int k = 0; k < 3; ++k) {
    cudaError_t e = cudaMemcpy2DAsync(dst[k], row, src[k], c->L.pitch * es,
                                      row,
                                      c->p.ny, cudaMemcpyDeviceToHost,
                                      c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpy2DAsync(D2H)");
  }
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize");
  c->err[0] = '\0';
  return LBM_OK;
}

namespace {

// Picks the context's tile variant (first step): the model's choice, or its
// twin with the clean-tile code when the grid is large and at least 3/4 of
// the warp tiles are clean (the flags are read to the host once).
int select_variant(lbm_ctx *c) {
  int v = lbmtau1::choose_variant(c->p.nx, c->p.ny, c->p.storage);
  const int d = lbmtau1::dual_variant(v, c->p.nx, c->p.ny);
  if (d >= 0) {
    // the dual kernel when at least 3/4 of the warp tiles are clean (its
    // flags are v's: same tiles); one read of the flags to the host
    cudaError_t e = lbmtau1::launch_tile_flags(d, c->mask, c->p.nx, c->p.ny,
                                               c->L.pitch, c->clean,
                                               c->stream);
    const int64_t n = lbmtau1::launched_blocks(c->p.nx, c->p.ny, d) *
                      lbmtau1::kTileWarps;
    std::vector<uint8_t> h(static_cast<size_t>(n));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h.data(), c->clean, h.size(),
                          cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "tile flags");
    int64_t clean = 0;
    for (uint8_t f : h) clean += f;
    if (4 * clean >= 3 * n) v = d;
    c->clean_variant = v;  // same tiles either way
  }
  c->variant = v;
  return LBM_OK;
}

constexpr int64_t kGraphChunk = 16;  // steps per captured graph (even)

// kGraphChunk unreduced steps from the current copy as one graph launch
// (the copy holding the state is the same afterwards).  Falls back to direct
// launches when the stream cannot be captured or is being captured already.
int step_chunk(lbm_ctx *c, lbmtau1::StepLaunch a) {
  const int p = c->cur;
  auto direct = [&]() -> int {
    for (int64_t t = 0; t < kGraphChunk; ++t) {
      a.src = c->f[(p + t) & 1];
      a.dst = c->f[(p + t + 1) & 1];
      cudaError_t e = lbmtau1::launch_step(a, false, c->stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "step kernel launch");
    }
    return LBM_OK;
  };
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (c->graphs_off || cudaStreamIsCapturing(c->stream, &cs) != cudaSuccess ||
      cs != cudaStreamCaptureStatusNone) {
    (void)cudaGetLastError();
    return direct();
  }
  if (!c->graph[p] || c->graph_variant[p] != c->variant) {
    if (c->graph[p]) cudaGraphExecDestroy(c->graph[p]);
    c->graph[p] = nullptr;
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) !=
        cudaSuccess) {
      (void)cudaGetLastError();
      c->graphs_off = true;
      return direct();
    }
    cudaError_t le = cudaSuccess;
    for (int64_t t = 0; t < kGraphChunk && le == cudaSuccess; ++t) {
      a.src = c->f[(p + t) & 1];
      a.dst = c->f[(p + t + 1) & 1];
      le = lbmtau1::launch_step(a, false, c->stream);
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (le != cudaSuccess || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda_fail(c, le != cudaSuccess ? le : e, "step graph capture");
    }
    e = cudaGraphInstantiate(&c->graph[p], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      c->graph[p] = nullptr;
      return cuda_fail(c, e, "cudaGraphInstantiate");
    }
    c->graph_variant[p] = c->variant;
  }
  cudaError_t e = cudaGraphLaunch(c->graph[p], c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphLaunch");
  return LBM_OK;
}

}  // namespace

int lbm_step(lbm_ctx *c, int64_t nsteps) {
  if (!c) return LBM_E_INVAL;
  if (nsteps < 0) return fail(c, LBM_E_INVAL, "nsteps < 0");
  if (!c->has_geometry)
    return fail(c, LBM_E_STATE, "lbm_set_geometry has not been called");
  if (nsteps == 0) return LBM_OK;
  lbmtau1::StepLaunch a;
  a.mask = c->mask;
  a.nx = c->p.nx;
  a.ny = c->p.ny;
  a.pitch = c->L.pitch;
  a.periodic_x = c->p.periodic_x != 0;
  a.periodic_y = c->p.periodic_y != 0;
  a.fx = static_cast<float>(c->p.fx);
  a.fy = static_cast<float>(c->p.fy);
  a.g_sc = static_cast<float>(c->p.sc_g);
  a.partials = c->partials;
  a.flag = c->flag;
  a.storage = c->p.storage;
  if (c->variant < 0) {
    const int st = select_variant(c);
    if (st) return st;
  }
  a.variant = c->variant;
  if (c->clean_variant != c->variant) {
    cudaError_t e = lbmtau1::launch_tile_flags(c->variant, c->mask, c->p.nx,
                                               c->p.ny, c->L.pitch, c->clean,
                                               c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "tile flags kernel launch");
    c->clean_variant = c->variant;
  }
  a.clean = c->clean;
  a.wait_ns = c->wait_ns;
  a.sr = lbmtau1::stochastic_rounding(c->p.storage, c->p.rounding);
  // Steps 1 .. nsteps - 2 go in captured graph chunks when the rounding
  // draws no per-step random bits (the graph replays fixed launch arguments);
  // the first step of each call (any one-time kernel set-up stays outside a
  // capture) and the reduced last step are launched directly.
  const bool graphs = !a.sr;
  for (int64_t s = 0; s < nsteps;) {
    if (graphs && s >= 1 && nsteps - 1 - s >= kGraphChunk) {
      const int st = step_chunk(c, a);
      if (st) return st;
      s += kGraphChunk;
      continue;
    }
    a.src = c->f[c->cur];
    a.dst = c->f[1 - c->cur];
    a.step = static_cast<uint32_t>(c->steps + s);
    cudaError_t e = lbmtau1::launch_step(a, s == nsteps - 1, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "step kernel launch");
    c->cur = 1 - c->cur;
    ++s;
  }
  cudaError_t e = lbmtau1::launch_finalize(
      c->partials, lbmtau1::launched_blocks(c->p.nx, c->p.ny, c->variant),
      c->result, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "finalize kernel launch");
  c->has_residual = true;
  c->steps += nsteps;
  return LBM_OK;
}

int lbm_step_count(const lbm_ctx *c, int64_t *steps) {
  if (!c || !steps) return LBM_E_INVAL;
  *steps = c->steps;
  return LBM_OK;
}

int lbm_set_step_count(lbm_ctx *c, int64_t steps) {
  if (!c) return LBM_E_INVAL;
  if (steps < 0) return fail(c, LBM_E_INVAL, "steps < 0");
  c->steps = steps;
  return LBM_OK;
}

int lbm_set_variant(lbm_ctx *c, int32_t variant) {
  if (!c) return LBM_E_INVAL;
  if (variant < -1 || variant >= lbmtau1::variant_count())
    return fail(c, LBM_E_INVAL, "variant %d out of range", int(variant));
  c->variant = variant;
  return LBM_OK;
}

int lbm_set_copy_wait_ns(lbm_ctx *c, int64_t ns) {
  if (!c) return LBM_E_INVAL;
  if (ns < 0 || ns > 1000000000ll)
    return fail(c, LBM_E_INVAL, "copy wait limit %lld ns out of range",
                static_cast<long long>(ns));
  c->wait_ns = static_cast<unsigned long long>(ns);
  // captured graphs hold the old limit in their launch arguments
  c->graph_variant[0] = c->graph_variant[1] = -1;
  return LBM_OK;
}

int32_t lbm_variant(lbm_ctx *c) {
  if (!c) return -1;
  if (c->variant < 0) {
    // before the node types are known only the model's choice (not kept)
    if (!c->has_geometry)
      return lbmtau1::choose_variant(c->p.nx, c->p.ny, c->p.storage);
    if (select_variant(c) != LBM_OK) return -1;
  }
  return c->variant;
}

int lbm_moments(lbm_ctx *c, double *rho, double *jx, double *jy) {
  if (!c) return LBM_E_INVAL;
  if (!rho || !jx || !jy) return fail(c, LBM_E_INVAL, "null moment array");
  if (!c->has_geometry)
    return fail(c, LBM_E_STATE, "lbm_set_geometry has not been called");
  int st = bind_device(c);
  if (st) return st;
  const int64_t nx = c->p.nx;
  for (int64_t y0 = 0; y0 < c->p.ny; y0 += c->L.staging_rows) {
    const int64_t rows =
        y0 + c->L.staging_rows <= c->p.ny ? c->L.staging_rows : c->p.ny - y0;
    const size_t n = static_cast<size_t>(rows) * nx;
    cudaError_t e = lbmtau1::launch_unpack(c->p.storage, c->f[c->cur],
                                           c->mask, c->staging, nx, c->L.pitch,
                                           y0, rows, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "unpack kernel");
    double *dst[3] = {rho, jx, jy};
    for (int k = 0; k < 3; ++k) {
      e = cudaMemcpyAsync(dst[k] + y0 * nx, c->staging + k * n,
                          n * sizeof(double), cudaMemcpyDeviceToHost,
                          c->stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpyAsync(D2H)");
    }
  }
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize");
  c->err[0] = '\0';
  return LBM_OK;
}

size_t lbm_snapshot_bytes(const lbm_params *p) {
  if (!params_ok(p)) return 0;
  return 3 * make_layout(p).field_bytes;
}

int lbm_snapshot(lbm_ctx *c, void *dev_buf, size_t bytes) {
  if (!c) return LBM_E_INVAL;
  if (!dev_buf || reinterpret_cast<uintptr_t>(dev_buf) % kAlign ||
      bytes < 3 * c->L.field_bytes)
    return fail(c, LBM_E_INVAL, "snapshot buffer missing, misaligned or small");
  if (!c->has_geometry)
    return fail(c, LBM_E_STATE, "lbm_set_geometry has not been called");
  int st = bind_device(c);
  if (st) return st;
  // the three planes of the current copy are contiguous in the workspace
  cudaError_t e = cudaMemcpyAsync(dev_buf, c->f[c->cur].d,
                                  3 * c->L.field_bytes,
                                  cudaMemcpyDeviceToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpyAsync(snapshot)");
  c->err[0] = '\0';
  return LBM_OK;
}

int lbm_change_since(lbm_ctx *c, const void *dev_buf, int64_t steps,
                     double *change) {
  if (!c) return LBM_E_INVAL;
  if (!dev_buf || reinterpret_cast<uintptr_t>(dev_buf) % kAlign || steps < 1 ||
      !change)
    return fail(c, LBM_E_INVAL, "bad snapshot buffer, step count or output");
  if (!c->has_geometry)
    return fail(c, LBM_E_STATE, "lbm_set_geometry has not been called");
  int st = bind_device(c);
  if (st) return st;
  const char *b = static_cast<const char *>(dev_buf);
  lbmtau1::Fields snap;
  snap.d = const_cast<char *>(b);
  snap.jx = const_cast<char *>(b + c->L.field_bytes);
  snap.jy = const_cast<char *>(b + 2 * c->L.field_bytes);
  // the reduction partials of the step serve as scratch (the step's own
  // result slot is not touched); one block of four warps per partial block
  int64_t blocks = (c->p.nx * c->p.ny + 127) / 128;
  if (blocks > c->L.nblocks) blocks = c->L.nblocks;
  if (blocks > 4096) blocks = 4096;
  double *out = c->result + 4;
  cudaError_t e = lbmtau1::launch_change(c->p.storage, c->f[c->cur], snap,
                                         c->mask, c->p.nx, c->p.ny,
                                         c->L.pitch, c->partials, blocks,
                                         c->stream);
  if (e == cudaSuccess)
    e = lbmtau1::launch_finalize(c->partials, blocks, out, c->stream);
  double h[3];
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h, out, sizeof h, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "change reduction");
  const double rel = h[1] > 0.0 ? sqrt(h[0] / h[1]) : sqrt(h[0]);
  *change = rel / static_cast<double>(steps);
  c->err[0] = '\0';
  return LBM_OK;
}

int lbm_residual(lbm_ctx *c, double *residual, double *mass) {
  if (!c) return LBM_E_INVAL;
  if (!c->has_residual)
    return fail(c, LBM_E_STATE, "no step has run since the state was set");
  int st = bind_device(c);
  if (st) return st;
  double h[4];
  cudaError_t e = cudaMemcpyAsync(h, c->result, sizeof h,
                                  cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpyAsync(result)");
  e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize");
  unsigned flag;
  memcpy(&flag, &h[3], sizeof flag);
  if (flag & 2u)
    return fail(c, LBM_E_CUDA,
                "a step's bulk row copy did not complete within the wait "
                "limit (%llu ns)", c->wait_ns);
  const double num = h[0], den = h[1];
  if (residual) *residual = den > 0.0 ? sqrt(num / den) : sqrt(num);
  if (mass) *mass = static_cast<double>(c->n_fluid) + h[2];
  if (flag & 1u)
    return fail(c, LBM_E_UNSTABLE,
                "a step produced rho <= 0 or a non-finite moment");
  c->err[0] = '\0';
  return LBM_OK;
}

void lbm_destroy(lbm_ctx *c) {
  if (!c) return;
  for (cudaGraphExec_t g : c->graph)
    if (g) cudaGraphExecDestroy(g);
  delete c;
}

const char *lbm_last_error(const lbm_ctx *c) {
  return c ? c->err : "null context";
}

const char *lbm_status_string(int status) {
  switch (status) {
    case LBM_OK: return "LBM_OK";
    case LBM_E_INVAL: return "LBM_E_INVAL";
    case LBM_E_WORKSPACE: return "LBM_E_WORKSPACE";
    case LBM_E_CUDA: return "LBM_E_CUDA";
    case LBM_E_UNSTABLE: return "LBM_E_UNSTABLE";
    case LBM_E_STATE: return "LBM_E_STATE";
    default: return "LBM_E_UNKNOWN";
  }
}

}  // extern "C"
