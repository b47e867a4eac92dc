// Batched stepping of many independent LBMTau1 domains (each an lbm_ctx) with
// one launch per time step for the whole batch.
//
// Every member keeps its own workspace (fields, node types, reduction
// partials); the batch holds a device table of member descriptors and a work
// list of block tiles (member, tile x, tile y).  A persistent grid walks the
// list through an atomic counter, so small and large domains share the GPU in
// one launch instead of one under-filled launch per domain.  Runs of steps
// between the first and the last step of a call are replayed from a CUDA
// graph of kChunk steps.  Each tile runs the same code as the single-domain
// kernel, so a member's state is bit for bit the one it would reach alone.
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

using lbmtau1::BatchLaunch;
using lbmtau1::BatchMember;

namespace {

constexpr int kChunk = 16;  // steps per captured graph (even)
constexpr size_t kAlign = 256;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct BatchLayout {
  size_t off_members = 0, off_items = 0, off_nitems = 0, off_counters = 0;
  size_t off_gather = 0;
  size_t total = 0;
};

BatchLayout batch_layout(int32_t capacity, int64_t max_tiles) {
  BatchLayout L;
  size_t off = 0;
  L.off_members = off;
  off += align_up(sizeof(BatchMember) * static_cast<size_t>(capacity), kAlign);
  L.off_items = off;
  off += align_up(sizeof(int4) * static_cast<size_t>(max_tiles) *
                      lbmtau1::kTileWarps,
                  kAlign);
  L.off_nitems = off;
  off += kAlign;
  L.off_counters = off;
  off += align_up(sizeof(unsigned) * (kChunk + 3), kAlign);
  L.off_gather = off;
  off += align_up(sizeof(double) * 4 * static_cast<size_t>(capacity), kAlign);
  L.total = off;
  return L;
}

}  // namespace

struct lbm_batch {
  int32_t capacity;
  int64_t max_tiles;
  BatchMember *d_members;
  int4 *d_items;
  int *d_nitems;
  unsigned *d_counters;  // [0, kChunk) graph steps, [kChunk] direct steps,
                         // [kChunk + 1] batch clock, [kChunk + 2] done count
  uint32_t clock;        // host mirror of the batch clock
  bool clock_set;        // device clock and done count zeroed
  double *d_gather;      // 4 doubles per member: result sums and flag
  cudaStream_t stream;
  std::vector<lbm_ctx *> slots;
  std::vector<BatchMember> h_members;
  std::vector<int4> h_items;
  std::vector<lbm_ctx *> packed;  // members in descriptor order
  int nitems;
  int variant;
  int storage;  // storage format of the members (-1 while empty)
  bool items_dirty;
  cudaGraphExec_t graph;
  int graph_variant;
  bool graphs_off;  // the stream cannot be captured: direct launches only
  char err[256];
};

namespace {

int bfail(lbm_batch *b, int status, const char *fmt, ...) {
  if (b) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b->err, sizeof b->err, fmt, ap);
    va_end(ap);
  }
  return status;
}

int bcuda(lbm_batch *b, cudaError_t e, const char *what) {
  return bfail(b, LBM_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

void drop_graph(lbm_batch *b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  b->graph_variant = -1;
}

// Refreshes the member table (every call: a member may have been stepped on
// its own since) and, when membership or the variant changed, the work list.
int upload(lbm_batch *b) {
  b->packed.clear();
  for (lbm_ctx *c : b->slots)
    if (c) b->packed.push_back(c);
  const int n = static_cast<int>(b->packed.size());
  int64_t tx = 0, ty = 0;
  lbmtau1::variant_tile(b->variant, &tx, &ty);
  b->h_members.resize(n);
  // A kernel with the clean-tile code takes the work list ordered by tile
  // kind (below), which depends on the flags.
  const bool by_kind = lbmtau1::variant_has_clean_code(b->variant);
  bool flags_changed = false;
  for (int i = 0; i < n; ++i) {
    lbm_ctx *c = b->packed[i];
    BatchMember &m = b->h_members[i];
    m.f[0] = c->f[0];
    m.f[1] = c->f[1];
    m.mask = c->mask;
    m.nx = c->p.nx;
    m.ny = c->p.ny;
    m.pitch = c->L.pitch;
    m.periodic_x = c->p.periodic_x != 0;
    m.periodic_y = c->p.periodic_y != 0;
    m.fx = static_cast<float>(c->p.fx);
    m.fy = static_cast<float>(c->p.fy);
    m.partials = c->partials;
    m.result = c->result;
    m.flag = c->flag;
    m.gx = (c->p.nx + tx - 1) / tx;
    m.nblocks = m.gx * ((c->p.ny + ty - 1) / ty);
    m.cur = c->cur;
    m.sr = lbmtau1::stochastic_rounding(c->p.storage, c->p.rounding);
    m.step_base = c->steps - static_cast<int64_t>(b->clock);
    if (c->clean_variant != b->variant) {  // clean-tile flags for our tiles
      cudaError_t e = lbmtau1::launch_tile_flags(
          b->variant, c->mask, c->p.nx, c->p.ny, c->L.pitch, c->clean,
          b->stream);
      if (e != cudaSuccess) return bcuda(b, e, "tile flags kernel launch");
      c->clean_variant = b->variant;
      flags_changed = true;
    }
    m.clean = c->clean;
  }
  if (by_kind && flags_changed) b->items_dirty = true;
  if (b->items_dirty) {
    b->h_items.clear();
    // With the clean-tile code in the kernel, the warp tiles that take the
    // general code come first and the clean ones after them: warps running
    // the two code paths side by side on an SM stall on instruction fetch
    // (ncu on the 512-domain mix: 2.4 no-instruction stalls per issue mixed,
    // 0.65 with the general kernel alone).  The flags are read to the host
    // once per rebuild of the list.
    std::vector<std::vector<uint8_t>> flags(by_kind ? n : 0);
    if (by_kind) {
      for (int i = 0; i < n; ++i) {
        flags[i].resize(static_cast<size_t>(b->h_members[i].nblocks) *
                        lbmtau1::kTileWarps);
        cudaError_t e = cudaMemcpyAsync(flags[i].data(), b->packed[i]->clean,
                                        flags[i].size(),
                                        cudaMemcpyDeviceToHost, b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "cudaMemcpyAsync(flags)");
      }
      cudaError_t e = cudaStreamSynchronize(b->stream);
      if (e != cudaSuccess) return bcuda(b, e, "cudaStreamSynchronize(flags)");
    }
    for (int pass = 0; pass < (by_kind ? 2 : 1); ++pass) {
      for (int i = 0; i < n; ++i) {
        const BatchMember &m = b->h_members[i];
        const int64_t gy = m.nblocks / m.gx;
        // every warp tile of every block tile (vertical neighbours next to
        // each other, for the rows they share)
        for (int64_t by = 0; by < gy; ++by)
          for (int64_t bx = 0; bx < m.gx; ++bx)
            for (int w = 0; w < lbmtau1::kTileWarps; ++w) {
              if (by_kind &&
                  (flags[i][(by * m.gx + bx) * lbmtau1::kTileWarps + w] != 0) !=
                      (pass == 1))
                continue;
              b->h_items.push_back(make_int4(i, static_cast<int>(bx),
                                             static_cast<int>(by), w));
            }
      }
    }
    const int64_t tiles =
        static_cast<int64_t>(b->h_items.size()) / lbmtau1::kTileWarps;
    if (tiles > b->max_tiles)
      return bfail(b, LBM_E_WORKSPACE,
                   "batch needs %lld tiles, its workspace holds %lld",
                   static_cast<long long>(tiles),
                   static_cast<long long>(b->max_tiles));
    b->nitems = static_cast<int>(b->h_items.size());
    if (b->nitems) {
      cudaError_t e = cudaMemcpyAsync(b->d_items, b->h_items.data(),
                                      sizeof(int4) * b->nitems,
                                      cudaMemcpyHostToDevice, b->stream);
      if (e != cudaSuccess) return bcuda(b, e, "cudaMemcpyAsync(items)");
    }
    cudaError_t e = cudaMemcpyAsync(b->d_nitems, &b->nitems, sizeof(int),
                                    cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "cudaMemcpyAsync(nitems)");
    b->items_dirty = false;
  }
  if (n) {
    cudaError_t e = cudaMemcpyAsync(b->d_members, b->h_members.data(),
                                    sizeof(BatchMember) * n,
                                    cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "cudaMemcpyAsync(members)");
  }
  return LBM_OK;
}

BatchLaunch launch_args(lbm_batch *b, unsigned *counter, int parity) {
  BatchLaunch L;
  L.members = b->d_members;
  L.items = b->d_items;
  L.nitems = b->d_nitems;
  L.counter = counter;
  L.parity = parity;
  L.storage = b->storage;
  L.clock = b->d_counters + kChunk + 1;
  L.done = b->d_counters + kChunk + 2;
  return L;
}

int direct_step(lbm_batch *b, int parity, bool reduce) {
  unsigned *counter = b->d_counters + kChunk;
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "cudaMemsetAsync(counter)");
  e = lbmtau1::launch_batch(b->variant, launch_args(b, counter, parity),
                            reduce, b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "batch kernel launch");
  return LBM_OK;
}

// kChunk unreduced steps starting at an even parity, as one graph (or as
// direct launches when the stream cannot be captured, e.g. the legacy
// default stream).
int graph_chunk(lbm_batch *b) {
  if (b->graphs_off) {
    for (int t = 0; t < kChunk; ++t) {
      int st = direct_step(b, t & 1, false);
      if (st) return st;
    }
    return LBM_OK;
  }
  if (!b->graph || b->graph_variant != b->variant) {
    drop_graph(b);
    cudaGraph_t g = nullptr;
    cudaError_t e =
        cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();  // not sticky: clear it, launch directly
      b->graphs_off = true;
      return graph_chunk(b);
    }
    cudaError_t le = cudaMemsetAsync(b->d_counters, 0,
                                     sizeof(unsigned) * kChunk, b->stream);
    for (int t = 0; t < kChunk && le == cudaSuccess; ++t)
      le = lbmtau1::launch_batch(b->variant,
                                 launch_args(b, b->d_counters + t, t & 1),
                                 false, b->stream);
    e = cudaStreamEndCapture(b->stream, &g);
    if (le != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return bcuda(b, le, "graph capture");
    }
    if (e != cudaSuccess) return bcuda(b, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      b->graph = nullptr;
      return bcuda(b, e, "cudaGraphInstantiate");
    }
    b->graph_variant = b->variant;
  }
  cudaError_t e = cudaGraphLaunch(b->graph, b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "cudaGraphLaunch");
  return LBM_OK;
}

}  // namespace

extern "C" {

size_t lbm_batch_workspace_bytes(int32_t capacity, int64_t max_tiles) {
  if (capacity < 1 || max_tiles < 1 || max_tiles > (int64_t(1) << 29) - 1)
    return 0;
  return batch_layout(capacity, max_tiles).total;
}

int32_t lbm_variant_count(void) { return lbmtau1::variant_count(); }

int lbm_variant_tile(int32_t variant, int64_t *tile_x, int64_t *tile_y,
                     int32_t *cols_per_lane) {
  if (variant < 0 || variant >= lbmtau1::variant_count() || !tile_x ||
      !tile_y)
    return LBM_E_INVAL;
  lbmtau1::variant_tile(variant, tile_x, tile_y);
  if (cols_per_lane)
    *cols_per_lane = static_cast<int32_t>(*tile_x / 30);
  return LBM_OK;
}

int32_t lbm_variant_has_clean_code(int32_t variant) {
  if (variant < 0 || variant >= lbmtau1::variant_count()) return -1;
  return lbmtau1::variant_has_clean_code(variant) ? 1 : 0;
}

int64_t lbm_tile_count(int64_t nx, int64_t ny, int32_t variant) {
  if (nx < 1 || ny < 1 || variant < -1 || variant >= lbmtau1::variant_count())
    return -1;
  if (variant < 0) return lbmtau1::step_blocks(nx, ny);
  int64_t tx = 0, ty = 0;
  lbmtau1::variant_tile(variant, &tx, &ty);
  return ((nx + tx - 1) / tx) * ((ny + ty - 1) / ty);
}

int lbm_batch_create(int32_t capacity, int64_t max_tiles, void *dev_workspace,
                     size_t workspace_bytes, void *cuda_stream,
                     lbm_batch **out) {
  if (!out) return LBM_E_INVAL;
  *out = nullptr;
  const size_t need = lbm_batch_workspace_bytes(capacity, max_tiles);
  if (need == 0) return LBM_E_INVAL;
  if (!dev_workspace || reinterpret_cast<uintptr_t>(dev_workspace) % kAlign ||
      workspace_bytes < need)
    return LBM_E_WORKSPACE;
  lbm_batch *b = new (std::nothrow) lbm_batch();
  if (!b) return LBM_E_INVAL;
  const BatchLayout L = batch_layout(capacity, max_tiles);
  char *base = static_cast<char *>(dev_workspace);
  b->capacity = capacity;
  b->max_tiles = max_tiles;
  b->d_members = reinterpret_cast<BatchMember *>(base + L.off_members);
  b->d_items = reinterpret_cast<int4 *>(base + L.off_items);
  b->d_nitems = reinterpret_cast<int *>(base + L.off_nitems);
  b->d_counters = reinterpret_cast<unsigned *>(base + L.off_counters);
  b->d_gather = reinterpret_cast<double *>(base + L.off_gather);
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  b->clock = 0;
  b->clock_set = false;
  b->slots.assign(capacity, nullptr);
  b->nitems = 0;
  b->storage = -1;
  b->variant = lbmtau1::default_variant();
  b->items_dirty = true;
  b->graph = nullptr;
  b->graph_variant = -1;
  b->graphs_off = cuda_stream == nullptr || b->stream == cudaStreamLegacy ||
                  b->stream == cudaStreamPerThread;
  b->err[0] = '\0';
  *out = b;
  return LBM_OK;
}

int lbm_batch_add(lbm_batch *b, lbm_ctx *ctx, int32_t *slot) {
  if (!b) return LBM_E_INVAL;
  if (!ctx) return bfail(b, LBM_E_INVAL, "null context");
  if (ctx->stream != b->stream)
    return bfail(b, LBM_E_INVAL, "member must use the batch's stream");
  if (!ctx->has_geometry)
    return bfail(b, LBM_E_STATE, "member has no geometry");
  if (ctx->p.sc_g != 0.0)
    return bfail(b, LBM_E_INVAL, "multiphase domains are stepped alone");
  if (lbm_batch_members(b) > 0 && ctx->p.storage != b->storage)
    return bfail(b, LBM_E_INVAL, "members must share one storage format");
  for (lbm_ctx *c : b->slots)
    if (c == ctx) return bfail(b, LBM_E_INVAL, "context already a member");
  for (int32_t i = 0; i < b->capacity; ++i)
    if (!b->slots[i]) {
      b->slots[i] = ctx;
      b->storage = ctx->p.storage;
      b->items_dirty = true;
      if (slot) *slot = i;
      b->err[0] = '\0';
      return LBM_OK;
    }
  return bfail(b, LBM_E_WORKSPACE, "batch is full (%d members)", b->capacity);
}

int lbm_batch_remove(lbm_batch *b, int32_t slot) {
  if (!b) return LBM_E_INVAL;
  if (slot < 0 || slot >= b->capacity || !b->slots[slot])
    return bfail(b, LBM_E_INVAL, "no member in slot %d", slot);
  b->slots[slot] = nullptr;
  b->items_dirty = true;
  b->err[0] = '\0';
  return LBM_OK;
}

int32_t lbm_batch_members(const lbm_batch *b) {
  if (!b) return 0;
  int32_t n = 0;
  for (lbm_ctx *c : b->slots) n += c != nullptr;
  return n;
}

int lbm_batch_set_variant(lbm_batch *b, int32_t variant) {
  if (!b) return LBM_E_INVAL;
  if (variant < 0 || variant >= lbmtau1::variant_count())
    return bfail(b, LBM_E_INVAL, "no tile variant %d", variant);
  if (variant != b->variant) {
    b->variant = variant;
    b->items_dirty = true;
  }
  return LBM_OK;
}

int32_t lbm_batch_variant(const lbm_batch *b) { return b ? b->variant : -1; }

int lbm_batch_step(lbm_batch *b, int64_t nsteps) {
  if (!b) return LBM_E_INVAL;
  if (nsteps < 0) return bfail(b, LBM_E_INVAL, "nsteps < 0");
  if (nsteps == 0 || lbm_batch_members(b) == 0) return LBM_OK;
  int st = upload(b);
  if (st) return st;
  if (!b->clock_set) {  // the batch clock and the done count start at zero
    cudaError_t e = cudaMemsetAsync(b->d_counters + kChunk + 1, 0,
                                    2 * sizeof(unsigned), b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "cudaMemsetAsync(clock)");
    b->clock_set = true;
  }
  int64_t s = 0;
  // first step direct (one-time kernel set-up stays outside any capture)
  for (; s < nsteps && s < 2; ++s) {
    st = direct_step(b, static_cast<int>(s & 1), s == nsteps - 1);
    if (st) return st;
  }
  while (s + kChunk <= nsteps - 1) {
    st = graph_chunk(b);
    if (st) return st;
    s += kChunk;
  }
  for (; s < nsteps; ++s) {
    st = direct_step(b, static_cast<int>(s & 1), s == nsteps - 1);
    if (st) return st;
  }
  cudaError_t e = lbmtau1::launch_batch_finalize(
      b->d_members, static_cast<int>(b->packed.size()), b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "batch finalize launch");
  for (lbm_ctx *c : b->packed) {
    c->cur ^= static_cast<int>(nsteps & 1);
    c->has_residual = true;
    c->steps += nsteps;
  }
  b->clock += static_cast<uint32_t>(nsteps);
  b->err[0] = '\0';
  return LBM_OK;
}

int lbm_batch_autotune(lbm_batch *b, int32_t steps_per_variant,
                       int32_t *chosen, double *ms_per_step) {
  if (!b) return LBM_E_INVAL;
  if (steps_per_variant < 2 || steps_per_variant % 2)
    return bfail(b, LBM_E_INVAL, "steps_per_variant must be even and >= 2");
  const int nv = lbmtau1::variant_count();
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return LBM_E_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return LBM_E_CUDA;
  }
  int best = b->variant;
  float best_ms = -1.f;
  int st = LBM_OK;
  for (int v = 0; v < nv && st == LBM_OK; ++v) {
    st = lbm_batch_set_variant(b, v);
    if (st) break;
    st = lbm_batch_step(b, 2);  // warm-up, builds this variant's set-up
    if (st) break;
    cudaEventRecord(e0, b->stream);
    st = lbm_batch_step(b, steps_per_variant);
    if (st) break;
    cudaEventRecord(e1, b->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      st = LBM_E_CUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= static_cast<float>(steps_per_variant);
    if (ms_per_step) ms_per_step[v] = ms;
    if (best_ms < 0.f || ms < best_ms) {
      best_ms = ms;
      best = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) return st;
  st = lbm_batch_set_variant(b, best);
  if (chosen) *chosen = best;
  return st;
}

int lbm_batch_residuals(lbm_batch *b, double *residual, double *mass,
                        int32_t *status) {
  if (!b) return LBM_E_INVAL;
  if (!residual || !mass || !status)
    return bfail(b, LBM_E_INVAL, "null output array");
  for (int32_t i = 0; i < b->capacity; ++i) {
    residual[i] = mass[i] = 0.0;
    status[i] = LBM_E_STATE;
  }
  int st = upload(b);  // descriptors in slot order of the current members
  if (st) return st;
  const int n = static_cast<int>(b->packed.size());
  if (n == 0) return LBM_OK;
  cudaError_t e = lbmtau1::launch_batch_gather(b->d_members, n, b->d_gather,
                                               b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "gather kernel");
  std::vector<double> h(4 * static_cast<size_t>(n));
  e = cudaMemcpyAsync(h.data(), b->d_gather, sizeof(double) * h.size(),
                      cudaMemcpyDeviceToHost, b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "cudaMemcpyAsync(gather)");
  e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "cudaStreamSynchronize");
  int k = 0;
  for (int32_t i = 0; i < b->capacity; ++i) {
    lbm_ctx *c = b->slots[i];
    if (!c) continue;
    const double *r = &h[4 * static_cast<size_t>(k++)];
    unsigned flag;
    memcpy(&flag, &r[3], sizeof flag);
    residual[i] = r[1] > 0.0 ? sqrt(r[0] / r[1]) : sqrt(r[0]);
    mass[i] = static_cast<double>(c->n_fluid) + r[2];
    status[i] = !c->has_residual ? LBM_E_STATE
                : (flag & 2u)    ? LBM_E_CUDA
                : (flag & 1u)    ? LBM_E_UNSTABLE
                                 : LBM_OK;
  }
  b->err[0] = '\0';
  return LBM_OK;
}

void lbm_batch_destroy(lbm_batch *b) {
  if (!b) return;
  drop_graph(b);
  delete b;
}

const char *lbm_batch_last_error(const lbm_batch *b) {
  return b ? b->err : "null batch";
}

}  // extern "C"
