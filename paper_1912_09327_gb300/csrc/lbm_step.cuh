// Launch interface of the LBMTau1 D2Q9 step kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbmtau1 {

// Warps per block tile (stacked in y).  A reduced step writes one partial
// triple per warp tile: kTileWarps triples per block tile.
constexpr int kTileWarps = 4;

// Storage formats (the LBM_STORAGE_* values of the C ABI).
constexpr int kStorageF32 = 0;
constexpr int kStorageF16 = 1;
constexpr int kStorageBF16 = 2;
int storage_bytes(int storage);  // bytes per stored element

// Fields of one ping-pong copy: rho - 1 and the momentum j = rho u in the
// storage format, rows of `pitch` elements (pitch % 32 == 0).
struct Fields {
  void *d;
  void *jx;
  void *jy;
};

struct StepLaunch {
  Fields src;           // copy read (time t)
  Fields dst;           // copy written (time t + 1)
  const uint8_t *mask;  // node types, same pitch as the fields
  int64_t nx, ny, pitch;
  int periodic_x, periodic_y;
  float fx, fy;
  double *partials;     // 3 doubles per warp tile (reduced steps only)
  unsigned int *flag;   // sticky instability flag (reduced steps only)
  int storage = kStorageF32;
  int variant = 0;      // tile variant (see choose_variant)
  int sr = 0;           // stochastic rounding (16-bit: all fields; FP32: j)
  uint32_t step = 0;    // the domain's step count (seeds the rounding)
  // one byte per warp tile of this launch's tile variant: 1 when the tile
  // is clean (launch_tile_flags); null: every tile takes the general code
  const uint8_t *clean = nullptr;
  // how long a warp waits for a staged row before it gives up (raising
  // kFlagCopyTimeout); 0 gives up at once.  Draining the copies still in
  // flight before a warp leaves its tile always keeps the one-second bound.
  unsigned long long wait_ns = 1000000000ull;
  // Shan-Chen coupling g of the multiphase step (0: single phase; FP32
  // storage only)
  float g_sc = 0.0f;
};

// One member of a batch (see launch_batch): both field copies, the copy that
// holds its current state, its node types and problem data, and its own
// reduction partials and result slot.
struct BatchMember {
  Fields f[2];
  const uint8_t *mask;
  int64_t nx, ny, pitch;
  int periodic_x, periodic_y;
  float fx, fy;
  double *partials;  // one triple per warp tile
  double *result;    // 3 doubles, then the flag word
  unsigned int *flag;
  int64_t gx;        // block tiles along x for the batch's tile variant
  int64_t nblocks;   // block tiles of the member
  int cur;           // copy holding the state when the batch step starts
  int sr;            // stochastic rounding (as StepLaunch::sr)
  int64_t step_base; // member's step count minus the batch clock
  const uint8_t *clean;  // clean-tile flags for the batch's variant
};

struct BatchLaunch {
  const BatchMember *members;
  const int4 *items;    // (member, tile x, tile y, warp): one per warp tile
  const int *nitems;
  unsigned int *counter;  // zeroed before the launch
  int parity;             // step index within the call, mod 2
  int storage;            // storage format shared by all members
  unsigned int *clock;    // batch steps taken (advanced by each launch)
  unsigned int *done;     // blocks finished in this launch (zero between)
};

// The launchers of one storage format.  The kernels are templates on the
// storage type, instantiated once per format in its own translation unit
// (lbm_step_f32.cu, lbm_step_f16.cu, lbm_step_bf16.cu); the entry points
// below dispatch on the format through these tables.
struct StorageOps {
  cudaError_t (*step)(const StepLaunch &a, bool reduce, cudaStream_t s);
  cudaError_t (*batch)(int v, const BatchLaunch &b, bool reduce,
                       cudaStream_t s);
  int (*choose)(int64_t nx, int64_t ny);
  cudaError_t (*pack)(const double *staging, Fields f, int64_t nx,
                      int64_t pitch, int64_t y0, int64_t rows,
                      cudaStream_t s);
  cudaError_t (*unpack)(Fields f, const uint8_t *mask, double *staging,
                        int64_t nx, int64_t pitch, int64_t y0, int64_t rows,
                        cudaStream_t s);
  cudaError_t (*solid)(Fields f, const uint8_t *mask, int64_t n, float fx,
                       float fy, cudaStream_t s);
  cudaError_t (*change)(Fields now, Fields snap, const uint8_t *mask,
                        int64_t nx, int64_t ny, int64_t pitch,
                        double *partials, int64_t blocks, cudaStream_t s);
};
extern const StorageOps kOpsF32, kOpsF16, kOpsBF16;

// Tile variants: their number, the block tile size of variant v, and the
// default variant of the single-domain path.
int variant_count();
void variant_tile(int v, int64_t *tile_x, int64_t *tile_y);
// True when variant v's kernel carries the clean-tile code (reads the flags).
bool variant_has_clean_code(int v);
int default_variant();

// Enqueues one batched step with tile variant v over a persistent grid; the
// counter must have been zeroed on the stream before.
cudaError_t launch_batch(int v, const BatchLaunch &b, bool reduce,
                         cudaStream_t s);
cudaError_t launch_batch_finalize(const BatchMember *members, int nmembers,
                                  cudaStream_t s);
// Gathers each member's 3 result sums and flag word into out (4 doubles per
// member, descriptor order).
cudaError_t launch_batch_gather(const BatchMember *members, int nmembers,
                                double *out, cudaStream_t s);

// Upper bound on the thread blocks (reduction partials) of one step launch,
// over every tile variant; and the count of the variant in use.
int64_t step_blocks(int64_t nx, int64_t ny);
int64_t launched_blocks(int64_t nx, int64_t ny, int variant);

// Tile variant for a single-domain step of nx x ny nodes: the one forced by
// the LBMTAU1_STEP_VARIANT environment variable, else the one whose grid best
// fills the device (queries the current device once).  All variants give
// bit-identical results.
int choose_variant(int64_t nx, int64_t ny, int storage);

// The variant with v's tiles and, in the same kernel, the code for clean
// tiles (see launch_tile_flags), when v's grid for an nx x ny domain is large
// enough for it to pay off and no variant is forced; else -1.  The caller
// takes it when most warp tiles are clean.
int dual_variant(int v, int64_t nx, int64_t ny);

// Writes one byte per warp tile of tile variant v for an nx x ny domain
// (block tiles in row-major order, kTileWarps per block tile): 1 when every
// row and column the warp tile marches (its rows plus one above and below,
// its lanes' columns including the halo lanes) lies inside the domain and
// holds a fluid node (type 0).  out holds launched_blocks(nx, ny, v) *
// kTileWarps bytes.
cudaError_t launch_tile_flags(int v, const uint8_t *mask, int64_t nx,
                              int64_t ny, int64_t pitch, uint8_t *out,
                              cudaStream_t s);

// Enqueues one step; `reduce` also writes block partials of
// (sum |du|^2, sum |u|^2, sum (rho - 1)) and raises the flag on instability.
cudaError_t launch_step(const StepLaunch &a, bool reduce, cudaStream_t s);

// Sums the partial triples of `nblocks` block tiles (kTileWarps each, added
// in warp order per block) in FP64 in a fixed order into out[0..2].
cudaError_t launch_finalize(const double *partials, int64_t nblocks,
                            double *out, cudaStream_t s);

// Host-format conversion: rows [y0, y0 + rows) of the state, staged as three
// consecutive planes of rows*nx doubles (rho, jx, jy).
cudaError_t launch_pack(int storage, const double *staging, Fields f,
                        int64_t nx, int64_t pitch, int64_t y0, int64_t rows,
                        cudaStream_t s);
cudaError_t launch_unpack(int storage, Fields f, const uint8_t *mask,
                          double *staging, int64_t nx, int64_t pitch,
                          int64_t y0, int64_t rows, cudaStream_t s);

// Sums |u_now - u_snap|^2 and |u_now|^2 over the fluid nodes into `blocks`
// blocks of four partial triples (finalize them with launch_finalize).
cudaError_t launch_change(int storage, Fields now, Fields snap,
                          const uint8_t *mask, int64_t nx, int64_t ny,
                          int64_t pitch, double *partials, int64_t blocks,
                          cudaStream_t s);

// Storage convention of the step kernel: a solid node holds rho - 1 = 0 and
// j = -F (what a solid source contributes, with no test of the node type).
// Writes those values into every solid node of f (n = pitch * ny entries).
cudaError_t launch_solid_storage(int storage, Fields f, const uint8_t *mask,
                                 int64_t n, float fx, float fy,
                                 cudaStream_t s);

}  // namespace lbmtau1
