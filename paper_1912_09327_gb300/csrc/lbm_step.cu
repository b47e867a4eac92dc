// Dispatch of the LBMTau1 step kernels over the storage formats, and the
// kernels that do not depend on the format (tile flags, reductions).
#include "lbm_kernels.cuh"

namespace lbmtau1 {
namespace {

// One warp per warp tile: 1 when the tile is clean (see launch_tile_flags).
template <int kC, int kRows>
__global__ void tile_flags_kernel(const uint8_t *__restrict__ mask,
                                  int64_t nx, int64_t ny, int64_t pitch,
                                  int64_t gx, int64_t ntiles,
                                  uint8_t *__restrict__ out) {
  constexpr int kTile = (kLanes - 2) * kC;
  const int64_t t = (static_cast<int64_t>(blockIdx.x) * blockDim.x +
                     threadIdx.x) / kLanes;
  const int lane = threadIdx.x & (kLanes - 1);
  if (t >= ntiles) return;  // whole warps leave together
  const int64_t block = t / kWarps, w = t % kWarps;
  const int64_t x0 = (block % gx) * kTile, y0 = (block / gx * kWarps + w) * kRows;
  // rows y0 - 1 .. y0 + kRows and columns x0 - kC .. x0 + 31 kC - 1
  bool ok = x0 - kC >= 0 && x0 + (kLanes - 1) * kC <= nx && y0 >= 1 &&
            y0 + kRows <= ny - 1;
  if (ok) {
    const int64_t xb = x0 - kC + static_cast<int64_t>(kC) * lane;
    for (int64_t y = y0 - 1; y <= y0 + kRows && ok; ++y) {
      const uint8_t *p = mask + y * pitch + xb;
      unsigned m;
      if constexpr (kC == 4)
        m = *reinterpret_cast<const unsigned *>(p);
      else
        m = *reinterpret_cast<const unsigned short *>(p);
      ok = __all_sync(kFull, m == 0u);
    }
  }
  if (lane == 0) out[t] = ok ? 1 : 0;
}

// Copies every member's result slot (3 sums and the flag word) into out,
// 4 doubles per member in descriptor order.
__global__ void batch_gather_kernel(const BatchMember *__restrict__ members,
                                    int nmembers, double *__restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nmembers)
    for (int q = 0; q < 4; ++q) out[4 * i + q] = members[i].result[q];
}

// The partial triple of block tile b: its warps' triples added in warp order.
__device__ __forceinline__ double block_partial(const double *partials,
                                               int64_t b, int q) {
  double s = 0.0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) s += partials[3 * (b * kWarps + w) + q];
  return s;
}

// One block per batch member: sums its partials (fixed order) into its
// result slot.
__global__ void __launch_bounds__(256)
    batch_finalize_kernel(const BatchMember *__restrict__ members) {
  __shared__ double buf[3][256];
  const BatchMember &m = members[blockIdx.x];
  double s[3] = {0.0, 0.0, 0.0};
  for (int64_t k = threadIdx.x; k < m.nblocks; k += 256)
    for (int q = 0; q < 3; ++q) s[q] += block_partial(m.partials, k, q);
  for (int q = 0; q < 3; ++q) buf[q][threadIdx.x] = s[q];
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int q = 0; q < 3; ++q) buf[q][threadIdx.x] += buf[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 3) m.result[threadIdx.x] = buf[threadIdx.x][0];
}

constexpr int kFinalizeThreads = 1024;

__global__ void __launch_bounds__(kFinalizeThreads)
    finalize_kernel(const double *__restrict__ partials, int64_t nblocks,
                    double *__restrict__ out) {
  __shared__ double buf[3][kFinalizeThreads];
  double s[3] = {0.0, 0.0, 0.0};
  for (int64_t b = threadIdx.x; b < nblocks; b += kFinalizeThreads) {
    // the block tile's kWarps triples: 12 contiguous doubles, 16-byte aligned
    const double2 *p = reinterpret_cast<const double2 *>(partials + 3 * kWarps * b);
    double v[3 * kWarps];
#pragma unroll
    for (int i = 0; i < 3 * kWarps / 2; ++i) {
      const double2 t = p[i];
      v[2 * i] = t.x;
      v[2 * i + 1] = t.y;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double t = 0.0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) t += v[3 * w + k];
      s[k] += t;
    }
  }
  for (int k = 0; k < 3; ++k) buf[k][threadIdx.x] = s[k];
  __syncthreads();
  for (int w = kFinalizeThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int k = 0; k < 3; ++k) buf[k][threadIdx.x] += buf[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 3) out[threadIdx.x] = buf[threadIdx.x][0];
}

// the launchers of a storage format
const StorageOps &ops(int storage) {
  switch (storage) {
    case kStorageF16: return kOpsF16;
    case kStorageBF16: return kOpsBF16;
    default: return kOpsF32;
  }
}

}  // namespace


int64_t step_blocks(int64_t nx, int64_t ny) {
  // the largest grid over all variants, so a workspace fits any of them
  int64_t most = 0;
  for (int i = 0; i < kNumVariants; ++i) {
    const Variant v = kVariants[i];
    const int64_t tile_x = (kLanes - 2) * v.cols;
    const int64_t tile_y = static_cast<int64_t>(kWarps) * v.rows;
    const int64_t b = ((nx + tile_x - 1) / tile_x) * ((ny + tile_y - 1) / tile_y);
    most = b > most ? b : most;
  }
  return most;
}

int variant_count() { return kNumVariants; }

void variant_tile(int v, int64_t *tile_x, int64_t *tile_y) {
  const Variant t = kVariants[(v >= 0 && v < kNumVariants) ? v : 0];
  *tile_x = (kLanes - 2) * t.cols;
  *tile_y = static_cast<int64_t>(kWarps) * t.rows;
}

bool variant_has_clean_code(int v) {
  return v >= 0 && v < kNumVariants && kVariants[v].dual;
}

int default_variant() { return active_variant(); }

cudaError_t launch_batch(int v, const BatchLaunch &b, bool reduce,
                         cudaStream_t s) {
  if (v < 0 || v >= kNumVariants) return cudaErrorInvalidValue;
  return ops(b.storage).batch(v, b, reduce, s);
}

cudaError_t launch_batch_finalize(const BatchMember *members, int nmembers,
                                  cudaStream_t s) {
  if (nmembers <= 0) return cudaSuccess;
  (void)cudaGetLastError();
  batch_finalize_kernel<<<nmembers, 256, 0, s>>>(members);
  return cudaGetLastError();
}

cudaError_t launch_batch_gather(const BatchMember *members, int nmembers,
                                double *out, cudaStream_t s) {
  if (nmembers <= 0) return cudaSuccess;
  (void)cudaGetLastError();
  batch_gather_kernel<<<(nmembers + 127) / 128, 128, 0, s>>>(members, nmembers,
                                                             out);
  return cudaGetLastError();
}

int64_t launched_blocks(int64_t nx, int64_t ny, int variant) {
  const dim3 g = step_grid(nx, ny, variant);
  return static_cast<int64_t>(g.x) * g.y;
}

int dual_variant(int v, int64_t nx, int64_t ny) {
  if (forced_variant() >= 0 || v < 0 || v >= kNumVariants) return -1;
  const Variant b = kVariants[v];
  if (b.dual) return -1;
  static int sms = [] {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) !=
            cudaSuccess)
      n = 0;
    return n;
  }();
  // the clean-tile code pays off once every SM runs a few blocks; on
  // smaller grids the general code's shorter tiles win
  if (sms <= 0 || launched_blocks(nx, ny, v) < 2 * static_cast<int64_t>(sms))
    return -1;
  for (int i = 0; i < kNumVariants; ++i) {
    const Variant d = kVariants[i];
    if (d.dual && d.cols == b.cols && d.rows == b.rows &&
        d.min_blocks == b.min_blocks && d.stages == b.stages)
      return i;
  }
  return -1;
}

int choose_variant(int64_t nx, int64_t ny, int storage) {
  const int f = forced_variant();
  if (f >= 0) return f;
  return ops(storage).choose(nx, ny);
}

cudaError_t launch_step(const StepLaunch &a, bool reduce, cudaStream_t s) {
  if (a.ny >= (int64_t(1) << 30) || a.nx >= (int64_t(1) << 30))
    return cudaErrorInvalidValue;  // the tile loop indexes rows in 32 bits
  return ops(a.storage).step(a, reduce, s);
}

cudaError_t launch_tile_flags(int v, const uint8_t *mask, int64_t nx,
                              int64_t ny, int64_t pitch, uint8_t *out,
                              cudaStream_t s) {
  if (v < 0 || v >= kNumVariants) return cudaErrorInvalidValue;
  const dim3 g = step_grid(nx, ny, v);
  const int64_t ntiles = static_cast<int64_t>(g.x) * g.y * kWarps;
  const int64_t blocks = (ntiles * kLanes + 255) / 256;
  (void)cudaGetLastError();
  with_variant(v, [&](auto kv) {
    constexpr Variant t = kVariants[decltype(kv)::value];
    tile_flags_kernel<t.cols, t.rows><<<static_cast<unsigned>(blocks), 256, 0,
                                        s>>>(mask, nx, ny, pitch, g.x, ntiles,
                                             out);
    return 0;
  });
  return cudaGetLastError();
}

cudaError_t launch_finalize(const double *partials, int64_t nblocks,
                            double *out, cudaStream_t s) {
  (void)cudaGetLastError();
  finalize_kernel<<<1, kFinalizeThreads, 0, s>>>(partials, nblocks, out);
  return cudaGetLastError();
}


cudaError_t launch_pack(int storage, const double *staging, Fields f,
                        int64_t nx, int64_t pitch, int64_t y0, int64_t rows,
                        cudaStream_t s) {
  return ops(storage).pack(staging, f, nx, pitch, y0, rows, s);
}

cudaError_t launch_unpack(int storage, Fields f, const uint8_t *mask,
                          double *staging, int64_t nx, int64_t pitch,
                          int64_t y0, int64_t rows, cudaStream_t s) {
  return ops(storage).unpack(f, mask, staging, nx, pitch, y0, rows, s);
}

cudaError_t launch_change(int storage, Fields now, Fields snap,
                          const uint8_t *mask, int64_t nx, int64_t ny,
                          int64_t pitch, double *partials, int64_t blocks,
                          cudaStream_t s) {
  return ops(storage).change(now, snap, mask, nx, ny, pitch, partials, blocks,
                             s);
}

cudaError_t launch_solid_storage(int storage, Fields f, const uint8_t *mask,
                                 int64_t n, float fx, float fy,
                                 cudaStream_t s) {
  return ops(storage).solid(f, mask, n, fx, fy, s);
}

int storage_bytes(int storage) {
  return storage == kStorageF16 || storage == kStorageBF16 ? 2 : 4;
}

}  // namespace lbmtau1
