// One LBMTau1 step with its residual reduction, on caller-owned device
// fields, that allocates no memory at all.
//
// The regular entry points keep their reduction scratch (per-warp-tile partial
// sums and the instability flag) in the device workspace that the caller
// allocates for a context.  Some callers cannot allocate even that: a host
// application that owns every byte of device memory through its own pool
// allocator and forbids side allocations, or a loop with a hard latency
// budget in which cudaMalloc / cudaFree (cudaFree synchronises the device)
// are not acceptable.  For them, lbm_step_noalloc takes the fields and the
// node-type array they already hold and keeps its scratch in the fixed-size
// device array below, which every GPU that loads this library holds until
// the process exits.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/lbmtau1.h"
#include "lbm_step.cuh"

namespace {

// Largest step launch the scratch can serve, in thread blocks (block tiles);
// the tile variant chosen for a domain makes that about 10^8 nodes for the
// short tiles small domains get and 2 * 10^9 for the tall ones of large
// domains.
constexpr int64_t kNoAllocMaxBlocks = int64_t(1) << 16;
constexpr int64_t kNoAllocPartials = kNoAllocMaxBlocks * lbmtau1::kTileWarps;
constexpr int kMaxDevices = 64;

// Per-warp-tile partial triples (6 MB), then one slot whose low 4 bytes
// hold the flag.
static __device__ __align__(256) double
    g_step_scratch[3 * kNoAllocPartials + 1];

std::once_flag g_setup_once[kMaxDevices];
double *g_scratch_addr[kMaxDevices];
cudaError_t g_setup_status[kMaxDevices];

bool aligned16(const void *p) {
  return (reinterpret_cast<uintptr_t>(p) & 15u) == 0;
}

}  // namespace

extern "C" int lbm_step_noalloc(const float *drho_in, const float *jx_in,
                                const float *jy_in, float *drho_out,
                                float *jx_out, float *jy_out,
                                const uint8_t *mask, int64_t nx, int64_t ny,
                                int64_t pitch, int32_t periodic_x,
                                int32_t periodic_y, double fx, double fy,
                                double *dev_sums, uint32_t *dev_flags,
                                void *cuda_stream) {
  if (!drho_in || !jx_in || !jy_in || !drho_out || !jx_out || !jy_out ||
      !mask || !dev_sums || !dev_flags)
    return LBM_E_INVAL;
  if (nx < 1 || ny < 1 || nx >= (int64_t(1) << 30) || ny >= (int64_t(1) << 30) ||
      pitch < nx || pitch % 32 != 0)
    return LBM_E_INVAL;
  const void *ptrs[7] = {drho_in, jx_in, jy_in, drho_out, jx_out, jy_out, mask};
  for (const void *p : ptrs)
    if (!aligned16(p)) return LBM_E_INVAL;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return LBM_E_CUDA;
  const int variant = lbmtau1::choose_variant(nx, ny, lbmtau1::kStorageF32);
  const int64_t blocks = lbmtau1::launched_blocks(nx, ny, variant);
  if (blocks > kNoAllocMaxBlocks)
    return LBM_E_INVAL;  // domain larger than the static scratch serves
  // Set-up on the first call on each device: the device address of the
  // scratch array (the host-side name is only a stand-in for it).
  std::call_once(g_setup_once[dev], [dev] {
    g_setup_status[dev] = cudaGetSymbolAddress(
        reinterpret_cast<void **>(&g_scratch_addr[dev]), g_step_scratch);
  });
  if (g_setup_status[dev] != cudaSuccess) return LBM_E_CUDA;
  double *partials = g_scratch_addr[dev];
  unsigned *flag = reinterpret_cast<unsigned *>(partials + 3 * kNoAllocPartials);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

  // The array keeps the previous call's contents: the flag must start at
  // zero; the partials are all rewritten by the step launch.
  if (cudaMemsetAsync(flag, 0, sizeof(unsigned), s) != cudaSuccess)
    return LBM_E_CUDA;
  lbmtau1::StepLaunch a;
  a.src.d = const_cast<float *>(drho_in);
  a.src.jx = const_cast<float *>(jx_in);
  a.src.jy = const_cast<float *>(jy_in);
  a.dst.d = drho_out;
  a.dst.jx = jx_out;
  a.dst.jy = jy_out;
  a.mask = mask;
  a.nx = nx;
  a.ny = ny;
  a.pitch = pitch;
  a.periodic_x = periodic_x != 0;
  a.periodic_y = periodic_y != 0;
  a.fx = static_cast<float>(fx);
  a.fy = static_cast<float>(fy);
  a.partials = partials;
  a.flag = flag;
  a.variant = variant;
  if (lbmtau1::launch_step(a, true, s) != cudaSuccess) return LBM_E_CUDA;
  if (lbmtau1::launch_finalize(partials, blocks, dev_sums, s) != cudaSuccess)
    return LBM_E_CUDA;
  if (cudaMemcpyAsync(dev_flags, flag, sizeof(unsigned),
                      cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return LBM_E_CUDA;
  return LBM_OK;
}
