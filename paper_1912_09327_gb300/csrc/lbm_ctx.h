// Internal definitions shared by the library's translation units: the
// workspace layout and the context behind the opaque lbm_ctx handle.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/lbmtau1.h"
#include "lbm_step.cuh"

namespace lbmtau1 {

// Whether a context rounds its stored moments stochastically: always for
// LBM_ROUND_STOCHASTIC, for the 16-bit formats under LBM_ROUND_DEFAULT.
inline bool stochastic_rounding(int storage, int rounding) {
  return rounding == LBM_ROUND_STOCHASTIC ||
         (rounding == LBM_ROUND_DEFAULT && storage != LBM_STORAGE_F32);
}

struct Layout {
  int64_t pitch = 0, staging_rows = 0, nblocks = 0;
  size_t field_bytes = 0;   // one field plane
  size_t off_fields = 0;    // 6 planes: copy 0 (d, jx, jy), copy 1 (d, jx, jy)
  size_t off_mask = 0;
  size_t off_partials = 0;
  size_t off_clean = 0;     // one byte per warp tile: clean-tile flags
  size_t off_result = 0;    // 3 doubles + flag
  size_t off_staging = 0;
  size_t total = 0;
};

}  // namespace lbmtau1

struct lbm_ctx {
  lbm_params p;
  lbmtau1::Layout L;
  char *base;
  lbmtau1::Fields f[2];
  uint8_t *mask;
  double *partials;
  uint8_t *clean;       // clean-tile flags of tile variant clean_variant
  int clean_variant;    // -1: not computed for the current node types
  double *result;       // sum |du|^2, sum |u|^2, sum (rho - 1)
  unsigned *flag;       // follows the three doubles
  double *staging;
  cudaStream_t stream;
  int cur;              // copy holding the current state
  int variant;          // tile variant, chosen at the first step (-1 before)
  int64_t steps;        // steps taken (seeds stochastic rounding)
  // 16 unreduced steps captured as one CUDA graph, one per starting copy
  // (rebuilt when the tile variant changes); none on an uncapturable stream
  cudaGraphExec_t graph[2];
  int graph_variant[2];
  bool graphs_off;
  unsigned long long wait_ns;  // staged-row wait limit of the step kernel
  bool has_geometry;
  bool has_residual;
  int64_t n_fluid;
  char err[256];
};
