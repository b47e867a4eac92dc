// Launch interface of the LBMTau1 D2Q9 step kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbmtau1 {

// Fields of one ping-pong copy: rho - 1 and the momentum j = rho u, FP32,
// rows of `pitch` elements (pitch % 32 == 0, rows 128-byte aligned).
struct Fields {
  float *d;
  float *jx;
  float *jy;
};

struct StepLaunch {
  Fields src;           // copy read (time t)
  Fields dst;           // copy written (time t + 1)
  const uint8_t *mask;  // node types, same pitch as the fields
  int64_t nx, ny, pitch;
  int periodic_x, periodic_y;
  float fx, fy;
  double *partials;     // 3 doubles per block (reduced steps only)
  unsigned int *flag;   // sticky instability flag (reduced steps only)
};

// Upper bound on the thread blocks (reduction partials) of one step launch,
// over every tile variant; and the count of the variant in use.
int64_t step_blocks(int64_t nx, int64_t ny);
int64_t launched_blocks(int64_t nx, int64_t ny);

// Enqueues one step; `reduce` also writes block partials of
// (sum |du|^2, sum |u|^2, sum (rho - 1)) and raises the flag on instability.
cudaError_t launch_step(const StepLaunch &a, bool reduce, cudaStream_t s);

// Sums `nblocks` partial triples in FP64 in a fixed order into out[0..2].
cudaError_t launch_finalize(const double *partials, int64_t nblocks,
                            double *out, cudaStream_t s);

// Host-format conversion: rows [y0, y0 + rows) of the state, staged as three
// consecutive planes of rows*nx doubles (rho, jx, jy).
cudaError_t launch_pack(const double *staging, Fields f, int64_t nx,
                        int64_t pitch, int64_t y0, int64_t rows,
                        cudaStream_t s);
cudaError_t launch_unpack(Fields f, const uint8_t *mask, double *staging,
                          int64_t nx, int64_t pitch, int64_t y0, int64_t rows,
                          cudaStream_t s);

// Storage convention of the step kernel: a solid node holds rho - 1 = 0 and
// j = -F (what a solid source contributes, with no test of the node type).
// Writes those values into every solid node of f (n = pitch * ny entries).
cudaError_t launch_solid_storage(Fields f, const uint8_t *mask, int64_t n,
                                 float fx, float fy, cudaStream_t s);

}  // namespace lbmtau1
