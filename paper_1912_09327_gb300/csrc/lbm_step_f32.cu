// The LBMTau1 step kernels instantiated for FP32 storage (one translation
// unit per storage format, so that the formats compile in parallel).
#include "lbm_kernels.cuh"

namespace lbmtau1 {
const StorageOps kOpsF32 = make_ops<float>();
}  // namespace lbmtau1
