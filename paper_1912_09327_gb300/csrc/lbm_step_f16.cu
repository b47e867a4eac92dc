// The LBMTau1 step kernels instantiated for FP16 storage (one translation
// unit per storage format, so that the formats compile in parallel).
#include "lbm_kernels.cuh"

namespace lbmtau1 {
const StorageOps kOpsF16 = make_ops<__half>();
}  // namespace lbmtau1
