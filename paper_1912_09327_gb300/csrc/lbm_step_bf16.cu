// The LBMTau1 step kernels instantiated for BF16 storage (one translation
// unit per storage format, so that the formats compile in parallel).
#include "lbm_kernels.cuh"

namespace lbmtau1 {
const StorageOps kOpsBF16 = make_ops<__nv_bfloat16>();
}  // namespace lbmtau1
