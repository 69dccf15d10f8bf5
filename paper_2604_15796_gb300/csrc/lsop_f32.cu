// Instantiation of the operator passes for complex FP32 fields.
#include "lsop_kernels.cuh"

namespace fwi {
#define FWI_T float
FWI_DEFINE_LSOP(float)
#undef FWI_T
}  // namespace fwi
