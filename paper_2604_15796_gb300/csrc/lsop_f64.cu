// Instantiation of the operator passes for complex FP64 fields.
#include "lsop_kernels.cuh"

namespace fwi {
#define FWI_T double
FWI_DEFINE_LSOP(double)
#undef FWI_T
}  // namespace fwi
