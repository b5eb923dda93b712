// The x-row kernels (gbd_row.cuh) with the radix-16 stages on the tensor cores in split FP16.
#include "gbd_row.cuh"

namespace gbd {
template bool row_dispatch_p<2>(int, int, const RowArgs*, const float2*, cudaStream_t);
}  // namespace gbd
