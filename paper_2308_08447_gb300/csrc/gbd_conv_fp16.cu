// The convolution kernels (gbd_conv.cuh) with the radix-16 stages on the tensor cores in split FP16.
#include "gbd_conv.cuh"

namespace gbd {
template bool film_dispatch_p<2>(int, int, const ColArgs*, const float2*, cudaStream_t);
template bool z_dispatch_p<2>(int, int, const ColArgs*, const float2*, cudaStream_t);
}  // namespace gbd
