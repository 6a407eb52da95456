// Narrow i-pass kernels (the shifted transform of a few slots) for float32,
// transform lengths 128, 256, 512, persistent.
#include "conv_impl.cuh"

namespace bae {

template bool launch_conv_i_narrow<float, 128, 0, true>(const ConvArgs<float>&, dim3, size_t, cudaStream_t);
template bool launch_conv_i_narrow<float, 256, 0, true>(const ConvArgs<float>&, dim3, size_t, cudaStream_t);
template bool launch_conv_i_narrow<float, 512, 0, true>(const ConvArgs<float>&, dim3, size_t, cudaStream_t);

}  // namespace bae
