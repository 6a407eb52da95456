// Narrow i-pass kernels (the shifted transform of a few slots) for
// double-float, transform lengths 128, 256, 512, one tile per CTA.
#include "conv_impl.cuh"

namespace bae {

template bool launch_conv_i_narrow<dsf, 128, 0, false>(const ConvArgs<dsf>&, dim3, size_t, cudaStream_t);
template bool launch_conv_i_narrow<dsf, 256, 0, false>(const ConvArgs<dsf>&, dim3, size_t, cudaStream_t);
template bool launch_conv_i_narrow<dsf, 512, 0, false>(const ConvArgs<dsf>&, dim3, size_t, cudaStream_t);

}  // namespace bae
