// Kernels of the potential apply for double-float, transform length 256.
#include "conv_impl.cuh"

namespace bae {

template void run_conv<dsf, 256>(const ConvArgs<dsf>&, cudaStream_t);
template void conv_configure<dsf, 256>();

}  // namespace bae
