// Kernels of the potential apply for double-float, transform length 512.
#include "conv_impl.cuh"

namespace bae {

template void run_conv<dsf, 512>(const ConvArgs<dsf>&, cudaStream_t);
template void conv_configure<dsf, 512>();

}  // namespace bae
