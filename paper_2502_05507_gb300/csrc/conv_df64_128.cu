// Kernels of the potential apply for double-float, transform length 128.
#include "conv_impl.cuh"

namespace bae {

template void run_conv<dsf, 128>(const ConvArgs<dsf>&, cudaStream_t);
template void conv_configure<dsf, 128>();

}  // namespace bae
