// Kernels of the potential apply for double-float, transform lengths 16, 32, 64.
#include "conv_impl.cuh"

namespace bae {

template void run_conv<dsf, 16>(const ConvArgs<dsf>&, cudaStream_t);
template void conv_configure<dsf, 16>();
template void run_conv<dsf, 32>(const ConvArgs<dsf>&, cudaStream_t);
template void conv_configure<dsf, 32>();
template void run_conv<dsf, 64>(const ConvArgs<dsf>&, cudaStream_t);
template void conv_configure<dsf, 64>();

}  // namespace bae
