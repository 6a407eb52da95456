// Kernels of the potential apply for float32, transform lengths 16, 32, 64, 128, 256, 512.
#include "conv_impl.cuh"

namespace bae {

template void run_conv<float, 16>(const ConvArgs<float>&, cudaStream_t);
template void conv_configure<float, 16>();
template void run_conv<float, 32>(const ConvArgs<float>&, cudaStream_t);
template void conv_configure<float, 32>();
template void run_conv<float, 64>(const ConvArgs<float>&, cudaStream_t);
template void conv_configure<float, 64>();
template void run_conv<float, 128>(const ConvArgs<float>&, cudaStream_t);
template void conv_configure<float, 128>();
template void run_conv<float, 256>(const ConvArgs<float>&, cudaStream_t);
template void conv_configure<float, 256>();
template void run_conv<float, 512>(const ConvArgs<float>&, cudaStream_t);
template void conv_configure<float, 512>();

}  // namespace bae
