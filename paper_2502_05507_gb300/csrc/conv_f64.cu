// Kernels of the potential apply for float64, transform lengths 16, 32, 64, 128, 256, 512.
#include "conv_impl.cuh"

namespace bae {

template void run_conv<double, 16>(const ConvArgs<double>&, cudaStream_t);
template void conv_configure<double, 16>();
template void run_conv<double, 32>(const ConvArgs<double>&, cudaStream_t);
template void conv_configure<double, 32>();
template void run_conv<double, 64>(const ConvArgs<double>&, cudaStream_t);
template void conv_configure<double, 64>();
template void run_conv<double, 128>(const ConvArgs<double>&, cudaStream_t);
template void conv_configure<double, 128>();
template void run_conv<double, 256>(const ConvArgs<double>&, cudaStream_t);
template void conv_configure<double, 256>();
template void run_conv<double, 512>(const ConvArgs<double>&, cudaStream_t);
template void conv_configure<double, 512>();

}  // namespace bae
