// Cluster plane kernels of the potential apply for float64, transform lengths 256, 512.
#include "conv_cplane.cuh"

namespace bae {

template bool cplane_ready<double, 256>();
template void cplane_launch<double, 256>(const ConvArgs<double>&, cudaStream_t, bool);
template bool cplane_ready<double, 512>();
template void cplane_launch<double, 512>(const ConvArgs<double>&, cudaStream_t, bool);

}  // namespace bae
