// Cluster plane kernels of the potential apply for double-float, transform length 256.
#include "conv_cplane.cuh"

namespace bae {

template bool cplane_ready<dsf, 256>();
template void cplane_launch<dsf, 256>(const ConvArgs<dsf>&, cudaStream_t, bool);

}  // namespace bae
