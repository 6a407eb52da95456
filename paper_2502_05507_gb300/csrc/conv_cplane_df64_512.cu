// Cluster plane kernels of the potential apply for double-float, transform length 512.
#include "conv_cplane.cuh"

namespace bae {

template bool cplane_ready<dsf, 512>();
template void cplane_launch<dsf, 512>(const ConvArgs<dsf>&, cudaStream_t, bool);

}  // namespace bae
