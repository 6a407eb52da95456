// Cluster plane kernels of the potential apply for float32, transform length 512.
#include "conv_cplane.cuh"

namespace bae {

template bool cplane_ready<float, 512>();
template void cplane_launch<float, 512>(const ConvArgs<float>&, cudaStream_t, bool);

}  // namespace bae
