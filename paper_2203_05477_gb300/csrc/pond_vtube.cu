// pond_vtube.cu -- the persistent batched-tube kernel in both precisions: every variant.
#include "pond_variants.cuh"

namespace pond {
template void launch_tube<float>(int, unsigned, const TubeParams<float> &, int, int, cudaStream_t);
template void launch_tube<double>(int, unsigned, const TubeParams<double> &, int, int, cudaStream_t);
}  // namespace pond
