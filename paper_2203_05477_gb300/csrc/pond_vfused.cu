// pond_vfused.cu -- the fused step kernels (faces and cell update of a tile in one kernel),
// every tile variant of D1Q4 and D2Q16 grids in both precisions.
#include "pond_variants.cuh"

namespace pond {
template void launch_step_fused<1, float>(int, const Params<1, float> &, cudaStream_t);
template void launch_step_fused<1, double>(int, const Params<1, double> &, cudaStream_t);
template void launch_step_fused<2, float>(int, const Params<2, float> &, cudaStream_t);
template void launch_step_fused<2, double>(int, const Params<2, double> &, cudaStream_t);
}  // namespace pond
