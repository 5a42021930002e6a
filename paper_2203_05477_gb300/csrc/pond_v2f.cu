// pond_v2f.cu -- the D2Q16 FP32 step kernels: every face- and cell-kernel variant.
#include "pond_variants.cuh"

namespace pond {
template void launch_face<2, float>(int, bool, const Params<2, float> &, cudaStream_t);
template void launch_cell<2, float>(int, const Params<2, float> &, cudaStream_t);
}  // namespace pond
