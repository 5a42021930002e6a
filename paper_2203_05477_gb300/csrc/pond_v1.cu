// pond_v1.cu -- the D1Q4 grid step kernels in both precisions: every face- and cell-kernel variant.
#include "pond_variants.cuh"

namespace pond {
template void launch_face_m<1, float, FACE_PLAIN>(int, const Params<1, float> &, cudaStream_t);
template void launch_cell<1, float>(int, const Params<1, float> &, cudaStream_t);
template void launch_face_m<1, double, FACE_PLAIN>(int, const Params<1, double> &, cudaStream_t);
template void launch_cell<1, double>(int, const Params<1, double> &, cudaStream_t);
}  // namespace pond
