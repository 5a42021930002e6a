// pond_v2d.cu -- the D2Q16 FP64 step kernels: every face-kernel variant in the plain,
// pair-collecting and learned modes, and every cell-kernel variant.
#include "pond_variants.cuh"

namespace pond {
template void launch_face_m<2, double, FACE_PLAIN>(int, const Params<2, double> &, cudaStream_t);
template void launch_face_m<2, double, FACE_COLLECT>(int, const Params<2, double> &, cudaStream_t);
template void launch_face_m<2, double, FACE_LEARNED>(int, const Params<2, double> &, cudaStream_t);
template void launch_cell<2, double>(int, const Params<2, double> &, cudaStream_t);
}  // namespace pond
