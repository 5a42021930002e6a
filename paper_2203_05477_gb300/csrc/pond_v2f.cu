// pond_v2f.cu -- the D2Q16 FP32 step kernels: every plain face-kernel variant, the
// pair-collecting face kernel, and every cell-kernel variant.
#include "pond_variants.cuh"

namespace pond {
template void launch_face_m<2, float, FACE_PLAIN>(int, const Params<2, float> &, cudaStream_t);
template void launch_face_m<2, float, FACE_COLLECT>(int, const Params<2, float> &, cudaStream_t);
template void launch_cell<2, float>(int, const Params<2, float> &, cudaStream_t);
}  // namespace pond
