// pond_v2f_learned.cu -- the D2Q16 FP32 face kernels that start from the learned prediction,
// every variant (a translation unit of its own, so they compile in parallel with the others).
#include "pond_variants.cuh"

namespace pond {
template void launch_face_m<2, float, FACE_LEARNED>(int, const Params<2, float> &, cudaStream_t);
}  // namespace pond
