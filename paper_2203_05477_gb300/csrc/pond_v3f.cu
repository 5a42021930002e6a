// D3Q64 kernels, FP32 populations.
#include "pond_v3_impl.cuh"

namespace pond {
POND_V3(float)
}  // namespace pond
