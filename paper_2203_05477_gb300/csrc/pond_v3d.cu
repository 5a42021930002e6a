// D3Q64 kernels, FP64 populations.
#include "pond_v3_impl.cuh"

namespace pond {
POND_V3(double)
}  // namespace pond
