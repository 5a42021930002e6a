// pond_v2d.cu -- the D2Q16 FP64 step kernels: every face- and cell-kernel variant.
#include "pond_variants.cuh"

namespace pond {
template void launch_face<2, double>(int, bool, const Params<2, double> &, cudaStream_t);
template void launch_cell<2, double>(int, const Params<2, double> &, cudaStream_t);
}  // namespace pond
