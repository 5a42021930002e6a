// pond_veq.cu -- the step kernels with the equilibration alternative of Sec. II.C (an
// ablation of Grad's projection), D1Q4 and D2Q16 grids in both precisions: one face-kernel
// tile and one cell-kernel block size each.
#include "pond_variants.cuh"

namespace pond {
template void launch_face_m<1, float, FACE_EQUIL>(int, const Params<1, float> &, cudaStream_t);
template void launch_face_m<1, double, FACE_EQUIL>(int, const Params<1, double> &, cudaStream_t);
template void launch_face_m<2, float, FACE_EQUIL>(int, const Params<2, float> &, cudaStream_t);
template void launch_face_m<2, double, FACE_EQUIL>(int, const Params<2, double> &, cudaStream_t);
template void launch_cell_eq<1, float>(const Params<1, float> &, cudaStream_t);
template void launch_cell_eq<1, double>(const Params<1, double> &, cudaStream_t);
template void launch_cell_eq<2, float>(const Params<2, float> &, cudaStream_t);
template void launch_cell_eq<2, double>(const Params<2, double> &, cudaStream_t);
}  // namespace pond
