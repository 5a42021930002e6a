// pond3_launch.cuh -- launches of the D3Q64 kernels (instantiated in pond_v3f.cu and pond_v3d.cu through pond_v3_impl.cuh).
#pragma once

#include <cstdio>

#include "pond3.cuh"

namespace pond {

// dynamic shared memory of the face kernel above the default limit
template <typename R>
cudaError_t prepare3();
// the face kernel of tile variant v (0 .. face3_variant_count - 1) and the cell kernel of
// block variant v (0 .. cell3_variant_count - 1); names for the autotuner's report
constexpr int face3_variant_count = 3, cell3_variant_count = 3;
template <typename R>
void launch_face3(int v, const Params3<R> &P, cudaStream_t st);
template <typename R>
void launch_cell3(int v, const Params3<R> &P, cudaStream_t st);
template <typename R>
void face3_name(int v, char *buf, size_t n);
inline void cell3_name(int v, char *buf, size_t n)
{
    static const int threads[cell3_variant_count] = {128, 256, 64};
    std::snprintf(buf, n, "cell3 %d threads", threads[(v >= 0 && v < cell3_variant_count) ? v : 0]);
}
template <typename R>
void launch_init3(const Params3<R> &P, const double *rho, const double *ux, const double *uy, const double *uz,
                  const double *p, cudaStream_t st);
template <typename R>
void launch_conserved3(const Params3<R> &P, double *rho, double *mx, double *my, double *mz, double *E, cudaStream_t st);
template <typename R>
void launch_export3(const Params3<R> &P, double *cf, double *cg, double *fr, cudaStream_t st);

}  // namespace pond
