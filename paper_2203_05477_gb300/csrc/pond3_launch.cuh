// pond3_launch.cuh -- launches of the D3Q64 kernels (instantiated in pond_v3f.cu and pond_v3d.cu through pond_v3_impl.cuh).
#pragma once

#include "pond3.cuh"

namespace pond {

// dynamic shared memory of the face kernel above the default limit
template <typename R>
cudaError_t prepare3();
template <typename R>
void launch_face3(const Params3<R> &P, cudaStream_t st);
template <typename R>
void launch_cell3(const Params3<R> &P, cudaStream_t st);
template <typename R>
void launch_init3(const Params3<R> &P, const double *rho, const double *ux, const double *uy, const double *uz,
                  const double *p, cudaStream_t st);
template <typename R>
void launch_conserved3(const Params3<R> &P, double *rho, double *mx, double *my, double *mz, double *E, cudaStream_t st);
template <typename R>
void launch_export3(const Params3<R> &P, double *cf, double *cg, double *fr, cudaStream_t st);

}  // namespace pond
