// pond_v3_impl.cuh -- launch shapes of the D3Q64 kernels; pond_v3f.cu and pond_v3d.cu
// instantiate them for FP32 and FP64 (two translation units compiled in parallel).
#pragma once

#include "pond3_launch.cuh"

namespace pond {

namespace {
unsigned blocks_of(long long n, int threads) { return unsigned((n + threads - 1) / threads); }
}  // namespace

template <typename R>
cudaError_t prepare3()
{
    return cudaFuncSetAttribute(face3_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(Face3Tile<R>::smem));
}

template <typename R>
void launch_face3(const Params3<R> &P, cudaStream_t st)
{
    using T = Face3Tile<R>;
    const dim3 g(unsigned((P.nx + T::TX) / T::TX), unsigned((P.ny + T::TY) / T::TY), unsigned((P.nz + T::TZ) / T::TZ));
    face3_kernel<R><<<g, T::THREADS, T::smem, st>>>(P);
}

template <typename R>
void launch_cell3(const Params3<R> &P, cudaStream_t st)
{
    cell3_kernel<R><<<blocks_of(P.ncell(), 128), 128, 0, st>>>(P);
}

template <typename R>
void launch_init3(const Params3<R> &P, const double *rho, const double *ux, const double *uy, const double *uz,
                  const double *p, cudaStream_t st)
{
    init_cells3_kernel<R><<<blocks_of(P.ncell(), 256), 256, 0, st>>>(P, rho, ux, uy, uz, p);
    init_faces3_kernel<R><<<blocks_of(P.nf(0) + P.nf(1) + P.nf(2), 256), 256, 0, st>>>(P);
}

template <typename R>
void launch_conserved3(const Params3<R> &P, double *rho, double *mx, double *my, double *mz, double *E, cudaStream_t st)
{
    conserved3_kernel<R><<<blocks_of(P.ncell(), 256), 256, 0, st>>>(P, rho, mx, my, mz, E);
}

template <typename R>
void launch_export3(const Params3<R> &P, double *cf, double *cg, double *fr, cudaStream_t st)
{
    export_state3_kernel<R><<<blocks_of(P.ncell(), 256), 256, 0, st>>>(P, cf, cg, fr);
}

#define POND_V3(R)                                                                                                  \
    template cudaError_t prepare3<R>();                                                                             \
    template void launch_face3<R>(const Params3<R> &, cudaStream_t);                                                \
    template void launch_cell3<R>(const Params3<R> &, cudaStream_t);                                                \
    template void launch_init3<R>(const Params3<R> &, const double *, const double *, const double *, const double *, \
                                  const double *, cudaStream_t);                                                   \
    template void launch_conserved3<R>(const Params3<R> &, double *, double *, double *, double *, double *, cudaStream_t); \
    template void launch_export3<R>(const Params3<R> &, double *, double *, double *, cudaStream_t);

}  // namespace pond
