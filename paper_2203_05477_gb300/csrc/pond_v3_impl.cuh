// pond_v3_impl.cuh -- launch shapes of the D3Q64 kernels; pond_v3f.cu and pond_v3d.cu
// instantiate them for FP32 and FP64 (two translation units compiled in parallel).
#pragma once

#include <cstdio>
#include <type_traits>

#include "pond3_launch.cuh"

namespace pond {

namespace {
unsigned blocks_of(long long n, int threads) { return unsigned((n + threads - 1) / threads); }
}  // namespace

// Tile variants of the 3D face kernel (the autotuner's search space; entry 0 is the default):
// TX x TY x TZ cells and CTAs per SM for the register budget.
template <typename R, int V>
struct Face3Var;
template <typename R>
struct Face3Var<R, 0> { using type = Face3Tile<R>; };
template <typename R>
struct Face3Var<R, 1> { using type = std::conditional_t<sizeof(R) == 4, Face3Tile<R, 4, 4, 2, 3>, Face3Tile<R, 4, 4, 4, 1>>; };
template <typename R>
struct Face3Var<R, 2> { using type = std::conditional_t<sizeof(R) == 4, Face3Tile<R, 8, 4, 2, 2>, Face3Tile<R, 4, 2, 2, 3>>; };

template <typename R, int V>
cudaError_t prepare3_one()
{
    using T = typename Face3Var<R, V>::type;
    return cudaFuncSetAttribute(face3_kernel<R, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(T::smem));
}

template <typename R>
cudaError_t prepare3()
{
    cudaError_t e = prepare3_one<R, 0>();
    if (e == cudaSuccess) e = prepare3_one<R, 1>();
    if (e == cudaSuccess) e = prepare3_one<R, 2>();
    return e;
}

template <typename R, int V>
void launch_face3_one(const Params3<R> &P, cudaStream_t st)
{
    using T = typename Face3Var<R, V>::type;
    const dim3 g(unsigned((P.nx + T::TX) / T::TX), unsigned((P.ny + T::TY) / T::TY), unsigned((P.nz + T::TZ) / T::TZ));
    face3_kernel<R, T><<<g, T::THREADS, T::smem, st>>>(P);
}

template <typename R>
void launch_face3(int v, const Params3<R> &P, cudaStream_t st)
{
    switch (v) {
    case 1: launch_face3_one<R, 1>(P, st); break;
    case 2: launch_face3_one<R, 2>(P, st); break;
    default: launch_face3_one<R, 0>(P, st); break;
    }
}

template <typename R>
void launch_cell3(int v, const Params3<R> &P, cudaStream_t st)
{
    switch (v) {
    case 1: cell3_kernel<R, 256><<<blocks_of(P.ncell(), 256), 256, 0, st>>>(P); break;
    case 2: cell3_kernel<R, 64><<<blocks_of(P.ncell(), 64), 64, 0, st>>>(P); break;
    default: cell3_kernel<R, 128><<<blocks_of(P.ncell(), 128), 128, 0, st>>>(P); break;
    }
}

template <typename R, int V>
void face3_name_one(char *buf, size_t n)
{
    using T = typename Face3Var<R, V>::type;
    std::snprintf(buf, n, "face3 %dx%dx%d cells, %d threads, %d CTA/SM", T::TX, T::TY, T::TZ, T::THREADS, T::MINB);
}

template <typename R>
void face3_name(int v, char *buf, size_t n)
{
    if (v == 1) face3_name_one<R, 1>(buf, n);
    else if (v == 2) face3_name_one<R, 2>(buf, n);
    else face3_name_one<R, 0>(buf, n);
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
    template void launch_face3<R>(int, const Params3<R> &, cudaStream_t);                                           \
    template void launch_cell3<R>(int, const Params3<R> &, cudaStream_t);                                           \
    template void face3_name<R>(int, char *, size_t);                                                               \
    template void launch_init3<R>(const Params3<R> &, const double *, const double *, const double *, const double *, \
                                  const double *, cudaStream_t);                                                   \
    template void launch_conserved3<R>(const Params3<R> &, double *, double *, double *, double *, double *, cudaStream_t); \
    template void launch_export3<R>(const Params3<R> &, double *, double *, double *, cudaStream_t);

}  // namespace pond
