// pond_variants.cuh -- definitions of the variant launchers declared in pond_launch.cuh.
// Included only by the pond_v*.cu translation units, each of which instantiates the
// launchers (and so the kernels) of one dimension and precision.
#pragma once

#include "pond_launch.cuh"

namespace pond {

template <int D, typename R, int MODE, typename V>
void launch_face_one(const Params<D, R> &P, cudaStream_t st)
{
    const dim3 g(unsigned((P.nx + 1 + V::TX - 1) / V::TX), D == 2 ? unsigned((P.ny + 1 + V::TY - 1) / V::TY) : 1u);
    if constexpr (V::TMA) {
        // the tensor maps of the buffer that holds the state now; without them (a grid whose
        // rows are not 16-byte multiples) the same tile stages every cell per thread
        if (P.stage_maps) {
            for (int b = 0; b < 2; ++b)
                if (P.stage_maps[b].key == P.sf) {
                    face_tma_kernel<D, R, MODE, V><<<g, V::THREADS, 0, st>>>(P, P.stage_maps[b]);
                    return;
                }
        }
    }
    face_kernel<D, R, MODE, V><<<g, V::THREADS, 0, st>>>(P);
}

template <int D, typename R, int MODE, typename V, typename... Rest>
void launch_face_at(int v, const Params<D, R> &P, cudaStream_t st)
{
    if constexpr (sizeof...(Rest) == 0) {
        launch_face_one<D, R, MODE, V>(P, st);
    } else {
        if (v <= 0) launch_face_one<D, R, MODE, V>(P, st);
        else launch_face_at<D, R, MODE, Rest...>(v - 1, P, st);
    }
}

template <int D, typename R, int MODE, typename L>
struct FaceLaunch;
template <int D, typename R, int MODE, typename... Vs>
struct FaceLaunch<D, R, MODE, VList<Vs...>> {
    static void launch(int v, const Params<D, R> &P, cudaStream_t st) { launch_face_at<D, R, MODE, Vs...>(v, P, st); }
};

// the face kernel of variant v in one mode; the pair-collecting kernel exists for variant 0
template <int D, typename R, int MODE>
void launch_face_m(int v, const Params<D, R> &P, cudaStream_t st)
{
    if constexpr (MODE == FACE_COLLECT || MODE == FACE_EQUIL) {
        using V0 = FaceVariant<D, D == 2 ? 32 : 128, 4, D == 2 && sizeof(R) == 4 ? 2 : 1>;
        launch_face_one<D, R, MODE, V0>(P, st);
    } else {
        FaceLaunch<D, R, MODE, typename FaceList<D, R>::type>::launch(v, P, st);
    }
}

template <int D, typename R>
void launch_cell(int v, const Params<D, R> &P, cudaStream_t st)
{
    const long long n = P.ncell();
    auto blocks = [&](int t) { return unsigned((n + t - 1) / t); };
    // grid-stride variants: at most one wave at full thread occupancy (2048 threads per SM)
    auto gs_blocks = [&](int t) {
        const long long need = (n + t - 1) / t, cap = (long long)(P.sms > 0 ? P.sms : 1) * (2048 / t);
        return unsigned(need < cap ? need : cap);
    };
    switch (v) {
    case 7: cell_kernel<D, R, 128, 3, false, true><<<gs_blocks(128), 128, 0, st>>>(P); break;
    case 8: cell_kernel<D, R, 128, 1, false, true><<<gs_blocks(128), 128, 0, st>>>(P); break;
    case 1: cell_kernel<D, R, 128><<<blocks(128), 128, 0, st>>>(P); break;
    case 2: cell_kernel<D, R, 512><<<blocks(512), 512, 0, st>>>(P); break;
    case 3: cell_kernel<D, R, 256, 3><<<blocks(256), 256, 0, st>>>(P); break;
    case 4: cell_kernel<D, R, 256, 4><<<blocks(256), 256, 0, st>>>(P); break;
    case 5: cell_kernel<D, R, 128, 6><<<blocks(128), 128, 0, st>>>(P); break;
    case 6: cell_kernel<D, R, 32><<<blocks(32), 32, 0, st>>>(P); break;
    default: cell_kernel<D, R, 256><<<blocks(256), 256, 0, st>>>(P); break;
    }
}

template <int D, typename R, typename V>
void launch_step_one(const Params<D, R> &P, cudaStream_t st)
{
    const dim3 g(unsigned((P.nx + V::TX - 1) / V::TX), D == 2 ? unsigned((P.ny + V::TY - 1) / V::TY) : 1u);
    step_kernel<D, R, V><<<g, V::THREADS, 0, st>>>(P);
}
template <int D, typename R, typename V, typename... Rest>
void launch_step_at(int v, const Params<D, R> &P, cudaStream_t st)
{
    if constexpr (sizeof...(Rest) == 0) {
        launch_step_one<D, R, V>(P, st);
    } else {
        if (v <= 0) launch_step_one<D, R, V>(P, st);
        else launch_step_at<D, R, Rest...>(v - 1, P, st);
    }
}
template <int D, typename R, typename L>
struct StepLaunch;
template <int D, typename R, typename... Vs>
struct StepLaunch<D, R, VList<Vs...>> {
    static void launch(int v, const Params<D, R> &P, cudaStream_t st) { launch_step_at<D, R, Vs...>(v, P, st); }
};
template <int D, typename R>
void launch_step_fused(int v, const Params<D, R> &P, cudaStream_t st)
{
    StepLaunch<D, R, typename StepList<D, R>::type>::launch(v, P, st);
}

template <int D, typename R>
void launch_cell_eq(const Params<D, R> &P, cudaStream_t st)
{
    const long long n = P.ncell();
    cell_kernel<D, R, 256, 1, true><<<unsigned((n + 255) / 256), 256, 0, st>>>(P);
}

template <typename R>
void launch_tube(int v, unsigned n_tubes, const TubeParams<R> &P, int steps, int cur, cudaStream_t st)
{
    if constexpr (sizeof(R) == 4) {
        switch (v) {
        case 1: tube_kernel<R, 64, 8><<<n_tubes, 64, 0, st>>>(P, steps, cur); break;
        case 2: tube_kernel<R, 256, 2><<<n_tubes, 256, 0, st>>>(P, steps, cur); break;
        case 3: tube_kernel<R, 256, 3><<<n_tubes, 256, 0, st>>>(P, steps, cur); break;
        case 4: tube_kernel<R, 128, 6><<<n_tubes, 128, 0, st>>>(P, steps, cur); break;
        default: tube_kernel<R, 128, 4><<<n_tubes, 128, 0, st>>>(P, steps, cur); break;
        }
    } else {
        switch (v) {
        case 1: tube_kernel<R, 128, 2><<<n_tubes, 128, 0, st>>>(P, steps, cur); break;
        case 2: tube_kernel<R, 64, 4><<<n_tubes, 64, 0, st>>>(P, steps, cur); break;
        default: tube_kernel<R, 256, 1><<<n_tubes, 256, 0, st>>>(P, steps, cur); break;
        }
    }
}

}  // namespace pond
