// pond_launch.cuh -- the compiled variants of the step kernels: lists, names and the
// declarations of their launchers.
//
// These lists are the autotuner's search space: tile shapes of the face kernel (cells per
// CTA, CTAs per SM), block sizes of the cell kernel, and thread counts of the persistent
// tube kernel.  Entry 0 of each list is the default used before (or without) tuning.  The
// launchers are defined in pond_variants.cuh and instantiated in separate translation
// units (pond_v*.cu), so the heavy kernels compile in parallel.
#pragma once

#include <cstdio>

#include "pond_batch.cuh"

namespace pond {

template <typename... Vs>
struct VList {
    static constexpr int size = sizeof...(Vs);
};

// ---------------------------------------------------------------- face kernel

template <int D, typename R>
struct FaceList;
template <>
struct FaceList<2, float> {
    using type = VList<FaceVariant<2, 32, 4, 2>, FaceVariant<2, 16, 8, 2>, FaceVariant<2, 64, 2, 2>,
                       FaceVariant<2, 16, 4, 4>, FaceVariant<2, 32, 4, 1>, FaceVariant<2, 16, 8, 3>,
                       FaceVariant<2, 16, 4, 6>, FaceVariant<2, 8, 8, 4>, FaceVariant<2, 8, 8, 4, 1>,
                       FaceVariant<2, 8, 8, 4, 2>, FaceVariant<2, 16, 4, 4, 2>, FaceVariant<2, 8, 8, 4, 1, true>,
                       FaceVariant<2, 8, 8, 3, 1, true>, FaceVariant<2, 8, 8, 4, 2, true>>;
};
template <>
struct FaceList<2, double> {
    using type = VList<FaceVariant<2, 32, 4, 1>, FaceVariant<2, 16, 8, 1>, FaceVariant<2, 16, 4, 2>, FaceVariant<2, 8, 8, 2>>;
};
template <typename R>
struct FaceList<1, R> {
    using type = VList<FaceVariant<1, 128, 1, 1>, FaceVariant<1, 64, 1, 2>, FaceVariant<1, 256, 1, 1>,
                       FaceVariant<1, 32, 1, 8>>;
};

template <int D, typename R, typename V, typename... Rest>
void face_name_at(int v, char *buf, size_t n)
{
    if (v <= 0 || sizeof...(Rest) == 0) {
        if (D == 2)
            std::snprintf(buf, n, "face %dx%d cells, %d threads, %d CTA/SM%s%s", V::TX, V::TY, V::THREADS, V::MINB,
                          V::SCR == 1 ? ", centre cells in shared scratch"
                                      : V::SCR == 2 ? ", centre cells and moment sums in shared scratch" : "",
                          V::TMA ? ", TMA staging" : "");
        else std::snprintf(buf, n, "face %d cells, %d threads, %d CTA/SM", V::TX, V::THREADS, V::MINB);
    } else if constexpr (sizeof...(Rest) > 0) {
        face_name_at<D, R, Rest...>(v - 1, buf, n);
    }
}

template <int D, typename R, typename L>
struct FaceNames;
template <int D, typename R, typename... Vs>
struct FaceNames<D, R, VList<Vs...>> {
    static void name(int v, char *buf, size_t n) { face_name_at<D, R, Vs...>(v, buf, n); }
};

template <int D, typename R>
constexpr int face_variants() { return FaceList<D, R>::type::size; }

// the face kernel of variant v in one mode (FACE_PLAIN, FACE_COLLECT: variant 0 only,
// FACE_LEARNED: D2Q16 only), defined in pond_variants.cuh and instantiated in the pond_v*.cu
// translation units
template <int D, typename R, int MODE>
void launch_face_m(int v, const Params<D, R> &P, cudaStream_t st);

// the face kernel of variant v: pair-collecting with collect, else learned when the
// parameters ask for the learned predictor, else plain
template <int D, typename R>
inline void launch_face(int v, bool collect, const Params<D, R> &P, cudaStream_t st)
{
    if (P.equilibrate) return launch_face_m<D, R, FACE_EQUIL>(0, P, st);
    if constexpr (D == 2) {
        if (collect) return launch_face_m<D, R, FACE_COLLECT>(0, P, st);
        if (P.use_learned) return launch_face_m<D, R, FACE_LEARNED>(v, P, st);
    }
    launch_face_m<D, R, FACE_PLAIN>(v, P, st);
}

// ---------------------------------------------------------------- fused step kernel

template <int D, typename R>
struct StepList;
template <>
struct StepList<2, float> {
    using type = VList<StepVariant<2, 8, 8, 3>, StepVariant<2, 16, 4, 3>, StepVariant<2, 8, 4, 5>, StepVariant<2, 8, 8, 2>>;
};
template <>
struct StepList<2, double> {
    using type = VList<StepVariant<2, 8, 4, 2>, StepVariant<2, 4, 4, 4>>;
};
template <typename R>
struct StepList<1, R> {
    using type = VList<StepVariant<1, 124, 1, 4>, StepVariant<1, 60, 1, 8>>;
};

template <int D, typename R>
constexpr int step_variants() { return StepList<D, R>::type::size; }

template <int D, typename R, typename V, typename... Rest>
void step_name_at(int v, char *buf, size_t n)
{
    if (v <= 0 || sizeof...(Rest) == 0) {
        if (D == 2) std::snprintf(buf, n, "step %dx%d cells fused, %d threads, %d CTA/SM", V::TX, V::TY, V::THREADS, V::MINB);
        else std::snprintf(buf, n, "step %d cells fused, %d threads, %d CTA/SM", V::TX, V::THREADS, V::MINB);
    } else if constexpr (sizeof...(Rest) > 0) {
        step_name_at<D, R, Rest...>(v - 1, buf, n);
    }
}
template <int D, typename R, typename L>
struct StepNames;
template <int D, typename R, typename... Vs>
struct StepNames<D, R, VList<Vs...>> {
    static void name(int v, char *buf, size_t n) { step_name_at<D, R, Vs...>(v, buf, n); }
};

// the fused step kernel of variant v (defined in pond_variants.cuh, instantiated in pond_vfused.cu)
template <int D, typename R>
void launch_step_fused(int v, const Params<D, R> &P, cudaStream_t st);

// ---------------------------------------------------------------- cell kernel

constexpr int kCellBlocks[9] = {256, 128, 512, 256, 256, 128, 32, 128, 128};
constexpr int kCellMinBlocks[9] = {1, 1, 1, 3, 4, 6, 1, 3, 1};   // CTAs per SM asked of the register allocator
constexpr bool kCellGridStride[9] = {false, false, false, false, false, false, false, true, true};
constexpr int kCellVariants = 9;

template <int D, typename R>
void launch_cell(int v, const Params<D, R> &P, cudaStream_t st);

// the cell kernel with the equilibration alternative in the flux (default block size)
template <int D, typename R>
void launch_cell_eq(const Params<D, R> &P, cudaStream_t st);

// the cell kernel of variant v, or the equilibration one when the parameters ask for it
template <int D, typename R>
inline void launch_cell_any(int v, const Params<D, R> &P, cudaStream_t st)
{
    if (P.equilibrate) launch_cell_eq<D, R>(P, st);
    else launch_cell<D, R>(v, P, st);
}

inline void cell_name(int v, char *buf, size_t n)
{
    const int k = (v >= 0 && v < kCellVariants) ? v : 0;
    const char *gs = kCellGridStride[k] ? ", grid-stride" : "";
    if (kCellMinBlocks[k] > 1) std::snprintf(buf, n, "cell %d threads, %d CTA/SM%s", kCellBlocks[k], kCellMinBlocks[k], gs);
    else std::snprintf(buf, n, "cell %d threads%s", kCellBlocks[k], gs);
}

// ---------------------------------------------------------------- tube kernel

template <typename R>
constexpr int tube_variants() { return sizeof(R) == 4 ? 5 : 3; }

template <typename R>
void launch_tube(int v, unsigned n_tubes, const TubeParams<R> &P, int steps, int cur, cudaStream_t st);

template <typename R>
void tube_name(int v, char *buf, size_t n)
{
    static const int f32[5][2] = {{128, 4}, {64, 8}, {256, 2}, {256, 3}, {128, 6}},
                     f64[3][2] = {{256, 1}, {128, 2}, {64, 4}};
    const int k = (v >= 0 && v < tube_variants<R>()) ? v : 0;
    const int *c = sizeof(R) == 4 ? f32[k] : f64[k];
    std::snprintf(buf, n, "tube %d threads, %d CTA/SM", c[0], c[1]);
}

}  // namespace pond
