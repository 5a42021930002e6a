// pond_core.cuh -- device arithmetic of the regularized PonD step, in Hermite-coefficient
// form.
//
// A population set f_i on the D1Q4 / D2Q16 lattice (Table I, Eq. wi) in a frame
// lambda = (u, T) is held through its Hermite moments A_rs = sum_i f_i He_r(c_ix) He_s(c_iy)
// (probabilists' Hermite polynomials, T_L = 1).  The Grad projection of Eq. (f_transformed)
// is exactly the truncation of that expansion to r + s <= 3 (f) or <= 2 (g):
//     f_i = W_i sum_{r+s<=N} A_rs He_r(c_ix) He_s(c_iy) / (r! s!).
// The regularized change of frame of Sec. II.C keeps the moments of order <= N (Eq.
// Mcondition); with xi = (v - u')/sqrt(T') = s c + d, s = sqrt(T/T'), d = (u - u')/sqrt(T'),
// the new coefficients are A'_rs = sum_{p<=r, q<=s} X(r,p) Y(s,q) A_pq, where X and Y are the
// one-dimensional lower-triangular maps of He_r(s c + d) onto He_p(c) along x and y
// (derived from He_r(x) = x^r - ...; see the factors below).  Writing them with
// (s^2 - 1) and d keeps the identity transform free of cancellation.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pond {

// ---------------------------------------------------------------- lattice constants
// D1Q4 (Table I): nodes +-sqrt(3 -+ sqrt 6), weights (3 +- sqrt 6)/12, T_L = 1.
constexpr double kCLo = 0x1.7be2ad58cb100p-1;  // sqrt(3 - sqrt 6)
constexpr double kCHi = 0x1.2ace15c98aa9fp+1;  // sqrt(3 + sqrt 6)
constexpr double kWLo = 0x1.d105eb806161fp-2;  // (3 + sqrt 6)/12, weight of +-kCLo
constexpr double kWHi = 0x1.77d0a3fcf4f0bp-5;  // (3 - sqrt 6)/12, weight of +-kCHi

// node m = 0..3 in increasing order
__host__ __device__ constexpr double node_c(int m) { return m == 0 ? -kCHi : m == 1 ? -kCLo : m == 2 ? kCLo : kCHi; }
__host__ __device__ constexpr double node_w(int m) { return (m == 0 || m == 3) ? kWHi : kWLo; }
// He_k(c_m)
__host__ __device__ constexpr double he(int k, int m)
{
    return k == 0 ? 1.0 : k == 1 ? node_c(m) : k == 2 ? node_c(m) * node_c(m) - 1.0
                                                      : node_c(m) * node_c(m) * node_c(m) - 3.0 * node_c(m);
}
// He_k(c_m) / k!
__host__ __device__ constexpr double hen(int k, int m)
{
    return k == 0 ? 1.0 : k == 1 ? he(1, m) : k == 2 ? he(2, m) * 0.5 : he(3, m) * (1.0 / 6.0);
}

// node tables for loops over m that are not unrolled: c_m, He_a(c_m)/a!, w_m He_a(c_m)
template <typename R>
struct NodeTab {
    R c[4];
    R hen[4][4];
    R whe[4][4];
};
#define POND_NODE_TAB(T)                                                                               \
    {{T(node_c(0)), T(node_c(1)), T(node_c(2)), T(node_c(3))},                                         \
     {{T(hen(0, 0)), T(hen(1, 0)), T(hen(2, 0)), T(hen(3, 0))},                                        \
      {T(hen(0, 1)), T(hen(1, 1)), T(hen(2, 1)), T(hen(3, 1))},                                        \
      {T(hen(0, 2)), T(hen(1, 2)), T(hen(2, 2)), T(hen(3, 2))},                                        \
      {T(hen(0, 3)), T(hen(1, 3)), T(hen(2, 3)), T(hen(3, 3))}},                                       \
     {{T(node_w(0) * he(0, 0)), T(node_w(0) * he(1, 0)), T(node_w(0) * he(2, 0)), T(node_w(0) * he(3, 0))}, \
      {T(node_w(1) * he(0, 1)), T(node_w(1) * he(1, 1)), T(node_w(1) * he(2, 1)), T(node_w(1) * he(3, 1))}, \
      {T(node_w(2) * he(0, 2)), T(node_w(2) * he(1, 2)), T(node_w(2) * he(2, 2)), T(node_w(2) * he(3, 2))}, \
      {T(node_w(3) * he(0, 3)), T(node_w(3) * he(1, 3)), T(node_w(3) * he(2, 3)), T(node_w(3) * he(3, 3))}}}
static __constant__ NodeTab<float> kTabF = POND_NODE_TAB(float);
static __constant__ NodeTab<double> kTabD = POND_NODE_TAB(double);
template <typename R> __device__ __forceinline__ const NodeTab<R> &node_tab();
template <> __device__ __forceinline__ const NodeTab<float> &node_tab<float>() { return kTabF; }
template <> __device__ __forceinline__ const NodeTab<double> &node_tab<double>() { return kTabD; }

// index of A_rs (r + s <= 3) in the packed 2D coefficient array: order n = r + s blocks,
// s increasing inside a block: 00 | 10 01 | 20 11 02 | 30 21 12 03
__host__ __device__ constexpr int hidx(int r, int s) { return (r + s) * (r + s + 1) / 2 + s; }
template <int D, int N> struct NCoef;
template <int N> struct NCoef<1, N> { static constexpr int value = N + 1; };
template <int N> struct NCoef<2, N> { static constexpr int value = (N + 1) * (N + 2) / 2; };

// ------------------------------------------------------------ one-dimensional map
// Entries T(r, p) of He_r(s c + d) = sum_p T(r,p) He_p(c) for r <= 3, in terms of
// s, e = s^2 - 1 and d:
//   T00 = 1
//   T10 = d,              T11 = s
//   T20 = e + d^2,        T21 = 2 s d,           T22 = s^2
//   T30 = d (3 e + d^2),  T31 = 3 s (e + d^2),   T32 = 3 s^2 d,   T33 = s^3
template <typename R>
struct Map1 {
    R t10, t11, t20, t21, t22, t30, t31, t32, t33;
    __device__ __forceinline__ Map1(R s, R e, R d)
    {
        const R d2 = d * d, s2 = e + R(1);
        t10 = d;
        t11 = s;
        t20 = e + d2;
        t21 = R(2) * s * d;
        t22 = s2;
        t30 = d * (R(3) * e + d2);
        t31 = R(3) * s * (e + d2);
        t32 = R(3) * s2 * d;
        t33 = s2 * s;
    }
    __device__ __forceinline__ R get(int r, int p) const
    {
        // r and p are compile-time constants after unrolling
        if (p > r) return R(0);
        if (r == 0) return R(1);
        if (r == 1) return p == 0 ? t10 : t11;
        if (r == 2) return p == 0 ? t20 : (p == 1 ? t21 : t22);
        return p == 0 ? t30 : (p == 1 ? t31 : (p == 2 ? t32 : t33));
    }
};

// 1D: out_r = sum_{p<=r} X(r,p) in_p, r <= N.  Z1: in_1 is known to be zero (coefficients in
// the frame of their own first moment) and its terms are skipped.
template <int N, typename R, bool Z1 = false>
__device__ __forceinline__ void shift_scale_1d(const R *in, const Map1<R> &X, R *out)
{
#pragma unroll
    for (int r = 0; r <= N; ++r) {
        R acc = R(0);
#pragma unroll
        for (int p = 0; p <= r; ++p)
            if (!(Z1 && p == 1)) acc += X.get(r, p) * in[p];
        out[r] = acc;
    }
}

// 2D: out_rs = sum_{p<=r} X(r,p) sum_{q<=s} Y(s,q) in_pq, r + s <= N.  Z1: in_10 = in_01 = 0;
// their terms are skipped, and so is the intermediate B_10 (= Y(0,0) in_10 = 0).
template <int N, typename R, bool Z1 = false>
__device__ __forceinline__ void shift_scale_2d(const R *in, const Map1<R> &X, const Map1<R> &Y, R *out)
{
    R B[NCoef<2, N>::value];
#pragma unroll
    for (int p = 0; p <= N; ++p)
#pragma unroll
        for (int s = 0; s + p <= N; ++s) {
            R acc = R(0);
#pragma unroll
            for (int q = 0; q <= s; ++q)
                if (!(Z1 && p + q == 1)) acc += Y.get(s, q) * in[hidx(p, q)];
            B[hidx(p, s)] = acc;
        }
#pragma unroll
    for (int r = 0; r <= N; ++r)
#pragma unroll
        for (int s = 0; s + r <= N; ++s) {
            R acc = R(0);
#pragma unroll
            for (int p = 0; p <= r; ++p)
                if (!(Z1 && p == 1 && s == 0)) acc += X.get(r, p) * B[hidx(p, s)];
            out[hidx(r, s)] = acc;
        }
}

template <int D, int N, typename R, bool Z1 = false>
__device__ __forceinline__ void shift_scale(const R *in, const Map1<R> &X, const Map1<R> &Y, R *out)
{
    if constexpr (D == 1) shift_scale_1d<N, R, Z1>(in, X, out);
    else shift_scale_2d<N, R, Z1>(in, X, Y, out);
}

// ----------------------------------------------- reciprocal, square root, division
// In the working precision R of the step kernels.  FP64: the IEEE operations.  FP32: the
// single-instruction approximations of PTX (rcp.approx, sqrt.approx), whose relative
// error is a few units in the last place over the normal range; they keep the corrector's
// inner loops free of the multi-instruction IEEE sequences and their slow-path branches.
// The FP32 path is held to its tolerance against the FP64 oracle, not to IEEE rounding.
template <typename R> __device__ __forceinline__ R w_rcp(R x) { return R(1) / x; }
template <typename R> __device__ __forceinline__ R w_sqrt(R x) { return sqrt(x); }
template <typename R> __device__ __forceinline__ R w_div(R a, R b) { return a / b; }
template <> __device__ __forceinline__ float w_rcp<float>(float x)
{
    float r;
    asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
template <> __device__ __forceinline__ float w_sqrt<float>(float x)
{
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
template <> __device__ __forceinline__ float w_div<float>(float a, float b) { return a * w_rcp<float>(b); }

// Sum of a small non-negative count over the 32 lanes of a warp (every lane calls it) in one
// warp-reduce instruction; the warp's total must fit in 32 bits.
template <typename T>
__device__ __forceinline__ T warp_sum_count(T x)
{
    return T(__reduce_add_sync(0xffffffffu, (unsigned int)x));
}

// --------------------------------------------------------------------- limiters
// Slope limiters of Sec. III.B.3 on one-sided differences a (upstream) and b (downstream).
template <typename R>
__device__ __forceinline__ R vanleer(R a, R b)
{
    // (sgn a + sgn b)|a||b|/(|a|+|b|) = 2ab/(a+b) when ab > 0, else 0
    const R ab = a * b;
    if constexpr (sizeof(R) == 4) return ab > R(0) ? __fdividef(R(2) * ab, a + b) : R(0);
    else return ab > R(0) ? R(2) * ab / (a + b) : R(0);
}
template <typename R>
__device__ __forceinline__ R minmod(R a, R b)
{
    if (a * b <= R(0)) return R(0);
    return fabs(a) < fabs(b) ? a : b;
}
template <typename R>
__device__ __forceinline__ R limit(int kind, R a, R b) { return kind == 1 ? minmod(a, b) : vanleer(a, b); }

__device__ __forceinline__ bool finite_d(double x) { return isfinite(x); }

}  // namespace pond
