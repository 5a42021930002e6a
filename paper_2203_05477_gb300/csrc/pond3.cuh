// pond3.cuh -- the finite-volume step on D3Q64 grids: the tensor product of the D1Q4 rule
// (Table I) in three dimensions, the extension the paper names as future work (Sec. V,
// with the slow-moment count q = 20 of Sec. II.C for D = 3).
//
// The arithmetic is that of the D1Q4/D2Q16 kernels with a third axis.  A population set is
// held through its Hermite coefficients A_rst = sum_i f_i He_r(c_ix) He_s(c_iy) He_t(c_iz)
// (r + s + t <= 3 for f: 20 coefficients; <= 2 for g: 10), and the regularized change of
// frame (Sec. II.C) is the product of three one-dimensional lower-triangular maps.
//
// Data layout (structure of arrays, x fastest, then y):
//   cell state : f coefficients in the cell's own frame without the three (zero) first-order
//                ones (17 planes), g coefficients (10 planes), frame (ux, uy, uz, T) as
//                frame words (FP64, or float-float pairs with FP32 populations);
//   faces      : per axis, the face populations' coefficients in the face frame (20 + 10
//                planes) and that frame (4 words), which also seeds the next step's corrector.
// x-face (i, j, k) lies between cells (i-1, j, k) and (i, j, k), i = 0..nx, and likewise for
// y- and z-faces.
//
// Per step (Sec. III.B.4): face3_kernel (steps 2a-2b for the faces of all three axes), then
// cell3_kernel (step 3 fused with step 1 of the next step and the CFL time step).
#pragma once

#include "pond_kernels.cuh"

namespace pond {

// ------------------------------------------------------------ coefficient packing

// index of A_rst in the packed array: blocks of order n = r + s + t; inside a block the
// pairs (s, t) by j = s + t, then t: 000 | 100 010 001 | 200 110 101 020 011 002 | ...
__host__ __device__ constexpr int h3idx(int r, int s, int t)
{
    return (r + s + t) * (r + s + t + 1) * (r + s + t + 2) / 6 + (s + t) * (s + t + 1) / 2 + t;
}
// (s, t) index once the first axis is collapsed
__host__ __device__ constexpr int h2st(int s, int t) { return (s + t) * (s + t + 1) / 2 + t; }
template <int N>
struct NC3 {
    static constexpr int value = (N + 1) * (N + 2) * (N + 3) / 6;
};
constexpr int kNF3 = NC3<3>::value, kNG3 = NC3<2>::value, kNFS3 = kNF3 - 3;

// orders (r, s, t) of packed index k
__host__ __device__ constexpr int h3r(int k)
{
    for (int r = 0; r <= 3; ++r)
        for (int s = 0; r + s <= 3; ++s)
            for (int t = 0; r + s + t <= 3; ++t)
                if (h3idx(r, s, t) == k) return r;
    return 0;
}
__host__ __device__ constexpr int h3s(int k)
{
    for (int r = 0; r <= 3; ++r)
        for (int s = 0; r + s <= 3; ++s)
            for (int t = 0; r + s + t <= 3; ++t)
                if (h3idx(r, s, t) == k) return s;
    return 0;
}
__host__ __device__ constexpr int h3t(int k)
{
    for (int r = 0; r <= 3; ++r)
        for (int s = 0; r + s <= 3; ++s)
            for (int t = 0; r + s + t <= 3; ++t)
                if (h3idx(r, s, t) == k) return t;
    return 0;
}

// stored f plane of coefficient k (-1: a first-order one, zero in the cell's own frame)
__host__ __device__ constexpr int fplane3(int k) { return k == 0 ? 0 : (k <= 3 ? -1 : k - 3); }

// out_rst = sum_{p<=r} X(r,p) sum_{q<=s} Y(s,q) sum_{w<=t} Z(t,w) in_pqw, r + s + t <= N.
// Z1: the first-order inputs are known to be zero (coefficients in the frame of their own
// first moment); their terms are skipped, and so are the intermediates they alone feed
// (B_100 = B_010 = 0 after the z stage, C_100 = 0 after the y stage).
template <int N, typename R, bool Z1 = false>
__device__ __forceinline__ void shift_scale_3d(const R *in, const Map1<R> &X, const Map1<R> &Y, const Map1<R> &Z, R *out)
{
    R B[NC3<N>::value], C[NC3<N>::value];
#pragma unroll
    for (int p = 0; p <= N; ++p)
#pragma unroll
        for (int q = 0; p + q <= N; ++q)
#pragma unroll
            for (int t = 0; p + q + t <= N; ++t) {
                R acc = R(0);
#pragma unroll
                for (int w = 0; w <= t; ++w)
                    if (!(Z1 && p + q + w == 1)) acc += Z.get(t, w) * in[h3idx(p, q, w)];
                B[h3idx(p, q, t)] = acc;
            }
#pragma unroll
    for (int p = 0; p <= N; ++p)
#pragma unroll
        for (int s = 0; p + s <= N; ++s)
#pragma unroll
            for (int t = 0; p + s + t <= N; ++t) {
                R acc = R(0);
#pragma unroll
                for (int q = 0; q <= s; ++q)
                    if (!(Z1 && t == 0 && p + q == 1)) acc += Y.get(s, q) * B[h3idx(p, q, t)];
                C[h3idx(p, s, t)] = acc;
            }
#pragma unroll
    for (int r = 0; r <= N; ++r)
#pragma unroll
        for (int s = 0; r + s <= N; ++s)
#pragma unroll
            for (int t = 0; r + s + t <= N; ++t) {
                R acc = R(0);
#pragma unroll
                for (int p = 0; p <= r; ++p)
                    if (!(Z1 && p == 1 && s == 0 && t == 0)) acc += X.get(r, p) * C[h3idx(p, s, t)];
                out[h3idx(r, s, t)] = acc;
            }
}

// Faces work in face axes (normal, first tangential, second tangential), the tangential
// axes being the other two in increasing order: x-face (x, y, z), y-face (y, x, z),
// z-face (z, x, y).  lab axis of face axis q:
__host__ __device__ __forceinline__ int face_axis(int dir, int q) { return q == 0 ? dir : (q == 1 ? (dir == 0 ? 1 : 0) : (dir == 2 ? 1 : 2)); }
// lab index of face-axis orders (r, s, t)
__host__ __device__ __forceinline__ int lab_of_face(int dir, int r, int s, int t)
{
    return dir == 0 ? h3idx(r, s, t) : (dir == 1 ? h3idx(s, r, t) : h3idx(s, t, r));
}
// lab index of face-axis coefficient k, per face axis (a warp-uniform constant-bank read)
struct FacePerm {
    signed char k[3][kNF3];
};
__host__ __device__ constexpr FacePerm make_face_perm()
{
    FacePerm P{};
    for (int d = 0; d < 3; ++d)
        for (int r = 0; r <= 3; ++r)
            for (int s = 0; r + s <= 3; ++s)
                for (int t = 0; r + s + t <= 3; ++t)
                    P.k[d][h3idx(r, s, t)] = (signed char)(d == 0 ? h3idx(r, s, t) : (d == 1 ? h3idx(s, r, t) : h3idx(s, t, r)));
    return P;
}
static __constant__ FacePerm kFacePerm = make_face_perm();

// the first NC3<N> coefficients of a staged cell in face axes (total orders are kept, so the
// g set (N = 2) is the head of the same permutation)
template <int N, typename R>
__device__ __forceinline__ void to_face(const R *lab, R *face, int dir)
{
#pragma unroll
    for (int k = 0; k < NC3<N>::value; ++k) face[k] = lab[kFacePerm.k[dir][k]];
}
// face-axis coefficients back to lab axes, by selects (the destination is a register array)
template <int N, typename R>
__device__ __forceinline__ void from_face(const R *face, R *lab, int dir)
{
#pragma unroll
    for (int r = 0; r <= N; ++r)
#pragma unroll
        for (int s = 0; r + s <= N; ++s)
#pragma unroll
            for (int t = 0; r + s + t <= N; ++t)
                lab[h3idx(r, s, t)] = dir == 0 ? face[h3idx(r, s, t)] : (dir == 1 ? face[h3idx(s, r, t)] : face[h3idx(t, r, s)]);
}

// ------------------------------------------------------------------ parameters

template <typename R>
struct Params3 {
    using W = typename FrameWords<R>::word;
    long long nx, ny, nz;
    double dx, dy, dz;
    int bc[6];                        // x-lo, x-hi, y-lo, y-hi, z-lo, z-hi
    double gamma, Cv, tau;
    R Cv_r, Cvh_r, tol_r;             // Cv, Cv - 3/2 and tol in the working precision
    int limiter;
    int max_iter, fixed_iters;
    R *sf;                            // [17][ncell]
    R *sg;                            // [10][ncell]
    W *sfr;                           // [4][ncell]
    R *ff[3], *fg[3];                 // per face axis: [20][nf], [10][nf]
    W *ffr[3];                        // [4][nf]
    Clock *clock;
    Diag *diag;
    __host__ __device__ long long ncell() const { return nx * ny * nz; }
    __host__ __device__ long long nf(int a) const
    {
        return a == 0 ? (nx + 1) * ny * nz : (a == 1 ? nx * (ny + 1) * nz : nx * ny * (nz + 1));
    }
    __host__ __device__ long long fidx(int a, long long i, long long j, long long k) const
    {
        return a == 0 ? (k * ny + j) * (nx + 1) + i : (a == 1 ? (k * (ny + 1) + j) * nx + i : (k * ny + j) * nx + i);
    }
};

// Ghost-cell rules along each axis (two layers): wrap-around, copy of the nearest cell, or
// the mirror image across a reflective wall (ghost -k mirrors cell k-1, ghost n-1+k mirrors
// cell n-k).  *flip receives the axes (bit a) across which the cell is a mirror image.
template <typename R>
__device__ __forceinline__ long long resolve3(const Params3<R> &P, long long i, long long j, long long k, int *flip)
{
    long long c[3] = {i, j, k};
    const long long n[3] = {P.nx, P.ny, P.nz};
    int fl = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (c[a] >= 0 && c[a] < n[a]) continue;
        const int b = c[a] < 0 ? P.bc[2 * a] : P.bc[2 * a + 1];   // selects: no run-time indexed parameter
        if (b == BC_REFLECTIVE) {
            c[a] = c[a] < 0 ? -1 - c[a] : 2 * n[a] - 1 - c[a];
            c[a] = clampll(c[a], 0, n[a] - 1);
            fl |= 1 << a;
        } else {
            c[a] = b == BC_PERIODIC ? wrapll(c[a], n[a]) : clampll(c[a], 0, n[a] - 1);
        }
    }
    *flip = fl;
    return (c[2] * P.ny + c[1]) * P.nx + c[0];
}

__host__ __device__ constexpr bool mirror_odd3(int k, int flip)
{
    return (((flip & 1) && (h3r(k) & 1)) != 0) != (((flip & 2) && (h3s(k) & 1)) != 0) != (((flip & 4) && (h3t(k) & 1)) != 0);
}

template <typename R>
struct StagedCell3 {
    R A[kNF3];
    R B[kNG3];
    R du[3];   // frame velocity relative to the tile reference (lab axes)
    R T;
    R pad;     // odd size in words: neighbouring threads' cells fall in distinct banks
};

template <typename R>
__device__ __forceinline__ void cell_velocity3(const Params3<R> &P, long long i, long long j, long long k,
                                               typename FrameWords<R>::word *u)
{
    int flip = 0;
    const long long idx = resolve3(P, i, j, k, &flip);
    const long long n = P.ncell();
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        u[a] = P.sfr[a * n + idx];
        if (flip & (1 << a)) u[a] = fr_neg(u[a]);
    }
}

// phi-bar-plus (Eq. Fbarplus) of cell (i, j, k), ghosts resolved: cp phi~ + ce phi^eq
template <typename R>
__device__ __forceinline__ void load_cell3(const Params3<R> &P, long long i, long long j, long long k, R cp, R ce,
                                           const typename FrameWords<R>::word *utile, StagedCell3<R> &c)
{
    using W = typename FrameWords<R>::word;
    int flip = 0;
    const long long idx = resolve3(P, i, j, k, &flip);
    const long long n = P.ncell();
#pragma unroll
    for (int q = 0; q < kNF3; ++q) {
        const int pl = fplane3(q);
        const R v = pl < 0 ? R(0) : P.sf[pl * n + idx];
        c.A[q] = mirror_odd3(q, flip) ? -v : v;
    }
#pragma unroll
    for (int q = 0; q < kNG3; ++q) {
        const R v = P.sg[q * n + idx];
        c.B[q] = mirror_odd3(q, flip) ? -v : v;
    }
    W u[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        u[a] = P.sfr[a * n + idx];
        if (flip & (1 << a)) u[a] = fr_neg(u[a]);
        c.du[a] = R(fr_rel(u[a], utile[a]));
    }
    const R T = R(fr_lead(P.sfr[3 * n + idx]));
    const R r = c.A[0];
    c.A[0] = cp * r + ce * r;
#pragma unroll
    for (int q = 1; q < kNF3; ++q) c.A[q] = cp * c.A[q];
    c.B[0] = cp * c.B[0] + ce * (P.Cvh_r * r * T);
#pragma unroll
    for (int q = 1; q < kNG3; ++q) c.B[q] = cp * c.B[q];
    c.T = T;
}

// ------------------------------------------------------------------ face corrector

// Stencil slots of a face (as in the oracle): 0 LL, 1 L, 2 R, 3 RR along the normal; 4 L-,
// 5 L+, 6 R-, 7 R+ along the first tangential axis; 8 L-, 9 L+, 10 R-, 11 R+ along the
// second.  Offsets in face axes from cell R (normal, first tangential, second tangential).
__device__ __forceinline__ void slot_offset(int s, int &on, int &o1, int &o2)
{
    if (s < 4) {
        on = s - 2;
        o1 = 0;
        o2 = 0;
    } else {
        const int side = ((s - 4) & 3) >> 1;   // 0: L, 1: R
        const int sg = (s & 1) ? 1 : -1;
        on = side - 1;
        o1 = s < 8 ? sg : 0;
        o2 = s < 8 ? 0 : sg;
    }
}

// the staged box of a CTA and the face's place in it
template <typename R>
struct FaceBox {
    const StagedCell3<R> *tile;
    int BX, BY;          // box extents along x and y (lab)
    int bx, by, bz;      // box coordinates of cell R of the face
    int dir;
    __device__ __forceinline__ const StagedCell3<R> *slot(int s) const
    {
        int on, o1, o2;
        slot_offset(s, on, o1, o2);
        // lab offsets by selects (no run-time indexed array)
        const int a1 = face_axis(dir, 1), a2 = face_axis(dir, 2);
        const int ox = (dir == 0 ? on : 0) + (a1 == 0 ? o1 : 0) + (a2 == 0 ? o2 : 0);
        const int oy = (dir == 1 ? on : 0) + (a1 == 1 ? o1 : 0) + (a2 == 1 ? o2 : 0);
        const int oz = (dir == 2 ? on : 0) + (a1 == 2 ? o1 : 0) + (a2 == 2 ? o2 : 0);
        return &tile[((bz + oz) * BY + (by + oy)) * BX + (bx + ox)];
    }
};

// frame maps of a staged cell into the pass frame, in face axes: s = sqrt(Tc/Tl),
// e = s^2 - 1, d = (uc - ul)/sqrt(Tl)
template <typename R>
__device__ __forceinline__ void cell_maps3(const StagedCell3<R> *c, int dir, const R *dref, const R *dl, R Tl, R invTl,
                                           R rsqTl, Map1<R> &X, Map1<R> &Y, Map1<R> &Z)
{
    const R s = sqrt(c->T * invTl);
    const R e = (c->T - Tl) * invTl;
    X = Map1<R>(s, e, (c->du[face_axis(dir, 0)] - dref[0] - dl[0]) * rsqTl);
    Y = Map1<R>(s, e, (c->du[face_axis(dir, 1)] - dref[1] - dl[1]) * rsqTl);
    Z = Map1<R>(s, e, (c->du[face_axis(dir, 2)] - dref[2] - dl[2]) * rsqTl);
}

// One corrector pass at a face (Sec. III.B.3) in frame (dl, Tl) (velocity relative to the
// face reference dref, face axes).  A population (m, n, p) is reconstructed as
// u + off_n lim(u - l, h - u) + off_1 lim(u - t1-, t1+ - u) + off_2 lim(u - t2-, t2+ - u)
// from its upwind cell u, that cell's normal neighbours l, h and its tangential neighbours,
// and only the moments of the reconstructions are kept; they are linear in the three terms,
// so each normal node m runs three sweeps (normal, first and second tangential slope), each
// needing the upwind cell and two neighbours.  The cells are re-expressed in the pass frame,
// collapsed along the normal at c_m and kept in a per-thread shared-memory scratch (3 slots
// of 16 values, slot-major, thread-minor over NT threads).  Phi: moments of f (order 3),
// Psi: of g (order 2), face axes.
template <typename R>
__device__ __forceinline__ void collapse_normal(const StagedCell3<R> *c, int dir, const R *dref, const R *dl, R Tl,
                                                R invTl, R rsqTl, const R *hn, R *slot, int NT)
{
    Map1<R> X(R(1), R(0), R(0)), Y = X, Z = X;
    cell_maps3<R>(c, dir, dref, dl, Tl, invTl, rsqTl, X, Y, Z);
    R tmp[kNF3], F[kNF3];
    to_face<3, R>(c->A, tmp, dir);
    shift_scale_3d<3, R, true>(tmp, X, Y, Z, F);   // staged f: zero first order
#pragma unroll
    for (int s2 = 0; s2 <= 3; ++s2)
#pragma unroll
        for (int t2 = 0; s2 + t2 <= 3; ++t2) {
            R acc = R(0);
#pragma unroll
            for (int r = 0; r + s2 + t2 <= 3; ++r) acc += F[h3idx(r, s2, t2)] * hn[r];
            slot[h2st(s2, t2) * NT] = acc;
        }
    R tg[kNG3], G[kNG3];
    to_face<2, R>(c->B, tg, dir);
    shift_scale_3d<2, R>(tg, X, Y, Z, G);
#pragma unroll
    for (int s2 = 0; s2 <= 2; ++s2)
#pragma unroll
        for (int t2 = 0; s2 + t2 <= 2; ++t2) {
            R acc = R(0);
#pragma unroll
            for (int r = 0; r + s2 + t2 <= 2; ++r) acc += G[h3idx(r, s2, t2)] * hn[r];
            slot[(10 + h2st(s2, t2)) * NT] = acc;
        }
}

// The populations (n, p = 0..3) of one sweep at normal node m, FP32: the three scratch slots
// (upwind cell, two neighbours; normal-collapsed) collapsed along the first tangential axis
// at c_n, evaluated at c_p, reconstructed (plain * upwind + off * limited slope) and their
// moments along the second tangential axis accumulated into S1f (f, orders 0..3) and S1g
// (g, 0..2).  f rides in lane x and g in lane y of FP32x2 pairs for the orders 0..2.
__device__ __forceinline__ void sweep_node_f32(const float *scr, int NT, int n, float off1, bool off_by_p, float plain,
                                               float sqTl, float u2, float h_d2, int limiter, float *S1f, float *S1g)
{
    const NodeTab<float> &tab = node_tab<float>();
    const float h0 = tab.hen[n][0], h1 = tab.hen[n][1], h2 = tab.hen[n][2], h3 = tab.hen[n][3];
    const float2 H0 = bc2(h0), H1 = bc2(h1), H2 = bc2(h2);
    // c[q][t2]: lane x f, lane y g (t2 = 0..2); cf3[q]: f at t2 = 3
    float2 c[3][3];
    float cf3[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float *b = scr + q * 16 * NT;
        auto F = [&](int s2, int t2) { return b[h2st(s2, t2) * NT]; };
        auto G = [&](int s2, int t2) { return b[(10 + h2st(s2, t2)) * NT]; };
        // t2 = 0: f sums s2 = 0..3, g s2 = 0..2
        float2 a0 = __fmul2_rn(make_float2(F(0, 0), G(0, 0)), H0);
        a0 = __ffma2_rn(make_float2(F(1, 0), G(1, 0)), H1, a0);
        a0 = __ffma2_rn(make_float2(F(2, 0), G(2, 0)), H2, a0);
        a0.x += F(3, 0) * h3;
        // t2 = 1: f s2 = 0..2, g s2 = 0..1
        float2 a1 = __fmul2_rn(make_float2(F(0, 1), G(0, 1)), H0);
        a1 = __ffma2_rn(make_float2(F(1, 1), G(1, 1)), H1, a1);
        a1.x += F(2, 1) * h2;
        // t2 = 2: f s2 = 0..1, g s2 = 0
        float2 a2 = __fmul2_rn(make_float2(F(0, 2), G(0, 2)), H0);
        a2.x += F(1, 2) * h1;
        c[q][0] = a0;
        c[q][1] = a1;
        c[q][2] = a2;
        cf3[q] = F(0, 3) * h0;
    }
    float2 S[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    float S3 = 0.f;
    const float2 minus1 = bc2(-1.f);
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const float off = off_by_p ? -(sqTl * float(node_c(p)) + u2) * h_d2 : off1;
        float2 v[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            float2 a = __fmul2_rn(c[q][0], bc2(float(hen(0, p))));
            a = __ffma2_rn(c[q][1], bc2(float(hen(1, p))), a);
            a = __ffma2_rn(c[q][2], bc2(float(hen(2, p))), a);
            a.x += cf3[q] * float(hen(3, p));
            v[q] = a;
        }
        const float2 lim = limit2(limiter, __ffma2_rn(v[1], minus1, v[0]), __ffma2_rn(v[0], minus1, v[2]));
        const float2 b = __ffma2_rn(bc2(off), lim, __fmul2_rn(bc2(plain), v[0]));
#pragma unroll
        for (int t2 = 0; t2 <= 2; ++t2) S[t2] = __ffma2_rn(bc2(float(node_w(p) * he(t2, p))), b, S[t2]);
        S3 += float(node_w(p) * he(3, p)) * b.x;
    }
#pragma unroll
    for (int t2 = 0; t2 <= 2; ++t2) {
        S1f[t2] = S[t2].x;
        S1g[t2] = S[t2].y;
    }
    S1f[3] = S3;
}

template <typename R, int NT>
__device__ __forceinline__ void corrector_pass3(const FaceBox<R> &box, const R *dref, const R *uabs, const R *dl, R Tl,
                                                R h_dn, R h_d1, R h_d2, int limiter, R *scr, R *Phi, R *Psi)
{
    const R invTl = R(1) / Tl;
    const R rsqTl = sqrt(invTl);
    const R sqTl = Tl * rsqTl;
    const NodeTab<R> &tab = node_tab<R>();
#pragma unroll
    for (int q = 0; q < kNF3; ++q) Phi[q] = R(0);
#pragma unroll
    for (int q = 0; q < kNG3; ++q) Psi[q] = R(0);
    const R un = uabs[0] + dl[0], u1 = uabs[1] + dl[1], u2 = uabs[2] + dl[2];
#pragma unroll 1
    for (int m = 0; m < 4; ++m) {
        const R vn = sqTl * tab.c[m] + un;
        const bool left = vn > R(0);
        const R offn = (left ? R(0.5) : R(-0.5)) - vn * h_dn;
        const R hn[4] = {tab.hen[m][0], tab.hen[m][1], tab.hen[m][2], tab.hen[m][3]};
        // scratch slot 0: the upwind cell
        collapse_normal<R>(box.slot(left ? 1 : 2), box.dir, dref, dl, Tl, invTl, rsqTl, hn, scr, NT);
        // moments over the tangential nodes of this normal node, in (s, t)
        R S2f[10], S2g[6];
#pragma unroll
        for (int q = 0; q < 10; ++q) S2f[q] = R(0);
#pragma unroll
        for (int q = 0; q < 6; ++q) S2g[q] = R(0);
#pragma unroll 1
        for (int sw = 0; sw < 3; ++sw) {
            // the two neighbours of the sweep: normal (l, h), then first and second tangential (-, +)
            const int sa = sw == 0 ? (left ? 0 : 1) : (left ? 4 : 6) + 4 * (sw - 1);
            const int sb = sw == 0 ? (left ? 2 : 3) : sa + 1;
            collapse_normal<R>(box.slot(sa), box.dir, dref, dl, Tl, invTl, rsqTl, hn, scr + 16 * NT, NT);
            collapse_normal<R>(box.slot(sb), box.dir, dref, dl, Tl, invTl, rsqTl, hn, scr + 32 * NT, NT);
            const R plain = sw == 0 ? R(1) : R(0);
#pragma unroll 1
            for (int n = 0; n < 4; ++n) {
                const R off1 = sw == 0 ? offn : -(sqTl * tab.c[n] + u1) * h_d1;
                R S1f[4] = {R(0), R(0), R(0), R(0)}, S1g[3] = {R(0), R(0), R(0)};
                if constexpr (sizeof(R) == 4) {
                    // FP32: f in lane x and g in lane y of FP32x2 pairs for the orders both carry
                    // (0..2), f's third order alone
                    sweep_node_f32(scr, NT, n, off1, sw == 2, plain, sqTl, u2, h_d2, limiter, S1f, S1g);
                } else {
                // collapse the three slots along the first tangential axis at c_n
                R cf[3][4], cg[3][3];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
#pragma unroll
                    for (int t2 = 0; t2 <= 3; ++t2) {
                        R acc = R(0);
#pragma unroll
                        for (int s2 = 0; s2 + t2 <= 3; ++s2) acc += scr[(q * 16 + h2st(s2, t2)) * NT] * tab.hen[n][s2];
                        cf[q][t2] = acc;
                    }
#pragma unroll
                    for (int t2 = 0; t2 <= 2; ++t2) {
                        R acc = R(0);
#pragma unroll
                        for (int s2 = 0; s2 + t2 <= 2; ++s2) acc += scr[(q * 16 + 10 + h2st(s2, t2)) * NT] * tab.hen[n][s2];
                        cg[q][t2] = acc;
                    }
                }
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    const R off = sw == 2 ? -(sqTl * R(node_c(p)) + u2) * h_d2 : off1;
                    R fv[3], gv[3];
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        R a = R(0), b = R(0);
#pragma unroll
                        for (int t2 = 0; t2 <= 3; ++t2) a += cf[q][t2] * R(hen(t2, p));
#pragma unroll
                        for (int t2 = 0; t2 <= 2; ++t2) b += cg[q][t2] * R(hen(t2, p));
                        fv[q] = a;
                        gv[q] = b;
                    }
                    const R fb = plain * fv[0] + off * limit<R>(limiter, fv[0] - fv[1], fv[2] - fv[0]);
                    const R gb = plain * gv[0] + off * limit<R>(limiter, gv[0] - gv[1], gv[2] - gv[0]);
#pragma unroll
                    for (int t2 = 0; t2 <= 3; ++t2) S1f[t2] += R(node_w(p) * he(t2, p)) * fb;
#pragma unroll
                    for (int t2 = 0; t2 <= 2; ++t2) S1g[t2] += R(node_w(p) * he(t2, p)) * gb;
                }
                }
#pragma unroll
                for (int s2 = 0; s2 <= 3; ++s2)
#pragma unroll
                    for (int t2 = 0; s2 + t2 <= 3; ++t2) S2f[h2st(s2, t2)] += tab.whe[n][s2] * S1f[t2];
#pragma unroll
                for (int s2 = 0; s2 <= 2; ++s2)
#pragma unroll
                    for (int t2 = 0; s2 + t2 <= 2; ++t2) S2g[h2st(s2, t2)] += tab.whe[n][s2] * S1g[t2];
            }
        }
#pragma unroll
        for (int r = 0; r <= 3; ++r)
#pragma unroll
            for (int s2 = 0; r + s2 <= 3; ++s2)
#pragma unroll
                for (int t2 = 0; r + s2 + t2 <= 3; ++t2) Phi[h3idx(r, s2, t2)] += tab.whe[m][r] * S2f[h2st(s2, t2)];
#pragma unroll
        for (int r = 0; r <= 2; ++r)
#pragma unroll
            for (int s2 = 0; r + s2 <= 2; ++s2)
#pragma unroll
                for (int t2 = 0; r + s2 + t2 <= 2; ++t2) Psi[h3idx(r, s2, t2)] += tab.whe[m][r] * S2g[h2st(s2, t2)];
    }
}

// frame of a pass's moments relative to the pass frame (face axes): rho, du, T
template <typename R>
__device__ __forceinline__ bool pass_frame3(const R *Phi, const R *Psi, R Tl, R Cv, R &rho, R *du, R &T)
{
    rho = Phi[0];
    const R sq = sqrt(Tl);
    du[0] = sq * Phi[h3idx(1, 0, 0)] / rho;
    du[1] = sq * Phi[h3idx(0, 1, 0)] / rho;
    du[2] = sq * Phi[h3idx(0, 0, 1)] / rho;
    const R k2 = du[0] * du[0] + du[1] * du[1] + du[2] * du[2];
    const R tr = Phi[h3idx(2, 0, 0)] + Phi[h3idx(0, 2, 0)] + Phi[h3idx(0, 0, 2)] + R(3) * Phi[0];
    T = (R(0.5) * Tl * tr + Psi[0] - R(0.5) * rho * k2) / (Cv * rho);
    return T > R(0) && isfinite(T) && isfinite(rho) && isfinite(du[0]) && isfinite(du[1]) && isfinite(du[2]);
}

template <typename R>
struct FaceOut3 {
    R F[kNF3];   // face populations' coefficients in the face frame (lab axes)
    R G[kNG3];
    R du[3];     // face frame velocity minus the predictor's (lab axes)
    R T;
    int iters, fallbacks;
    bool done, have;
};

// The predictor-corrector of one face (the readings of the D2Q16 kernel: convergence rule,
// restart once from the pooled moments of the stencil, the last valid pass's moments
// Grad-projected into the frame they define, then Eq. FluxTransf).
constexpr int kKeep3 = 3 * 16;   // first scratch slot of the kept frames (after the corrector's)

template <typename R, int NT>
__device__ __forceinline__ void solve_face3(const FaceBox<R> &box, const R *dref, const R *uabs, R Tpred, R h_dn, R h_d1,
                                            R h_d2, R Cv, R tol, R wb, R we, int limiter, int max_iter, int fixed_iters,
                                            R *scr, FaceOut3<R> &o)
{
    R dl[3] = {R(0), R(0), R(0)}, Tl = Tpred;
    // the last valid pass's frames (its frame dl, Tl, and the frame its moments define: du,
    // T1, rho1) wait in the thread's scratch after the corrector's 3 x 16 values, read and
    // written with volatile accesses, instead of staying live in registers across the passes
    auto kput = [&](int q, R v) { *reinterpret_cast<volatile R *>(&scr[(kKeep3 + q) * NT]) = v; };
    auto kget = [&](int q) -> R { return *reinterpret_cast<volatile R *>(&scr[(kKeep3 + q) * NT]); };
    bool have = false, done = false, restarted = false, last_valid = false, recompute = false;
    int iters = 0;
    o.fallbacks = 0;
    R Phi[kNF3], Psi[kNG3];
    // one call site of the pass: the last iteration of this loop recomputes the last valid
    // pass when the final one defined no frame
    for (int k = 0;; ++k) {
        const bool run = recompute || (k < max_iter && !done);
        if (!run) {
            if (have && !last_valid) {
                recompute = true;
                continue;
            }
            break;
        }
        R dlp[3] = {dl[0], dl[1], dl[2]}, Tlp = Tl;
        if (recompute) {
#pragma unroll
            for (int a = 0; a < 3; ++a) dlp[a] = kget(a);
            Tlp = kget(6);
        }
        corrector_pass3<R, NT>(box, dref, uabs, dlp, Tlp, h_dn, h_d1, h_d2, limiter, scr, Phi, Psi);
        if (recompute) break;
        R rho1, du[3], T1;
        const bool ok = pass_frame3<R>(Phi, Psi, Tl, Cv, rho1, du, T1);
        iters = k + 1;
        if (!ok) {
            ++o.fallbacks;
            last_valid = false;
            if (!restarted) {
                restarted = true;
                R r = R(0), mo[3] = {R(0), R(0), R(0)}, e = R(0);
#pragma unroll 1
                for (int s = 0; s < 12; ++s) {
                    const StagedCell3<R> *c = box.slot(s);
                    const R rc = c->A[0];
                    R v2 = R(0);
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const R d = c->du[face_axis(box.dir, a)] - dref[a];
                        mo[a] += rc * d;
                        v2 += d * d;
                    }
                    r += rc;
                    e += rc * (Cv * c->T + R(0.5) * v2);
                }
                r /= R(12);
                e /= R(12);
                R k2 = R(0);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    mo[a] /= R(12);
                    dl[a] = mo[a] / r;
                    k2 += mo[a] * mo[a];
                }
                Tl = (e - R(0.5) * k2 / r) / (Cv * r);
                continue;
            }
            // stop at the last pass that defined a frame
            done = false;
            max_iter = 0;
            continue;
        }
        have = true;
        last_valid = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            kput(a, dl[a]);
            kput(3 + a, du[a]);
        }
        kput(6, Tl);
        kput(7, T1);
        kput(8, rho1);
        if (fixed_iters > 0) {
            done = iters >= fixed_iters;
        } else {
            const R sq = sqrt(Tl);
            done = fabs(T1 - Tl) <= tol * Tl && fabs(du[0]) <= tol * sq && fabs(du[1]) <= tol * sq && fabs(du[2]) <= tol * sq;
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) dl[a] += du[a];
        Tl = T1;
    }
    o.iters = iters;
    o.done = done;
    o.have = have;
    if (!have) return;
    R keep_dl[3], out_du[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        keep_dl[a] = kget(a);
        out_du[a] = kget(3 + a);
    }
    const R keep_T = kget(6), out_T = kget(7), out_rho = kget(8);
    const R invT = R(1) / out_T, rs = sqrt(invT);
    const R sc = sqrt(keep_T * invT), e = (keep_T - out_T) * invT;
    Map1<R> X(sc, e, -out_du[0] * rs), Y(sc, e, -out_du[1] * rs), Z(sc, e, -out_du[2] * rs);
    R Fo[kNF3], Go[kNG3];
    shift_scale_3d<3, R>(Phi, X, Y, Z, Fo);
    shift_scale_3d<2, R>(Psi, X, Y, Z, Go);
    Fo[0] = wb * Fo[0] + we * out_rho;
#pragma unroll
    for (int q = 1; q < kNF3; ++q) Fo[q] = wb * Fo[q];
    Go[0] = wb * Go[0] + we * (Cv - R(1.5)) * out_rho * out_T;
#pragma unroll
    for (int q = 1; q < kNG3; ++q) Go[q] = wb * Go[q];
    from_face<3, R>(Fo, o.F, box.dir);
    from_face<2, R>(Go, o.G, box.dir);
    // face axes back to lab axes
    const R dn = keep_dl[0] + out_du[0], d1 = keep_dl[1] + out_du[1], d2 = keep_dl[2] + out_du[2];
    const int dir = box.dir;
    o.du[0] = dir == 0 ? dn : d1;
    o.du[1] = dir == 1 ? dn : (dir == 0 ? d1 : d2);
    o.du[2] = dir == 2 ? dn : d2;
    o.T = out_T;
}

// Tiles of the 3D face kernel: TX x TY x TZ cells per CTA, one thread per face of each axis
// (3 TX TY TZ threads), the box [i0-2, i0+TX] x [j0-2, j0+TY] x [k0-2, k0+TZ] staged in
// dynamic shared memory, followed by the per-thread scratch (the corrector's 3 x 16 values and
// the 9 kept-frame values); two CTAs per SM.
template <typename R, int TX_ = 4, int TY_ = 4, int TZ_ = (sizeof(R) == 4 ? 4 : 2), int MINB_ = 2>
struct Face3Tile {
    static constexpr int TX = TX_, TY = TY_, TZ = TZ_;
    static constexpr int THREADS = 3 * TX * TY * TZ;
    static constexpr int MINB = MINB_;
    static constexpr int BX = TX + 3, BY = TY + 3, BZ = TZ + 3;
    static constexpr size_t tile_bytes = sizeof(StagedCell3<R>) * BX * BY * BZ;
    static constexpr size_t scratch_bytes = sizeof(R) * (kKeep3 + 9) * THREADS;
    static constexpr size_t smem = tile_bytes + scratch_bytes;
    static_assert(smem <= 227 * 1024, "the tile and scratch fit one CTA's shared memory");
};

template <typename R, typename V = Face3Tile<R>>
__global__ void __launch_bounds__(V::THREADS, V::MINB)
face3_kernel(const Params3<R> P)
{
    using Tl_ = V;
    constexpr int TX = Tl_::TX, TY = Tl_::TY, TZ = Tl_::TZ, BX = Tl_::BX, BY = Tl_::BY, BZ = Tl_::BZ, NT = Tl_::THREADS;
    using W = typename FrameWords<R>::word;
    extern __shared__ __align__(16) unsigned char f3_dyn[];
    StagedCell3<R> *tile = reinterpret_cast<StagedCell3<R> *>(f3_dyn);
    R *scr = reinterpret_cast<R *>(f3_dyn + Tl_::tile_bytes) + threadIdx.x;
    __shared__ W utile[3];

    const Clock &K = *P.clock;
    // t_end reached (dt = 0): the step is a no-op; tested after the staging loads, so that
    // this load's latency overlaps theirs
    const double step_dt = K.dt;
    const StepC<R> &KC = step_c<R>(K);
    const long long i0 = (long long)blockIdx.x * TX, j0 = (long long)blockIdx.y * TY, k0 = (long long)blockIdx.z * TZ;

    const int dir = threadIdx.x / (TX * TY * TZ);
    const int tl = threadIdx.x - dir * TX * TY * TZ;
    const int tx = tl % TX, ty = (tl / TX) % TY, tz = tl / (TX * TY);
    const long long fi = i0 + tx, fj = j0 + ty, fk = k0 + tz;
    const bool active = fi < P.nx + (dir == 0) && fj < P.ny + (dir == 1) && fk < P.nz + (dir == 2);
    const long long nf = P.nf(dir), f = active ? P.fidx(dir, fi, fj, fk) : 0;
    // selects: a run-time index into the parameter arrays would copy them to local memory
    W *Frm = dir == 0 ? P.ffr[0] : (dir == 1 ? P.ffr[1] : P.ffr[2]);
    // the face's predictor frame, loaded before the staging so that the loads overlap
    W uref[3], Tpw;
#pragma unroll
    for (int a = 0; a < 3; ++a) uref[a] = active ? Frm[a * nf + f] : fr_word(R(0));
    Tpw = active ? Frm[3 * nf + f] : fr_word(R(1));
    // the tile's reference velocity: every thread reads it (the same words), so the
    // staging needs no barrier before it
    W ut[3];
    cell_velocity3<R>(P, i0, j0, k0, ut);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int a = 0; a < 3; ++a) utile[a] = ut[a];
    }
    for (int t = threadIdx.x; t < BX * BY * BZ; t += blockDim.x) {
        const int bx = t % BX, by = (t / BX) % BY, bz = t / (BX * BY);
        load_cell3<R>(P, i0 - 2 + bx, j0 - 2 + by, k0 - 2 + bz, KC.cp, KC.ce, ut, tile[t]);
    }
    if (!(step_dt > 0.0)) return;   // the same value in every thread
    __syncthreads();

    unsigned long long my_iters = 0, my_nonconv = 0, my_fallbacks = 0, my_nonphys = 0;
    if (active) {
        FaceBox<R> box;
        box.tile = tile;
        box.BX = BX;
        box.BY = BY;
        box.bx = tx + 2;
        box.by = ty + 2;
        box.bz = tz + 2;
        box.dir = dir;
        R *Fout = dir == 0 ? P.ff[0] : (dir == 1 ? P.ff[1] : P.ff[2]);
        R *Gout = dir == 0 ? P.fg[0] : (dir == 1 ? P.fg[1] : P.fg[2]);
        const R Tp = R(fr_lead(Tpw));
        // the predictor in face axes (selects: no run-time indexed array)
        const W un_w = dir == 0 ? uref[0] : (dir == 1 ? uref[1] : uref[2]);
        const W u1_w = dir == 0 ? uref[1] : uref[0];
        const W u2_w = dir == 2 ? uref[1] : uref[2];
        const W tn_w = dir == 0 ? utile[0] : (dir == 1 ? utile[1] : utile[2]);
        const W t1_w = dir == 0 ? utile[1] : utile[0];
        const W t2_w = dir == 2 ? utile[1] : utile[2];
        const R dref[3] = {R(fr_rel(un_w, tn_w)), R(fr_rel(u1_w, t1_w)), R(fr_rel(u2_w, t2_w))};
        const R uabs[3] = {R(fr_lead(un_w)), R(fr_lead(u1_w)), R(fr_lead(u2_w))};
        const R h_dn = dir == 0 ? KC.h_dx : (dir == 1 ? KC.h_dy : KC.h_dz);
        const R h_d1 = dir == 0 ? KC.h_dy : KC.h_dx;
        const R h_d2 = dir == 2 ? KC.h_dy : KC.h_dz;
        FaceOut3<R> o;
        solve_face3<R, NT>(box, dref, uabs, Tp, h_dn, h_d1, h_d2, P.Cv_r, P.tol_r, KC.wb, KC.we, P.limiter, P.max_iter,
                           P.fixed_iters, scr, o);
        my_iters = o.iters;
        my_nonconv = o.done ? 0 : 1;
        my_fallbacks = o.fallbacks;
        if (o.have) {
#pragma unroll
            for (int q = 0; q < kNF3; ++q) Fout[q * nf + f] = o.F[q];
#pragma unroll
            for (int q = 0; q < kNG3; ++q) Gout[q * nf + f] = o.G[q];
#pragma unroll
            for (int a = 0; a < 3; ++a) Frm[a * nf + f] = fr_add(uref[a], o.du[a]);
            Frm[3 * nf + f] = fr_word(o.T);
        } else {
            ++my_nonphys;
            const R nan = R(__longlong_as_double(0x7ff8000000000000ll));
#pragma unroll
            for (int q = 0; q < kNF3; ++q) Fout[q * nf + f] = nan;
#pragma unroll
            for (int q = 0; q < kNG3; ++q) Gout[q * nf + f] = nan;
            fr_store(Frm[3 * nf + f], double(nan));
        }
    }
    unsigned long long n_act = active ? 1ull : 0ull;
    my_iters = warp_sum_count(my_iters);
    my_nonconv = warp_sum_count(my_nonconv);
    my_fallbacks = warp_sum_count(my_fallbacks);
    my_nonphys = warp_sum_count(my_nonphys);
    n_act = warp_sum_count(n_act);
    if ((threadIdx.x & 31) == 0 && n_act) {
        atomicAdd(&P.diag->face_iters, my_iters);
        atomicAdd(&P.diag->face_solves, n_act);
        if (my_nonconv) { atomicAdd(&P.diag->nonconv, my_nonconv); atomicOr(&P.diag->flags, FLAG_NOT_CONVERGED); }
        if (my_fallbacks) atomicAdd(&P.diag->fallbacks, my_fallbacks);
        if (my_nonphys) { atomicAdd(&P.diag->nonphys, my_nonphys); atomicOr(&P.diag->flags, FLAG_NONPHYSICAL); }
    }
}

// ---------------------------------------------------------------- cell update

// -scale * H[v_a phi] of one face of axis A added to the cell's moments (H: f, G: g): the
// face populations re-expressed in the cell frame (Eq. fluxEq), times v_a = sqrt(T) c_a + u_a
// by c He_r(c) = He_{r+1}(c) + r He_{r-1}(c) along axis A (He_4 vanishes on the nodes).
template <typename R, int A>
__device__ __forceinline__ void add_face_flux3(const R *Fc, const R *Gc, const R *dv, R Tb, R Tc, R invTc, R rsqTc, R scale,
                                               R sqTc, R un, R *H, R *G)
{
    const R s = sqrt(Tb * invTc), e = (Tb - Tc) * invTc;
    Map1<R> X(s, e, dv[0] * rsqTc), Y(s, e, dv[1] * rsqTc), Z(s, e, dv[2] * rsqTc);
    R Fp[kNF3], Gp[kNG3];
    shift_scale_3d<3, R>(Fc, X, Y, Z, Fp);
    shift_scale_3d<2, R>(Gc, X, Y, Z, Gp);
#pragma unroll
    for (int k = 0; k < kNF3; ++k) {
        const int o[3] = {h3r(k), h3s(k), h3t(k)};
        R v = un * Fp[k];
        if (o[0] + o[1] + o[2] + 1 <= 3)
            v += sqTc * Fp[h3idx(o[0] + (A == 0), o[1] + (A == 1), o[2] + (A == 2))];
        if (o[A] >= 1) v += sqTc * R(o[A]) * Fp[h3idx(o[0] - (A == 0), o[1] - (A == 1), o[2] - (A == 2))];
        H[k] -= scale * v;
    }
#pragma unroll
    for (int k = 0; k < kNG3; ++k) {
        const int o[3] = {h3r(k), h3s(k), h3t(k)};
        R v = un * Gp[k];
        if (o[0] + o[1] + o[2] + 1 <= 2)
            v += sqTc * Gp[h3idx(o[0] + (A == 0), o[1] + (A == 1), o[2] + (A == 2))];
        if (o[A] >= 1) v += sqTc * R(o[A]) * Gp[h3idx(o[0] - (A == 0), o[1] - (A == 1), o[2] - (A == 2))];
        G[k] -= scale * v;
    }
}

template <typename R, int A>
__device__ __forceinline__ void cell_face_flux3(const Params3<R> &P, long long f, R scale, const typename FrameWords<R>::word *uc,
                                                R Tcr, R invTc, R rsqTc, R sqTc, R *H, R *G)
{
    const long long nf = P.nf(A);
    R Fc[kNF3], Gc[kNG3], dv[3];
#pragma unroll
    for (int q = 0; q < kNF3; ++q) Fc[q] = P.ff[A][q * nf + f];
#pragma unroll
    for (int q = 0; q < kNG3; ++q) Gc[q] = P.fg[A][q * nf + f];
#pragma unroll
    for (int a = 0; a < 3; ++a) dv[a] = R(fr_rel(P.ffr[A][a * nf + f], uc[a]));
    const R Tb = R(fr_lead(P.ffr[A][3 * nf + f]));
    add_face_flux3<R, A>(Fc, Gc, dv, Tb, Tcr, invTc, rsqTc, scale, sqTc, R(fr_lead(uc[A])), H, G);
}

template <typename R>
__device__ __forceinline__ double cell_rate3(const R *u, R T, const StepC<R> &KC)
{
    const R c = sqrt(T) * R(kCHi);
    R r = (fabs(u[0]) + c) * KC.inv_dx;
    r = max(r, (fabs(u[1]) + c) * KC.inv_dy);
    r = max(r, (fabs(u[2]) + c) * KC.inv_dz);
    return double(r);
}

// Step 3 of Sec. III.B.4 (Eqs. fluxEq, FinalUpdateDUGKS) through the six faces, fused with
// step 1 of the next step (the new co-moving frame from the conserved moments and the Grad
// projection into it) and the CFL reduction.
template <typename R, int THREADS = 128>
__global__ void __launch_bounds__(THREADS)
cell3_kernel(const Params3<R> P)
{
    const Clock &K = *P.clock;
    if (!(K.dt > 0.0)) return;
    const long long n = P.ncell();
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double rate = 0.0;
    using W = typename FrameWords<R>::word;
    const StepC<R> &KC = step_c<R>(K);
    if (c < n) {
        const long long i = c % P.nx, j = (c / P.nx) % P.ny, k = c / (P.nx * P.ny);
        W uc[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) uc[a] = P.sfr[a * n + c];
        const W Tc = P.sfr[3 * n + c];
        const R rho = P.sf[c];
        const R ca = KC.ca, cb = KC.cb, Cv = P.Cv_r;
        const R Tcr = R(fr_lead(Tc));
        const R invTc = R(1) / Tcr, rsqTc = sqrt(invTc), sqTc = Tcr * rsqTc;
        R H[kNF3], G[kNG3];
#pragma unroll
        for (int q = 0; q < kNF3; ++q) {
            const int pl = fplane3(q);
            H[q] = pl < 0 ? R(0) : ca * P.sf[pl * n + c];
        }
        H[0] += cb * rho;
#pragma unroll
        for (int q = 0; q < kNG3; ++q) G[q] = ca * P.sg[q * n + c];
        G[0] += cb * (Cv - R(1.5)) * rho * Tcr;
        const R sx = KC.dt_dx, sy = KC.dt_dy, sz = KC.dt_dz;
        cell_face_flux3<R, 0>(P, P.fidx(0, i, j, k), -sx, uc, Tcr, invTc, rsqTc, sqTc, H, G);
        cell_face_flux3<R, 0>(P, P.fidx(0, i + 1, j, k), sx, uc, Tcr, invTc, rsqTc, sqTc, H, G);
        cell_face_flux3<R, 1>(P, P.fidx(1, i, j, k), -sy, uc, Tcr, invTc, rsqTc, sqTc, H, G);
        cell_face_flux3<R, 1>(P, P.fidx(1, i, j + 1, k), sy, uc, Tcr, invTc, rsqTc, sqTc, H, G);
        cell_face_flux3<R, 2>(P, P.fidx(2, i, j, k), -sz, uc, Tcr, invTc, rsqTc, sqTc, H, G);
        cell_face_flux3<R, 2>(P, P.fidx(2, i, j, k + 1), sz, uc, Tcr, invTc, rsqTc, sqTc, H, G);
        // the new frame from the conserved moments (increments relative to the old frame)
        const R rn = H[0], irn = R(1) / rn;
        R du[3];
        du[0] = sqTc * H[h3idx(1, 0, 0)] * irn;
        du[1] = sqTc * H[h3idx(0, 1, 0)] * irn;
        du[2] = sqTc * H[h3idx(0, 0, 1)] * irn;
        const R k2 = du[0] * du[0] + du[1] * du[1] + du[2] * du[2];
        const R trH = H[h3idx(2, 0, 0)] + H[h3idx(0, 2, 0)] + H[h3idx(0, 0, 2)];
        const R dT = (R(0.5) * trH + G[0] * invTc - (Cv - R(1.5)) * rn - R(0.5) * rn * k2 * invTc) / (Cv * rn);
        bool ok = rn > R(0) && R(1) + dT > R(0) && isfinite(double(rn)) && isfinite(double(dT));
        const R s2 = R(1) / (R(1) + dT);
        const R sc = sqrt(s2), e = -dT * s2, rsqn = rsqTc * sc;
        Map1<R> X(sc, e, -du[0] * rsqn), Y(sc, e, -du[1] * rsqn), Z(sc, e, -du[2] * rsqn);
        R Ho[kNF3], Go[kNG3];
        shift_scale_3d<3, R>(H, X, Y, Z, Ho);
        shift_scale_3d<2, R>(G, X, Y, Z, Go);
        W un[3];
        R unr[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            un[a] = fr_add(uc[a], du[a]);
            unr[a] = R(fr_lead(un[a]));
        }
        const W Tn = fr_add(Tc, Tcr * dT);
        const R Tnr = R(fr_lead(Tn));
        ok = ok && Tnr > R(0) && isfinite(Tnr);
        if (!ok) {
            atomicOr(&P.diag->flags, FLAG_NONPHYSICAL);
            atomicAdd(&P.diag->nonphys, 1ull);
            atomicCAS((unsigned long long *)&P.diag->first_bad, (unsigned long long)-1ll, (unsigned long long)c);
        }
#pragma unroll
        for (int q = 0; q < kNF3; ++q) {
            const int pl = fplane3(q);
            if (pl >= 0) P.sf[pl * n + c] = Ho[q];
        }
#pragma unroll
        for (int q = 0; q < kNG3; ++q) P.sg[q * n + c] = Go[q];
#pragma unroll
        for (int a = 0; a < 3; ++a) P.sfr[a * n + c] = un[a];
        P.sfr[3 * n + c] = Tn;
        rate = ok ? cell_rate3<R>(unr, Tnr, KC) : 0.0;
    }
    reduce_rate_and_advance(P.clock, rate, true);
}

// ------------------------------------------------------- initial condition, read-back

// equilibria of Eqs. (feqPond), (geqPond) in each cell's frame from primitive fields
template <typename R>
__global__ void init_cells3_kernel(const Params3<R> P, const double *rho, const double *ux, const double *uy,
                                   const double *uz, const double *p)
{
    const long long n = P.ncell();
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double rate = 0.0;
    if (c < n) {
        const double r = rho[c], T = p[c] / r;
        const double u[3] = {ux[c], uy[c], uz[c]};
        P.sf[c] = R(r);
#pragma unroll
        for (int q = 1; q < kNFS3; ++q) P.sf[q * n + c] = R(0);
        P.sg[c] = R((P.Cv - 1.5) * r * T);
#pragma unroll
        for (int q = 1; q < kNG3; ++q) P.sg[q * n + c] = R(0);
#pragma unroll
        for (int a = 0; a < 3; ++a) fr_store(P.sfr[a * n + c], u[a]);
        fr_store(P.sfr[3 * n + c], T);
        const bool ok = r > 0.0 && T > 0.0 && isfinite(r) && isfinite(T);
        if (!ok) {
            atomicOr(&P.diag->flags, FLAG_NONPHYSICAL);
            atomicAdd(&P.diag->nonphys, 1ull);
            atomicCAS((unsigned long long *)&P.diag->first_bad, (unsigned long long)-1ll, (unsigned long long)c);
        }
        const double cm = sqrt(T) * kCHi;
        rate = ok ? fmax(fmax((fabs(u[0]) + cm) / P.dx, (fabs(u[1]) + cm) / P.dy), (fabs(u[2]) + cm) / P.dz) : 0.0;
    }
    reduce_rate_and_advance(P.clock, rate, false);
}

template <typename R>
__device__ __forceinline__ void cell_conserved3(const Params3<R> &P, long long i, long long j, long long k, double &r,
                                                double *m, double &E)
{
    int flip = 0;
    const long long idx = resolve3(P, i, j, k, &flip);
    const long long n = P.ncell();
    r = double(P.sf[idx]);
    const double T = fr_value(P.sfr[3 * n + idx]);
    double k2 = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double u = fr_value(P.sfr[a * n + idx]);
        if (flip & (1 << a)) u = -u;
        m[a] = r * u;
        k2 += u * u;
    }
    E = r * (P.Cv * T + 0.5 * k2);
}

// face predictor before the first step: the frame of the pooled moments of the two cells
template <typename R>
__global__ void init_faces3_kernel(const Params3<R> P)
{
    const long long n0 = P.nf(0), n1 = P.nf(1), n2 = P.nf(2);
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n0 + n1 + n2) return;
    const int dir = t < n0 ? 0 : (t < n0 + n1 ? 1 : 2);
    const long long f = t - (dir == 0 ? 0 : (dir == 1 ? n0 : n0 + n1));
    const long long ex = P.nx + (dir == 0), ey = P.ny + (dir == 1);
    const long long i = f % ex, j = (f / ex) % ey, k = f / (ex * ey);
    double ra, ma[3], Ea, rb, mb[3], Eb;
    cell_conserved3<R>(P, i - (dir == 0), j - (dir == 1), k - (dir == 2), ra, ma, Ea);
    cell_conserved3<R>(P, i, j, k, rb, mb, Eb);
    const double r = 0.5 * (ra + rb), E = 0.5 * (Ea + Eb);
    double k2 = 0.0;
    typename FrameWords<R>::word *Frm = P.ffr[dir];
    const long long nf = P.nf(dir);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double m = 0.5 * (ma[a] + mb[a]);
        fr_store(Frm[a * nf + f], m / r);
        k2 += m * m;
    }
    fr_store(Frm[3 * nf + f], (E - 0.5 * k2 / r) / (P.Cv * r));
}

template <typename R>
__global__ void conserved3_kernel(const Params3<R> P, double *rho, double *mx, double *my, double *mz, double *E)
{
    const long long n = P.ncell();
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    double r, m[3], e;
    cell_conserved3<R>(P, c % P.nx, (c / P.nx) % P.ny, c / (P.nx * P.ny), r, m, e);
    if (rho) rho[c] = r;
    if (mx) mx[c] = m[0];
    if (my) my[c] = m[1];
    if (mz) mz[c] = m[2];
    if (E) E[c] = e;
}

// stored state as full coefficient arrays [cells][20], [cells][10] and frames [cells][4]
template <typename R>
__global__ void export_state3_kernel(const Params3<R> P, double *cf, double *cg, double *fr)
{
    const long long n = P.ncell();
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
#pragma unroll
    for (int q = 0; q < kNF3; ++q) {
        const int pl = fplane3(q);
        cf[c * kNF3 + q] = pl < 0 ? 0.0 : double(P.sf[pl * n + c]);
    }
#pragma unroll
    for (int q = 0; q < kNG3; ++q) cg[c * kNG3 + q] = double(P.sg[q * n + c]);
#pragma unroll
    for (int a = 0; a <= 3; ++a) fr[c * 4 + a] = fr_value(P.sfr[a * n + c]);
}

}  // namespace pond
