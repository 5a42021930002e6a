// pond_kernels.cuh -- the CUDA kernels of one regularized PonD finite-volume step.
//
// Data layout in device memory (structure of arrays, x fastest):
//   cell state  : f coefficients in the cell's own frame without the (zero) first-order
//                 ones -- D1Q4: rho, a2, a3; D2Q16: rho, a20, a11, a02, a30, a21, a12, a03 --
//                 g coefficients b0..b2 (D1Q4) or b00, b10, b01, b20, b11, b02 (D2Q16), all in
//                 the population precision R; frame u (D values) and T in FP64.
//   face data   : per face the Hermite coefficients of the face populations phi(x_b, t_{n+1/2})
//                 (f: 4 or 10, g: 3 or 6, precision R) in the face frame, and that frame
//                 (u..., T) in FP64.  The frame doubles as the corrector predictor of the
//                 next step (Sec. III.B.3: lambda_0 = lambda(x_b, t_{n-1/2})).
// Faces: x-face (i, j) lies between cells (i-1, j) and (i, j), i = 0..nx; y-face (i, j)
// between (i, j-1) and (i, j), j = 0..ny.
//
// Per step (Sec. III.B.4): face_kernel (steps 2a-2b) then cell_kernel (step 3 fused with
// step 1 of the next step and the CFL time step of Sec. IV).
#pragma once

#include <cuda.h>   // CUtensorMap (the type only; maps are encoded through the runtime's driver entry point)

#include "pond_core.cuh"
#include "pond_mlp.cuh"

namespace pond {

// ------------------------------------------------------------------ frame words
//
// Frames (u, T) are stored in FP64 words when the populations are FP64.  With FP32
// populations they are float-float pairs, value = hi + lo with |lo| <= ulp(hi)/2 (Dekker's
// double-length arithmetic): about 48 significant bits, with every operation on the FP32
// pipes.  GB300 runs FP64 at 1/64 of the FP32 rate, so this keeps FP64 instructions out of
// the stencil loops.  Frame arithmetic only ever forms differences of nearby frames and adds
// FP32 increments formed relative to the old frame, which is what the pairs do exactly.

struct __align__(8) ffloat {
    float hi, lo;
};

// storage words of a frame component: word for cell and face frames, pred for a face
// predictor that only seeds the corrector
template <typename R>
struct FrameWords;
template <>
struct FrameWords<double> {
    using word = double;
    using pred = double;
};
template <>
struct FrameWords<float> {
    using word = ffloat;
    using pred = float;
};

__host__ __device__ __forceinline__ double fr_value(double x) { return x; }
__host__ __device__ __forceinline__ double fr_value(float x) { return double(x); }
__host__ __device__ __forceinline__ double fr_value(ffloat x) { return double(x.hi) + double(x.lo); }
__host__ __device__ __forceinline__ void fr_store(double &w, double v) { w = v; }
__host__ __device__ __forceinline__ void fr_store(float &w, double v) { w = float(v); }
__host__ __device__ __forceinline__ void fr_store(ffloat &w, double v)
{
    w.hi = float(v);
    w.lo = float(v - double(w.hi));
}
// -x
__host__ __device__ __forceinline__ double fr_neg(double x) { return -x; }
__host__ __device__ __forceinline__ ffloat fr_neg(ffloat x) { return ffloat{-x.hi, -x.lo}; }
// a working-precision value as a word
__device__ __forceinline__ double fr_word(double v) { return v; }
__device__ __forceinline__ ffloat fr_word(float v) { return ffloat{v, 0.f}; }
// leading value in the working precision
__device__ __forceinline__ double fr_lead(double x) { return x; }
__device__ __forceinline__ float fr_lead(ffloat x) { return x.hi; }
// x - ref in the working precision
__device__ __forceinline__ double fr_rel(double x, double ref) { return x - ref; }
__device__ __forceinline__ float fr_rel(ffloat x, ffloat ref) { return (x.hi - ref.hi) + (x.lo - ref.lo); }
__device__ __forceinline__ float fr_rel(float x, ffloat ref) { return (x - ref.hi) - ref.lo; }
// ref + d rounded to a face word
__device__ __forceinline__ double fr_face(double ref, double d) { return ref + d; }
__device__ __forceinline__ float fr_face(ffloat ref, float d) { return ref.hi + (ref.lo + d); }
// x + d: error-free sum of the leading words (Knuth's two-sum), then renormalised
__device__ __forceinline__ double fr_add(double x, double d) { return x + d; }
__device__ __forceinline__ ffloat fr_add(ffloat x, float d)
{
    const float s = __fadd_rn(x.hi, d);
    const float bb = __fsub_rn(s, x.hi);
    const float err = __fadd_rn(__fsub_rn(x.hi, __fsub_rn(s, bb)), __fsub_rn(d, bb)) + x.lo;
    ffloat o;
    o.hi = __fadd_rn(s, err);
    o.lo = __fsub_rn(err, __fsub_rn(o.hi, s));
    return o;
}


enum { BC_TRANSMISSIVE = 0, BC_PERIODIC = 1, BC_INFLOW = 2, BC_REFLECTIVE = 3 };
enum { FLAG_NONPHYSICAL = 1u, FLAG_NOT_CONVERGED = 2u, FLAG_TIMEOUT = 4u };

// constants of the step about to run, set with dt (Eqs. FinalUpdateDUGKS, Fbarplus,
// FluxTransf): update ca = (2tau-dt)/(2tau+dt), cb = 2dt/(2tau+dt); phi-bar-plus
// cp = (2tau-h)/(2tau+dt), ce = 3h/(2tau+dt); face populations wb = 2tau/(2tau+h),
// we = h/(2tau+h); departure offsets h/dx, h/dy (h/dz on D3Q64 grids); h = dt/2
template <typename T>
struct StepC {
    T ca, cb, cp, ce, wb, we, h_dx, h_dy, dt_dx, dt_dy, inv_dx, inv_dy;
    T h_dz, dt_dz, inv_dz;
};

struct Clock {
    double t, dt, t_end, cfl;
    double tau, dx, dy, dz;
    StepC<double> kd;               // formed in FP64
    StepC<float> kf;                // the same rounded to FP32
    long long steps;
    unsigned long long rate_bits;   // max CFL rate of the step being reduced (as double bits)
    unsigned int blocks_done;
    unsigned int pad;
};

template <typename R>
__host__ __device__ __forceinline__ const StepC<R> &step_c(const Clock &K)
{
    if constexpr (sizeof(R) == 8) return K.kd;
    else return K.kf;
}

__host__ __device__ inline void set_step_constants(Clock &c, double dt)
{
    const double tau = c.tau, h = 0.5 * dt;
    c.dt = dt;
    StepC<double> &k = c.kd;
    k.ca = (2.0 * tau - dt) / (2.0 * tau + dt);
    k.cb = 2.0 * dt / (2.0 * tau + dt);
    k.cp = (2.0 * tau - h) / (2.0 * tau + dt);
    k.ce = 3.0 * h / (2.0 * tau + dt);
    k.wb = 2.0 * tau / (2.0 * tau + h);
    k.we = h / (2.0 * tau + h);
    k.h_dx = h / c.dx;
    k.h_dy = h / c.dy;
    k.dt_dx = dt / c.dx;
    k.dt_dy = dt / c.dy;
    k.inv_dx = 1.0 / c.dx;
    k.inv_dy = 1.0 / c.dy;
    k.h_dz = h / c.dz;
    k.dt_dz = dt / c.dz;
    k.inv_dz = 1.0 / c.dz;
    c.kf = StepC<float>{float(k.ca),   float(k.cb),   float(k.cp),    float(k.ce),    float(k.wb),     float(k.we),
                        float(k.h_dx), float(k.h_dy), float(k.dt_dx), float(k.dt_dy), float(k.inv_dx), float(k.inv_dy),
                        float(k.h_dz), float(k.dt_dz), float(k.inv_dz)};
}

struct Diag {
    unsigned long long face_solves, face_iters, nonconv, fallbacks, nonphys;
    long long first_bad;
    unsigned int flags;
    unsigned int pad;
    unsigned long long tma_tiles;   // face-kernel tiles whose box was staged by tensor-map copies
};

// Tensor maps of the cell-state planes for the face kernel's TMA staging (D2Q16, FP32): the
// stored f planes [NFS][ny][nx], the g planes [NGC][ny][nx] and the frame words [D+1][ny][nx]
// as three-dimensional tensors, each copied as one box of kTmaBoxX x (TY + 3) x planes per
// tile.  key is the f-plane pointer they describe (the state planes alternate between two
// buffers under the fused step), so a launch uses them only while P.sf equals it.
constexpr int kTmaBoxX = 16;          // x extent of a copied box (cells i0 - 4 .. i0 + 11)
struct StageMaps {
    CUtensorMap sf, sg, sfr;
    const void *key;
};

template <int D, typename R>
struct Params {
    static constexpr int NFC = NCoef<D, 3>::value;   // f coefficients per face
    static constexpr int NGC = NCoef<D, 2>::value;   // g coefficients
    static constexpr int NFS = NFC - D;              // stored f planes (no first order)
    long long nx, ny;
    double dx, dy;
    int bc[4];
    long long lo[4], hi[4];
    double inflow[4][4];             // rho, ux, uy, p
    using W = typename FrameWords<R>::word;
    double gamma, Cv, tau;
    R Cv_r, Cvh_r, tol_r;             // Cv, Cv - D/2 and tol in the working precision
    int limiter;
    double tol;
    int max_iter, fixed_iters;
    R *sf;                            // [NFS][ncell]
    R *sg;                            // [NGC][ncell]
    W *sfr;                           // [D+1][ncell]
    R *xf, *xg;                       // [NFC][nxf], [NGC][nxf]
    W *xfr;                           // [D+1][nxf]
    R *yf, *yg;
    W *yfr;
    W *xlr, *ylr;                     // learned predictions per face [D+1][nf] (T not finite: none)
    // the fused step writes the new state and face frames here (the host then swaps them
    // with sf, sg, sfr, xfr, yfr)
    R *sf_n, *sg_n;
    W *sfr_n, *xfr_n, *yfr_n;
    int use_learned;                  // the face corrector tries the learned prediction first
    // activity of the learned predictor's tiles (16 x 4 faces of each axis): [2][tiles], the
    // step s + 1 stamped into row (s + 1) & 1 where a face of the tile needed more than one
    // corrector pass, or started from a prediction, in step s
    unsigned int *pred_active;
    int equilibrate;                  // the equilibration alternative of Sec. II.C (an ablation)
    Clock *clock;
    Diag *diag;
    // learned face-gauge predictor: parameters, and sampling of training pairs
    const float *mlp;
    float *pairs;
    unsigned long long *pair_count;
    long long pair_cap;
    int pair_every;
    float gauge_gate;                 // the prediction is used where its largest component exceeds this
    float gauge_trust;                // ... and does not exceed this (the corrector's basin of the
                                      // previous frame; larger moves may reach another fixed point)
    unsigned int *mlp_err;
    int sms;                          // SMs of the device (grid sizes of the grid-stride kernels)
    // host memory: tensor maps of the two state buffers for the TMA-staged face variant (null
    // where the grid does not allow them); read by the launcher, never by a kernel
    const StageMaps *stage_maps;
    __host__ __device__ long long ncell() const { return nx * ny; }
    __host__ __device__ long long nxf() const { return (nx + 1) * ny; }
    __host__ __device__ long long nyf() const { return nx * (ny + 1); }
};

// stored f plane of full coefficient k (or -1 when it is a first-order one, always zero)
template <int D>
__host__ __device__ constexpr int fplane(int k)
{
    return D == 1 ? (k == 0 ? 0 : k == 1 ? -1 : k - 1) : (k == 0 ? 0 : (k == 1 || k == 2) ? -1 : k - 2);
}

__device__ __forceinline__ long long clampll(long long v, long long lo, long long hi) { return v < lo ? lo : (v > hi ? hi : v); }
__device__ __forceinline__ long long wrapll(long long v, long long n) { long long r = v % n; return r < 0 ? r + n : r; }

// Ghost-cell rules (two layers; y sides first, then x sides).  Returns -1 and the linear
// cell index, or the side (0..3) whose inflow state the cell holds.  *flip receives the
// axes (bit 0 x, bit 1 y) across which the cell is a mirror image (reflective walls: ghost
// -k mirrors cell k-1, ghost n-1+k mirrors cell n-k); the holder of the cell reverses the
// normal components of its velocity and of its odd-order coefficients along those axes.
template <int D, typename R>
__device__ __forceinline__ int resolve(const Params<D, R> &P, long long i, long long j, long long *idx, int *flip)
{
    int fl = 0;
    if (D == 2 && (j < 0 || j >= P.ny)) {
        const int side = j < 0 ? 2 : 3;
        const long long ic = clampll(i, 0, P.nx - 1);
        if (P.bc[side] == BC_INFLOW && ic >= P.lo[side] && ic < P.hi[side]) { *flip = fl; return side; }
        if (P.bc[side] == BC_REFLECTIVE) {
            j = j < 0 ? -1 - j : 2 * P.ny - 1 - j;
            j = clampll(j, 0, P.ny - 1);  // grids thinner than the ghost layers
            fl |= 2;
        } else {
            j = P.bc[side] == BC_PERIODIC ? wrapll(j, P.ny) : clampll(j, 0, P.ny - 1);
        }
    }
    if (i < 0 || i >= P.nx) {
        const int side = i < 0 ? 0 : 1;
        if (P.bc[side] == BC_INFLOW && j >= P.lo[side] && j < P.hi[side]) { *flip = fl; return side; }
        if (P.bc[side] == BC_REFLECTIVE) {
            i = i < 0 ? -1 - i : 2 * P.nx - 1 - i;
            i = clampll(i, 0, P.nx - 1);
            fl |= 1;
        } else {
            i = P.bc[side] == BC_PERIODIC ? wrapll(i, P.nx) : clampll(i, 0, P.nx - 1);
        }
    }
    *idx = j * P.nx + i;
    *flip = fl;
    return -1;
}

// sign of coefficient (r, s) (orders along x and y) of a cell mirrored across the axes in flip
template <int D>
__device__ __forceinline__ bool mirror_odd(int k, int flip)
{
    int r = 0, s = 0;
    if (D == 1) {
        r = k;
    } else {
        int n = 0;
        while ((n + 1) * (n + 2) / 2 <= k) ++n;  // k = hidx(r, s) with r + s = n
        s = k - n * (n + 1) / 2;
        r = n - s;
    }
    return (((flip & 1) && (r & 1)) != 0) != (((flip & 2) && (s & 1)) != 0);
}

// Cell data as staged for the face corrector: phi-bar-plus coefficients (Eq. Fbarplus) in
// the cell frame, the frame, and the density.
// Records are padded to a multiple of 16 bytes and read with 16-byte loads (fetch): 5 loads
// instead of 19 for a D2Q16 FP32 record, and neighbouring threads' records (80 B apart)
// fall in distinct bank groups.
template <int D, typename R>
constexpr int staged_pad()
{
    constexpr int bytes = (NCoef<D, 3>::value + NCoef<D, 2>::value + D + 1) * int(sizeof(R));
    return ((16 - bytes % 16) % 16) / int(sizeof(R));
}
template <int D, typename R>
struct __align__(16) StagedCell {
    R A[NCoef<D, 3>::value];
    R B[NCoef<D, 2>::value];
    R du[D];    // frame velocity relative to the tile reference velocity
    R T;
    R pad[staged_pad<D, R>() > 0 ? staged_pad<D, R>() : 1];
};

// a staged record into registers with 16-byte shared-memory loads
template <int D, typename R>
__device__ __forceinline__ StagedCell<D, R> fetch(const StagedCell<D, R> *p)
{
    static_assert(sizeof(StagedCell<D, R>) % 16 == 0, "16-byte records");
    constexpr int N = int(sizeof(StagedCell<D, R>) / 16);
    union {
        StagedCell<D, R> c;
        float4 v[N];
    } u;
    const float4 *src = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int k = 0; k < N; ++k) u.v[k] = src[k];
    return u.c;
}

// Loads cell (i, j) (ghosts resolved) and forms phi-bar-plus = cp phi~ + ce phi^eq with
// phi^eq the co-moving equilibria (rho, 0, ...) and ((Cv - D/2) rho T, 0, ...).
template <int D, typename R>
__device__ __forceinline__ void cell_velocity(const Params<D, R> &P, long long i, long long j,
                                              typename FrameWords<R>::word *u)
{
    long long idx = 0;
    int flip = 0;
    const int side = resolve(P, i, j, &idx, &flip);
    if (side >= 0) {
        fr_store(u[0], P.inflow[side][1]);
        if constexpr (D == 2) fr_store(u[1], P.inflow[side][2]);
    } else {
#pragma unroll
        for (int a = 0; a < D; ++a) u[a] = P.sfr[a * P.ncell() + idx];
    }
#pragma unroll
    for (int a = 0; a < D; ++a)
        if (flip & (1 << a)) u[a] = fr_neg(u[a]);
}

// phi-bar-plus of a loaded cell record (stored coefficients in c.A, c.B, frame u, T): the
// frame velocity relative to the tile reference and Eq. (Fbarplus) with the co-moving
// equilibria (rho, 0, ...) and ((Cv - D/2) rho T, 0, ...)
template <int D, typename R>
__device__ __forceinline__ void finish_bar_plus(const Params<D, R> &P, R cp, R ce,
                                                const typename FrameWords<R>::word *utile,
                                                const typename FrameWords<R>::word *u, R T, StagedCell<D, R> &c)
{
    constexpr int NFC = NCoef<D, 3>::value, NGC = NCoef<D, 2>::value;
#pragma unroll
    for (int a = 0; a < D; ++a) c.du[a] = R(fr_rel(u[a], utile[a]));
    const R r = c.A[0];
    c.A[0] = cp * r + ce * r;
#pragma unroll
    for (int k = 1; k < NFC; ++k) c.A[k] = cp * c.A[k];
    c.B[0] = cp * c.B[0] + ce * (P.Cvh_r * r * T);
#pragma unroll
    for (int k = 1; k < NGC; ++k) c.B[k] = cp * c.B[k];
    c.T = T;
}

template <int D, typename R>
__device__ __forceinline__ void load_cell_bar_plus(const Params<D, R> &P, long long i, long long j, R cp, R ce,
                                                   const typename FrameWords<R>::word *utile, StagedCell<D, R> &c)
{
    constexpr int NFC = NCoef<D, 3>::value, NGC = NCoef<D, 2>::value;
    using W = typename FrameWords<R>::word;
    long long idx = 0;
    int flip = 0;
    const int side = resolve(P, i, j, &idx, &flip);
    W u[D];
    R T;
    if (side >= 0) {
        const double rho = P.inflow[side][0], Td = P.inflow[side][3] / rho;
        fr_store(u[0], P.inflow[side][1]);
        if constexpr (D == 2) fr_store(u[1], P.inflow[side][2]);
#pragma unroll
        for (int k = 0; k < NFC; ++k) c.A[k] = R(0);
#pragma unroll
        for (int k = 0; k < NGC; ++k) c.B[k] = R(0);
        c.A[0] = R(rho);
        c.B[0] = R((P.Cv - 0.5 * D) * rho * Td);
        T = R(Td);
    } else {
        const long long n = P.ncell();
#pragma unroll
        for (int k = 0; k < NFC; ++k) {
            const int pl = fplane<D>(k);
            c.A[k] = pl < 0 ? R(0) : P.sf[pl * n + idx];
        }
#pragma unroll
        for (int k = 0; k < NGC; ++k) c.B[k] = P.sg[k * n + idx];
#pragma unroll
        for (int a = 0; a < D; ++a) u[a] = P.sfr[a * n + idx];
        T = R(fr_lead(P.sfr[D * n + idx]));
    }
    if (flip) {
        // mirror image: odd orders along a flipped axis and that velocity component reverse
#pragma unroll
        for (int k = 0; k < NFC; ++k)
            if (mirror_odd<D>(k, flip)) c.A[k] = -c.A[k];
#pragma unroll
        for (int k = 0; k < NGC; ++k)
            if (mirror_odd<D>(k, flip)) c.B[k] = -c.B[k];
#pragma unroll
        for (int a = 0; a < D; ++a)
            if (flip & (1 << a)) u[a] = fr_neg(u[a]);
    }
    finish_bar_plus<D, R>(P, cp, ce, utile, u, T, c);
}

// ------------------------------------------------------------------ face corrector


// transposes coefficient arrays so that index r always refers to the face normal
template <int D, int N, typename R>
__device__ __forceinline__ void orient(const R *in, R *out, bool swap)
{
    if (D == 1 || !swap) {
#pragma unroll
        for (int k = 0; k < NCoef<D, N>::value; ++k) out[k] = in[k];
    } else {
#pragma unroll
        for (int r = 0; r <= N; ++r)
#pragma unroll
            for (int s = 0; s + r <= N; ++s) out[hidx(r, s)] = in[hidx(s, r)];
    }
}

// frame map of a staged cell into the corrector frame: s = sqrt(Tc/Tl), e = s^2 - 1,
// d = (uc - ul)/sqrt(Tl) with velocities relative to the face reference
template <int D, typename R>
__device__ __forceinline__ void cell_maps(R Tc, const R *dc, R Tl, R invTl, R rsqTl, const R *dl,
                                          Map1<R> &X, Map1<R> &Y)
{
    const R s = w_sqrt<R>(Tc * invTl);
    const R e = (Tc - Tl) * invTl;
    X = Map1<R>(s, e, (dc[0] - dl[0]) * rsqTl);
    if (D == 2) Y = Map1<R>(s, e, (dc[1] - dl[1]) * rsqTl);
    else Y = X;
}

// The stencil of one face in the staged tile: slot s at offsets (normal, tangential) from
// cell R -- 0 (-2, 0), 1 (-1, 0), 2 (0, 0), 3 (1, 0), 4 (-1, -1), 5 (-1, 1), 6 (0, -1),
// 7 (0, 1) -- with the strides (in cells) of the face's normal and tangential axes.  A base
// pointer and two strides instead of an array of eight pointers keeps registers free.
template <int D, typename R>
struct Stencil {
    const StagedCell<D, R> *base;
    int sn, st;
    __device__ __forceinline__ const StagedCell<D, R> *operator[](int s) const
    {
        const int on = s < 4 ? s - 2 : (s < 6 ? -1 : 0);
        const int ot = s < 4 ? 0 : ((s & 1) ? 1 : -1);
        return base + on * sn + ot * st;
    }
};

// frame velocity of a staged cell in face axes (normal, tangential) minus the face reference
template <int D, typename R>
__device__ __forceinline__ void rel_velocity(const StagedCell<D, R> *c, const R *dref, bool swap, R *out)
{
    if constexpr (D == 1) {
        out[0] = c->du[0] - dref[0];
    } else {
        out[0] = c->du[swap ? 1 : 0] - dref[0];
        out[1] = c->du[swap ? 0 : 1] - dref[1];
    }
}

// ---- FP32x2 helpers (packed FP32 arithmetic of sm_100 and later: one instruction, two lanes)
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }

// The limited slope of each lane divided by sc = limit_scale(kind): van Leer's 2ab/(a+b) as
// ab/(a+b) (the factor 2 goes into the departure offsets, an exact scaling), minmod as it is
__device__ __forceinline__ float limit_scale(int kind) { return kind == 1 ? 1.f : 2.f; }
__device__ __forceinline__ float2 limit2_scaled(int kind, float2 a, float2 b)
{
    const float2 ab = __fmul2_rn(a, b);
    if (kind == 1) return make_float2(minmod<float>(a.x, b.x), minmod<float>(a.y, b.y));
    const float2 den = __fadd2_rn(a, b);
    return make_float2(ab.x > 0.f ? __fdividef(ab.x, den.x) : 0.f, ab.y > 0.f ? __fdividef(ab.y, den.y) : 0.f);
}

// limited slope of each lane (van Leer or minmod), the products and sums packed
__device__ __forceinline__ float2 limit2(int kind, float2 a, float2 b)
{
    const float2 ab = __fmul2_rn(a, b);
    if (kind == 1) return make_float2(minmod<float>(a.x, b.x), minmod<float>(a.y, b.y));
    const float2 den = __fadd2_rn(a, b);
    const float2 num = __fmul2_rn(bc2(2.f), ab);
    return make_float2(ab.x > 0.f ? __fdividef(num.x, den.x) : 0.f, ab.y > 0.f ? __fdividef(num.y, den.y) : 0.f);
}

// The 16 populations of one normal node m at a 2D face (FP32): for each tangential node n,
// the upwind (u), outer (l), downstream (h) and tangential (-, +) cells' values from their
// column-collapsed coefficients (C: f, order <= 3; D: g, order <= 2), the limited MUSCL
// reconstruction at the departure point, and the moments S (f) and SG (g) along the
// tangent.  Lane x carries f and lane y carries g wherever both have the order.
// EQ: g also carries its third column (the fast components), evaluated in lane y.
template <bool EQ = false>
__device__ __forceinline__ void pair_populations(const float *Cu, const float *Cl, const float *Ch, const float *Cm,
                                                 const float *Cp, const float *Du, const float *Dl, const float *Dh,
                                                 const float *Dm, const float *Dp, float sqTl, float ut_abs, float h_dt,
                                                 float offn, int limiter, float *S, float *SG)
{
    const float2 minus1 = bc2(-1.f);
    float2 SS[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    float S3 = 0.f;
    // the limited slopes come divided by sc, the offsets multiplied by it
    const float sc = limit_scale(limiter), offn_s = sc * offn, h_dt_s = sc * h_dt;
#pragma unroll
    for (int n = 0; n < 4; ++n) {
        const float vt = sqTl * float(node_c(n)) + ut_abs;
        const float offt_s = -vt * h_dt_s;
        // order 0: He_0 = 1
        float2 u2 = make_float2(Cu[0], Du[0]), l2 = make_float2(Cl[0], Dl[0]), h2 = make_float2(Ch[0], Dh[0]),
               m2 = make_float2(Cm[0], Dm[0]), p2 = make_float2(Cp[0], Dp[0]);
#pragma unroll
        for (int b2 = 1; b2 <= 2; ++b2) {
            const float2 hn = bc2(float(hen(b2, n)));
            u2 = __ffma2_rn(make_float2(Cu[b2], Du[b2]), hn, u2);
            l2 = __ffma2_rn(make_float2(Cl[b2], Dl[b2]), hn, l2);
            h2 = __ffma2_rn(make_float2(Ch[b2], Dh[b2]), hn, h2);
            m2 = __ffma2_rn(make_float2(Cm[b2], Dm[b2]), hn, m2);
            p2 = __ffma2_rn(make_float2(Cp[b2], Dp[b2]), hn, p2);
        }
        const float h3 = float(hen(3, n));
        if constexpr (EQ) {
            const float2 h3b = bc2(h3);
            u2 = __ffma2_rn(make_float2(Cu[3], Du[3]), h3b, u2);
            l2 = __ffma2_rn(make_float2(Cl[3], Dl[3]), h3b, l2);
            h2 = __ffma2_rn(make_float2(Ch[3], Dh[3]), h3b, h2);
            m2 = __ffma2_rn(make_float2(Cm[3], Dm[3]), h3b, m2);
            p2 = __ffma2_rn(make_float2(Cp[3], Dp[3]), h3b, p2);
        } else {
            u2.x += Cu[3] * h3; l2.x += Cl[3] * h3; h2.x += Ch[3] * h3; m2.x += Cm[3] * h3; p2.x += Cp[3] * h3;
        }
        const float2 ln = limit2_scaled(limiter, __ffma2_rn(l2, minus1, u2), __ffma2_rn(u2, minus1, h2));
        const float2 lt = limit2_scaled(limiter, __ffma2_rn(m2, minus1, u2), __ffma2_rn(u2, minus1, p2));
        const float2 b = __ffma2_rn(bc2(offt_s), lt, __ffma2_rn(bc2(offn_s), ln, u2));
#pragma unroll
        for (int b2 = 0; b2 <= 2; ++b2) SS[b2] = __ffma2_rn(bc2(float(node_w(n) * he(b2, n))), b, SS[b2]);
        S3 += float(node_w(n) * he(3, n)) * b.x;
    }
#pragma unroll
    for (int b2 = 0; b2 <= 2; ++b2) {
        S[b2] = SS[b2].x;
        SG[b2] = SS[b2].y;
    }
    S[3] = S3;
}

// ---- the equilibration alternative of Sec. II.C (an ablation of Grad's projection)
// A population set moved into another frame keeps its slow moments (the Grad orders) and
// takes for its fast tensor-Hermite components A_rs (r, s <= 3, r + s above the Grad
// order) the values of the equilibrium with its own zeroth and first moments there:
// A_rs = A_00 d_x^r d_y^s with d = A_1 / A_00 (the first-order coefficients in the new frame;
// the Hermite moments of a Maxwellian of the frame's temperature shifted by d).  These
// helpers give the fast components the corrector and the flux need from the slow ones.
template <typename R>
struct FastEq {
    R a0, dx, dy;   // A_00 and d in the frame of the coefficients
    __device__ __forceinline__ R at(int r, int s) const
    {
        R v = a0;
#pragma unroll
        for (int k = 0; k < 3; ++k) if (k < r) v *= dx;
#pragma unroll
        for (int k = 0; k < 3; ++k) if (k < s) v *= dy;
        return v;
    }
};
template <int D, int N, typename R>
__device__ __forceinline__ FastEq<R> fast_eq(const R *A)
{
    FastEq<R> q;
    q.a0 = A[0];
    const R ia0 = w_rcp<R>(A[0]);
    if constexpr (D == 1) {
        q.dx = A[1] * ia0;
        q.dy = R(0);
    } else {
        q.dx = A[hidx(1, 0)] * ia0;
        q.dy = A[hidx(0, 1)] * ia0;
    }
    return q;
}

// Per-thread scratch in shared memory (FP32, 2D): the two centre cells' coefficients in the
// corrector frame (f: 10, g: 6 each; slots 0-7), the pass's moment sums (level 2: slots
// 8-11), the frames of the last valid pass (two slots after those) and, at level 2, the
// constants of the face output (one more slot),
// 16-byte slots, thread-minor so that a warp's accesses are contiguous.  They are touched
// once per normal node, so keeping them out of the registers across the node loop lowers
// the kernel's register demand.  The accesses are
// volatile so that the compiler neither hoists the loads out of the node loop nor moves
// them ahead of the stores.
struct FaceScratch {
    float4 *p;      // this thread's slot 0
    int stride;     // slots apart, in float4 (the block's thread count)
    __device__ __forceinline__ void put(int slot, float a, float b, float c, float d) const
    {
        const unsigned addr = (unsigned)__cvta_generic_to_shared(p + slot * stride);
        asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
                     : "memory");
    }
    __device__ __forceinline__ float4 get(int slot) const
    {
        const unsigned addr = (unsigned)__cvta_generic_to_shared(p + slot * stride);
        float4 v;
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                     : "r"(addr) : "memory");
        return v;
    }
    // f (10) and g (6) coefficients of one cell in slots base .. base + 3
    __device__ __forceinline__ void store(int base, const float *F, const float *G) const
    {
        put(base + 0, F[0], F[1], F[2], F[3]);
        put(base + 1, F[4], F[5], F[6], F[7]);
        put(base + 2, F[8], F[9], G[0], G[1]);
        put(base + 3, G[2], G[3], G[4], G[5]);
    }
    __device__ __forceinline__ void load(int base, float *F, float *G) const
    {
        const float4 a = get(base + 0), b = get(base + 1), c = get(base + 2), d = get(base + 3);
        F[0] = a.x; F[1] = a.y; F[2] = a.z; F[3] = a.w;
        F[4] = b.x; F[5] = b.y; F[6] = b.z; F[7] = b.w;
        F[8] = c.x; F[9] = c.y; G[0] = c.z; G[1] = c.w;
        G[2] = d.x; G[3] = d.y; G[4] = d.z; G[5] = d.w;
    }
};
__host__ __device__ constexpr int face_scratch_slots(int level) { return level > 1 ? 15 : 10; }
// slots of the last valid pass's frames (kept across the passes, read after the loop)
__host__ __device__ constexpr int face_keep_slot(int level) { return level > 1 ? 12 : 8; }

// One corrector pass at a face (Sec. III.B.3) in frame (dl, Tl) (velocity relative to the
// face reference uref): every stencil cell's phi-bar-plus is re-expressed in that frame,
// limited slopes are formed per population, each population is reconstructed by MUSCL
// at its departure point x_b - v_i dt/2 in the upwind cell, and the Hermite moments of
// the reconstructed f-bar and g-bar are returned (Phi: f, order 3; Psi: g, order 2).
// Stencil slots: 0 LL, 1 L, 2 R, 3 RR, 4 L-t, 5 L+t, 6 R-t, 7 R+t (t: tangential).
// EQ: the stencil cells are moved into the frame by the equilibration alternative
// (FastEq), so their populations also carry the fast components.
// SCR (FP32, 2D): 1, the centre cells' coefficients wait in the thread's shared scratch
// between the nodes; 2, the moment sums Phi, Psi also accumulate there (same arithmetic,
// same order).
template <int D, typename R, bool EQ = false, int SCR = 0, bool OUTER_ONCE = true>
__device__ __forceinline__ void corrector_pass(const Stencil<D, R> &cells, const R *dref,
                                               const R *dl, R Tl, R un_abs, R ut_abs, R h_dn, R h_dt,
                                               int limiter, R *Phi, R *Psi, FaceScratch scr = FaceScratch{nullptr, 0})
{
    static_assert(!SCR || (D == 2 && sizeof(R) == 4 && !EQ), "the scratch variants are FP32 2D Grad passes");
    constexpr int NFC = NCoef<D, 3>::value, NGC = NCoef<D, 2>::value;
    const R invTl = w_rcp<R>(Tl);
    const R rsqTl = w_sqrt<R>(invTl);
    const R sqTl = Tl * rsqTl;
    // the two cells next to the face, in the corrector frame
    R FL[NFC], FR[NFC], GL[NGC], GR[NGC];
    {
        Map1<R> X(R(1), R(0), R(0)), Y(R(1), R(0), R(0));
        R tmp[NFC], tmpg[NGC];
        R dcs[D];
        const StagedCell<D, R> cl = fetch<D, R>(cells[1]);
        rel_velocity<D, R>(&cl, dref, false, dcs);
        cell_maps<D, R>(cl.T, dcs, Tl, invTl, rsqTl, dl, X, Y);
        orient<D, 3, R>(cl.A, tmp, false);
        orient<D, 2, R>(cl.B, tmpg, false);
        shift_scale<D, 3, R, true>(tmp, X, Y, FL);   // staged f: zero first order
        shift_scale<D, 2, R>(tmpg, X, Y, GL);
        const StagedCell<D, R> cr = fetch<D, R>(cells[2]);
        rel_velocity<D, R>(&cr, dref, false, dcs);
        cell_maps<D, R>(cr.T, dcs, Tl, invTl, rsqTl, dl, X, Y);
        orient<D, 3, R>(cr.A, tmp, false);
        orient<D, 2, R>(cr.B, tmpg, false);
        shift_scale<D, 3, R, true>(tmp, X, Y, FR);
        shift_scale<D, 2, R>(tmpg, X, Y, GR);
    }
    if constexpr (SCR > 0) {
        scr.store(0, reinterpret_cast<const float *>(FL), reinterpret_cast<const float *>(GL));
        scr.store(4, reinterpret_cast<const float *>(FR), reinterpret_cast<const float *>(GR));
    }
#pragma unroll
    for (int k = 0; k < NFC; ++k) Phi[k] = R(0);
#pragma unroll
    for (int k = 0; k < NGC; ++k) Psi[k] = R(0);
    if constexpr (SCR > 1) scr.store(8, reinterpret_cast<const float *>(Phi), reinterpret_cast<const float *>(Psi));
    // 1D, OUTER_ONCE: the outer neighbours LL and RR in the frame, once per pass (each node
    // takes the one on its upwind side); else each node transforms its own (fewer live
    // registers, for kernels that run at a register cap)
    R FLL[D == 1 ? NFC : 1], GLL[D == 1 ? NGC : 1], FRR[D == 1 ? NFC : 1], GRR[D == 1 ? NGC : 1];
    if constexpr (D == 1 && OUTER_ONCE) {
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const StagedCell<D, R> sc = fetch<D, R>(cells[side ? 3 : 0]);
            R dcs[1];
            rel_velocity<D, R>(&sc, dref, false, dcs);
            Map1<R> X(R(1), R(0), R(0)), Y(R(1), R(0), R(0));
            cell_maps<D, R>(sc.T, dcs, Tl, invTl, rsqTl, dl, X, Y);
            shift_scale<D, 3, R, true>(sc.A, X, Y, side ? FRR : FLL);
            shift_scale<D, 2, R>(sc.B, X, Y, side ? GRR : GLL);
        }
    }

    const NodeTab<R> &tab = node_tab<R>();
    // normal node m: its populations, limited slopes and MUSCL values, summed into the
    // moments (unrolled in 1D, where the node's work is small; rolled in 2D, which keeps the
    // kernel within its register budget)
    auto node = [&](const int m) {
        const R vn = sqTl * tab.c[m] + un_abs;
        const bool left = vn > R(0);
        // departure point along the normal, in cells, from the upwind cell centre
        const R offn = (left ? R(0.5) : R(-0.5)) - vn * h_dn;
        if constexpr (D == 1) {
            // outer normal neighbour of the upwind cell, in the frame (chosen by selects so
            // that no array is indexed at run time)
            R FS[NFC], GS[NGC];
            R gL3 = R(0), gR3 = R(0), gS3 = R(0);   // fast g components at node m (EQ)
            if constexpr (OUTER_ONCE) {
#pragma unroll
                for (int k = 0; k < NFC; ++k) FS[k] = left ? FLL[k] : FRR[k];
#pragma unroll
                for (int k = 0; k < NGC; ++k) GS[k] = left ? GLL[k] : GRR[k];
            } else {
                const StagedCell<D, R> sc = fetch<D, R>(left ? cells[0] : cells[3]);
                R dcs[1];
                rel_velocity<D, R>(&sc, dref, false, dcs);
                Map1<R> X(R(1), R(0), R(0)), Y(R(1), R(0), R(0));
                cell_maps<D, R>(sc.T, dcs, Tl, invTl, rsqTl, dl, X, Y);
                shift_scale<D, 3, R, true>(sc.A, X, Y, FS);
                shift_scale<D, 2, R>(sc.B, X, Y, GS);
            }
            if constexpr (EQ) {
                // D1Q4 carries one fast component: g's third order
                const R h3 = tab.hen[m][3];
                gL3 = fast_eq<1, 2, R>(GL).at(3, 0) * h3;
                gR3 = fast_eq<1, 2, R>(GR).at(3, 0) * h3;
                gS3 = fast_eq<1, 2, R>(GS).at(3, 0) * h3;
            }
            if constexpr (sizeof(R) == 4 && !EQ) {
                // FP32: f (lane x) and g (lane y) side by side as FP32x2 pairs for the orders
                // they share; the same operations in the same order as the scalar form below
                // (van Leer's factor 2 scales the departure offset, an exact scaling)
                // (the 1D node loop is unrolled: m, and so these factors, are constants)
                const float h1 = float(hen(1, m)), h2 = float(hen(2, m)), h3 = float(hen(3, m));
                float2 pL = make_float2(FL[0], GL[0]), pR = make_float2(FR[0], GR[0]), pS = make_float2(FS[0], GS[0]);
                pL = __ffma2_rn(make_float2(FL[1], GL[1]), bc2(h1), pL);
                pR = __ffma2_rn(make_float2(FR[1], GR[1]), bc2(h1), pR);
                pS = __ffma2_rn(make_float2(FS[1], GS[1]), bc2(h1), pS);
                pL = __ffma2_rn(make_float2(FL[2], GL[2]), bc2(h2), pL);
                pR = __ffma2_rn(make_float2(FR[2], GR[2]), bc2(h2), pR);
                pS = __ffma2_rn(make_float2(FS[2], GS[2]), bc2(h2), pS);
                pL.x += FL[3] * h3; pR.x += FR[3] * h3; pS.x += FS[3] * h3;
                const float2 pu = left ? pL : pR, pl = left ? pS : pL, ph = left ? pR : pS;
                const float2 minus1 = bc2(-1.f);
                const float2 sl = limit2_scaled(limiter, __ffma2_rn(pl, minus1, pu), __ffma2_rn(pu, minus1, ph));
                const float2 pb = __ffma2_rn(bc2(limit_scale(limiter) * float(offn)), sl, pu);
#pragma unroll
                for (int a = 0; a <= 2; ++a) {
                    const float2 w = bc2(float(node_w(m) * he(a, m)));
                    const float2 acc = __ffma2_rn(w, pb, make_float2(Phi[a], Psi[a]));
                    Phi[a] = acc.x;
                    Psi[a] = acc.y;
                }
                Phi[3] += float(node_w(m) * he(3, m)) * pb.x;
                return;
            }
            // populations at node m (unweighted: the limiter is homogeneous of degree one,
            // so the weight w_m factors out) of L, R and the outer neighbour
            R fL = R(0), fR = R(0), fS = R(0), gL = gL3, gR = gR3, gS = gS3;
#pragma unroll
            for (int a = 0; a <= 3; ++a) {
                const R hn = tab.hen[m][a];
                fL += FL[a] * hn; fR += FR[a] * hn; fS += FS[a] * hn;
                if (a <= 2) { gL += GL[a] * hn; gR += GR[a] * hn; gS += GS[a] * hn; }
            }
            const R fu = left ? fL : fR, fl = left ? fS : fL, fh = left ? fR : fS;
            const R gu = left ? gL : gR, gl = left ? gS : gL, gh = left ? gR : gS;
            const R fb = fu + offn * limit<R>(limiter, fu - fl, fh - fu);
            const R gb = gu + offn * limit<R>(limiter, gu - gl, gh - gu);
#pragma unroll
            for (int a = 0; a <= 3; ++a) Phi[a] += tab.whe[m][a] * fb;
#pragma unroll
            for (int a = 0; a <= 2; ++a) Psi[a] += tab.whe[m][a] * gb;
        } else {
            // column collapse C_b = sum_a A_ab He_a(c_m)/a! of a coefficient set
            // (He_0 = 1: the order-0 term is the coefficient itself)
            auto collapse_f = [&](const R *A, R *C) {
#pragma unroll
                for (int b2 = 0; b2 <= 3; ++b2) {
                    R acc = A[hidx(0, b2)];
#pragma unroll
                    for (int a2 = 1; a2 + b2 <= 3; ++a2) acc += A[hidx(a2, b2)] * tab.hen[m][a2];
                    C[b2] = acc;
                }
            };
            auto collapse_g = [&](const R *A, R *C) {
#pragma unroll
                for (int b2 = 0; b2 <= 2; ++b2) {
                    R acc = A[hidx(0, b2)];
#pragma unroll
                    for (int a2 = 1; a2 + b2 <= 2; ++a2) acc += A[hidx(a2, b2)] * tab.hen[m][a2];
                    C[b2] = acc;
                }
            };
            // EQ: the fast components' part of the column collapse, f (r + s > 3) and g (> 2)
            auto collapse_fast = [&](const R *A, int order, R *C) {
                const FastEq<R> q = fast_eq<2, 3, R>(A);
#pragma unroll
                for (int b2 = 0; b2 <= 3; ++b2) {
                    R acc = R(0);
#pragma unroll
                    for (int a2 = 0; a2 <= 3; ++a2)
                        if (a2 + b2 > order) acc += q.at(a2, b2) * tab.hen[m][a2];
                    if (b2 <= order) C[b2] += acc;
                    else C[b2] = acc;
                }
            };
            constexpr int NGB = EQ ? 4 : 3;   // columns of the g collapse
            R CL[4], CR[4], DL[NGB], DR[NGB];
            if constexpr (SCR == 0) {
                collapse_f(FL, CL); collapse_f(FR, CR); collapse_g(GL, DL); collapse_g(GR, DR);
                if constexpr (EQ) {
                    collapse_fast(FL, 3, CL); collapse_fast(FR, 3, CR);
                    collapse_fast(GL, 2, DL); collapse_fast(GR, 2, DR);
                }
            }
            // outer normal neighbour (q = 0) and tangential neighbours (q = 1, 2) of the
            // upwind cell: transformed into the frame and collapsed one at a time
            R CS[3][4], DS[3][NGB];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                // slot (left, right upwind): q = 0 (0, 3), q = 1 (4, 6), q = 2 (5, 7); chosen by
                // selects so that no array is indexed at run time
                constexpr int sa[3] = {0, 4, 5}, sb[3] = {3, 6, 7};
                const StagedCell<D, R> sc = fetch<D, R>(left ? cells[sa[q]] : cells[sb[q]]);
                R dcs[D];
                rel_velocity<D, R>(&sc, dref, false, dcs);
                Map1<R> X(R(1), R(0), R(0)), Y(R(1), R(0), R(0));
                R tmp[NFC], tmpg[NGC], tr[NFC], trg[NGC];
                cell_maps<D, R>(sc.T, dcs, Tl, invTl, rsqTl, dl, X, Y);
                orient<D, 3, R>(sc.A, tmp, false);
                orient<D, 2, R>(sc.B, tmpg, false);
                shift_scale<D, 3, R, true>(tmp, X, Y, tr);
                shift_scale<D, 2, R>(tmpg, X, Y, trg);
                collapse_f(tr, CS[q]);
                collapse_g(trg, DS[q]);
                if constexpr (EQ) {
                    collapse_fast(tr, 3, CS[q]);
                    collapse_fast(trg, 2, DS[q]);
                }
            }
            if constexpr (SCR > 0) {
                // the centre cells from the scratch, after the neighbours (fewer live values)
                float Fs[10], Gs[6];
                scr.load(0, Fs, Gs);
                collapse_f(Fs, CL); collapse_g(Gs, DL);
                scr.load(4, Fs, Gs);
                collapse_f(Fs, CR); collapse_g(Gs, DR);
            }
            R Cu[4], Cl[4], Ch[4], Du[NGB], Dl[NGB], Dh[NGB];
#pragma unroll
            for (int b2 = 0; b2 <= 3; ++b2) {
                Cu[b2] = left ? CL[b2] : CR[b2];
                Cl[b2] = left ? CS[0][b2] : CL[b2];
                Ch[b2] = left ? CR[b2] : CS[0][b2];
            }
#pragma unroll
            for (int b2 = 0; b2 < NGB; ++b2) {
                Du[b2] = left ? DL[b2] : DR[b2];
                Dl[b2] = left ? DS[0][b2] : DL[b2];
                Dh[b2] = left ? DR[b2] : DS[0][b2];
            }
            R S[4] = {R(0), R(0), R(0), R(0)}, SG[3] = {R(0), R(0), R(0)};
            if constexpr (sizeof(R) == 4) {
                // FP32: the f and g populations run side by side as FP32x2 pairs (lane x: f,
                // lane y: g), so the shared orders 0..2 take one packed FMA for both
                pair_populations<EQ>(Cu, Cl, Ch, CS[1], CS[2], Du, Dl, Dh, DS[1], DS[2], sqTl, ut_abs, h_dt, offn,
                                     limiter, S, SG);
            } else {
#pragma unroll
            for (int n = 0; n < 4; ++n) {
                const R vt = sqTl * R(node_c(n)) + ut_abs;
                const R offt = -vt * h_dt;
                R fu = R(0), fl = R(0), fh = R(0), fm = R(0), fp = R(0);
#pragma unroll
                for (int b2 = 0; b2 <= 3; ++b2) {
                    const R hn = R(hen(b2, n));
                    fu += Cu[b2] * hn; fl += Cl[b2] * hn; fh += Ch[b2] * hn; fm += CS[1][b2] * hn; fp += CS[2][b2] * hn;
                }
                R gu = R(0), gl = R(0), gh = R(0), gm = R(0), gp = R(0);
#pragma unroll
                for (int b2 = 0; b2 < NGB; ++b2) {
                    const R hn = R(hen(b2, n));
                    gu += Du[b2] * hn; gl += Dl[b2] * hn; gh += Dh[b2] * hn; gm += DS[1][b2] * hn; gp += DS[2][b2] * hn;
                }
                const R fb = fu + offn * limit<R>(limiter, fu - fl, fh - fu) + offt * limit<R>(limiter, fu - fm, fp - fu);
                const R gb = gu + offn * limit<R>(limiter, gu - gl, gh - gu) + offt * limit<R>(limiter, gu - gm, gp - gu);
#pragma unroll
                for (int b2 = 0; b2 <= 3; ++b2) S[b2] += R(node_w(n) * he(b2, n)) * fb;
#pragma unroll
                for (int b2 = 0; b2 <= 2; ++b2) SG[b2] += R(node_w(n) * he(b2, n)) * gb;
            }
            }
#pragma unroll
            for (int a2 = 0; a2 <= 3; ++a2)
#pragma unroll
                for (int b2 = 0; a2 + b2 <= 3; ++b2) Phi[hidx(a2, b2)] += tab.whe[m][a2] * S[b2];
#pragma unroll
            for (int a2 = 0; a2 <= 2; ++a2)
#pragma unroll
                for (int b2 = 0; a2 + b2 <= 2; ++b2) Psi[hidx(a2, b2)] += tab.whe[m][a2] * SG[b2];
        }
    };
    // SCR 2: the node adds its moments to the sums waiting in the scratch
    auto node_scr = [&](const int m) {
        if constexpr (SCR > 1) {
            scr.load(8, reinterpret_cast<float *>(Phi), reinterpret_cast<float *>(Psi));
            node(m);
            scr.store(8, reinterpret_cast<const float *>(Phi), reinterpret_cast<const float *>(Psi));
        }
    };
    if constexpr (D == 1) {
#pragma unroll
        for (int m = 0; m < 4; ++m) node(m);
    } else if constexpr (SCR > 1) {
#pragma unroll 1
        for (int m = 0; m < 4; ++m) node_scr(m);
    } else {
#pragma unroll 1
        for (int m = 0; m < 4; ++m) node(m);
    }
}

// Frame defined by the moments of a pass (Eqs. correctorfieldsrhoDUGKS-TDUGKS), relative
// to the pass frame: rho, du (D) and T.  Returns false if it defines no frame.
template <int D, typename R>
__device__ __forceinline__ bool pass_frame(const R *Phi, const R *Psi, R Tl, R Cv, R &rho, R *du, R &T)
{
    rho = Phi[0];
    const R sq = w_sqrt<R>(Tl);
    R k2 = R(0), tr;
    if constexpr (D == 1) {
        du[0] = w_div<R>(sq * Phi[1], rho);
        k2 = du[0] * du[0];
        tr = Phi[2] + Phi[0];
    } else {
        du[0] = w_div<R>(sq * Phi[hidx(1, 0)], rho);
        du[1] = w_div<R>(sq * Phi[hidx(0, 1)], rho);
        k2 = du[0] * du[0] + du[1] * du[1];
        tr = Phi[hidx(2, 0)] + Phi[hidx(0, 2)] + R(2) * Phi[0];
    }
    // internal energy in the pass frame: T/2 sum f |c|^2 + sum g - rho |du|^2 / 2
    T = w_div<R>(R(0.5) * Tl * tr + Psi[0] - R(0.5) * rho * k2, Cv * rho);
    bool ok = T > R(0) && isfinite(T) && isfinite(rho);
#pragma unroll
    for (int a = 0; a < D; ++a) ok = ok && isfinite(du[a]);
    return ok;
}

template <typename R>
struct FaceCfg {
    R h_dn, h_dt;      // h/dx along the normal and the tangent
    R Cv, tol, wb, we;
    int limiter, max_iter, fixed_iters;
};

// a[k], k = 0 or 1, of a small register array by a select: an index known only at run time
// would put the array in local memory
template <typename T, int N>
__device__ __forceinline__ T sel(const T (&a)[N], int k)
{
    if constexpr (N == 1) return a[0];
    else return k ? a[1] : a[0];
}

template <int D, typename R>
struct FaceOut {
    R F[NCoef<D, 3>::value];   // f, g coefficients of phi(x_b, t_{n+1/2}) in the face frame (x, y order)
    R G[NCoef<D, 2>::value];
    R du[D];                   // face frame velocity minus the predictor's (x, y order)
    R T;
    int iters, fallbacks;
    bool done, have;
};

// The face predictor-corrector of Sec. III.B.3 at one face.  cells: stencil slots 0 LL,
// 1 L, 2 R, 3 RR, 4 L-t, 5 L+t, 6 R-t, 7 R+t (staged phi-bar-plus in face axes -- coefficient
// orders and velocities with the normal first --, velocities relative to the tile
// reference); swap: the face normal is y (the outputs go back to x, y order); the predictor lambda_0 is given by its
// velocity minus the tile reference (dref) and its absolute velocity (uabs, used only for
// upwinding and departure points), both in face axes (normal, tangential), and Tpred.
// Passes run until the frame converges (or fixed_iters passes); a pass whose moments define
// no frame restarts the corrector once from the frame of the pooled moments of the
// stencil, else the corrector stops at the last pass that did.  The face populations are
// Eq. (FluxTransf) at the frame of the last valid pass's moments.
// KEEP (FP32): 1, the last valid pass's frames wait in two slots of the thread's scratch
// (after the corrector's own slots) instead of staying live across the next pass; 2, the
// constants of the face output wait in one more slot
template <int D, typename R, bool EQ = false, int SCR = 0, bool OUTER_ONCE = true, int KEEP = (SCR > 1 ? 2 : SCR)>
__device__ __forceinline__ void solve_face(const Stencil<D, R> &cells, bool swap, const R *dref, const R *uabs,
                                           R Tpred, const FaceCfg<R> &cfg, FaceOut<D, R> &o,
                                           FaceScratch scr = FaceScratch{nullptr, 0})
{
    static_assert(KEEP == 0 || sizeof(R) == 4, "the kept frames are FP32 scratch words");
    constexpr int KS = SCR > 0 ? face_keep_slot(SCR) : 0;   // first slot of the kept frames
    o.fallbacks = 0;
    constexpr int NCELL = D == 2 ? 8 : 4;
    constexpr int NFC = NCoef<D, 3>::value, NGC = NCoef<D, 2>::value;
    const int na = swap ? 1 : 0, ta = swap ? 0 : 1;  // normal / tangential axes
    const R h_dn = cfg.h_dn, h_dt = cfg.h_dt;
    R uref_t = R(0);
    if constexpr (D == 2) uref_t = uabs[1];
    const R uref_n = uabs[0];
    const R Cv = cfg.Cv, tolR = cfg.tol;

    R dl[D], Tl = Tpred;
#pragma unroll
    for (int a = 0; a < D; ++a) dl[a] = R(0);
    R keep_dl[D], keep_T = R(0), out_du[D], out_T = R(0), out_rho = R(0);
    // level 2: the face output's constants wait in the scratch too
    if constexpr (KEEP > 1) scr.put(KS + 2, float(cfg.wb), float(cfg.we), float(cfg.Cv), 0.f);
    bool have = false, done = false, restarted = false, last_valid = false;
    int iters = 0;
    R Phi[NFC], Psi[NGC];
    for (int k = 0; k < cfg.max_iter && !done; ++k) {
        corrector_pass<D, R, EQ, SCR, OUTER_ONCE>(cells, dref, dl, Tl, uref_n + dl[0], D == 2 ? uref_t + dl[D - 1] : R(0),
                                      h_dn, h_dt, cfg.limiter, Phi, Psi, scr);
        R rho1, du[D], T1;
        const bool ok = pass_frame<D, R>(Phi, Psi, Tl, Cv, rho1, du, T1);
        iters = k + 1;
        if (!ok) {
            ++o.fallbacks;
            last_valid = false;
            if (!restarted) {
                // restart once from the frame of the pooled conserved moments of the stencil
                restarted = true;
                R r = R(0), m[D], e = R(0);
#pragma unroll
                for (int a = 0; a < D; ++a) m[a] = R(0);
#pragma unroll
                for (int s = 0; s < NCELL; ++s) {
                    const R rc = cells[s]->A[0];
                    R v2 = R(0), dcs[D];
                    rel_velocity<D, R>(cells[s], dref, false, dcs);
#pragma unroll
                    for (int a = 0; a < D; ++a) { m[a] += rc * dcs[a]; v2 += dcs[a] * dcs[a]; }
                    r += rc;
                    e += rc * (Cv * cells[s]->T + R(0.5) * v2);
                }
                r /= R(NCELL); e /= R(NCELL);
                R k2 = R(0);
#pragma unroll
                for (int a = 0; a < D; ++a) { m[a] /= R(NCELL); dl[a] = m[a] / r; k2 += m[a] * m[a]; }
                Tl = (e - R(0.5) * k2 / r) / (Cv * r);
                continue;
            }
            break;
        }
        have = true;
        last_valid = true;
        if constexpr (KEEP > 0) {
            // the kept frames wait in the scratch while the next pass runs
            scr.put(KS, float(dl[0]), float(dl[D - 1]), float(Tl), float(rho1));
            scr.put(KS + 1, float(du[0]), float(du[D - 1]), float(T1), 0.f);
        } else {
#pragma unroll
            for (int a = 0; a < D; ++a) { keep_dl[a] = dl[a]; out_du[a] = du[a]; }
            keep_T = Tl; out_T = T1; out_rho = rho1;
        }
        if (cfg.fixed_iters > 0) {
            done = iters >= cfg.fixed_iters;
        } else {
            bool c = fabs(T1 - Tl) <= tolR * Tl;
            const R sq = w_sqrt<R>(Tl);
#pragma unroll
            for (int a = 0; a < D; ++a) c = c && fabs(du[a]) <= tolR * sq;
            done = c;
        }
#pragma unroll
        for (int a = 0; a < D; ++a) dl[a] += du[a];
        Tl = T1;
    }
    o.iters = iters;
    o.done = done;
    o.have = have;
    if constexpr (KEEP > 0) {
        if (have) {
            const float4 a = scr.get(KS), b = scr.get(KS + 1);
            keep_dl[0] = R(a.x); keep_dl[D - 1] = R(a.y); keep_T = R(a.z); out_rho = R(a.w);
            out_du[0] = R(b.x); out_du[D - 1] = R(b.y); out_T = R(b.z);
        }
    }
    if (have) {
        if (!last_valid) {
            // the last pass defined no frame: recompute the last valid one
            corrector_pass<D, R, EQ, SCR, OUTER_ONCE>(cells, dref, keep_dl, keep_T, uref_n + keep_dl[0],
                                          D == 2 ? uref_t + keep_dl[D - 1] : R(0), h_dn, h_dt, cfg.limiter, Phi,
                                          Psi, scr);
        }
        // Eq. (FluxTransf) in the frame of the last valid pass's moments, with the exact
        // co-moving equilibria there: phi = (2 tau phibar + h phi^eq)/(2 tau + h)
        const R invT = w_rcp<R>(out_T);
        const R sk = w_sqrt<R>(keep_T * invT), rsq = w_sqrt<R>(invT);
        Map1<R> X(sk, (keep_T - out_T) * invT, -out_du[0] * rsq);
        Map1<R> Y = X;
        if (D == 2) Y = Map1<R>(sk, (keep_T - out_T) * invT, -out_du[D - 1] * rsq);
        R Fo[NFC], Go[NGC];
        shift_scale<D, 3, R>(Phi, X, Y, Fo);
        shift_scale<D, 2, R>(Psi, X, Y, Go);
        R wb = cfg.wb, we = cfg.we, Cvf = Cv;
        if constexpr (KEEP > 1) {
            const float4 w = scr.get(KS + 2);
            wb = R(w.x); we = R(w.y); Cvf = R(w.z);
        }
        // (the contractions written out, so that every variant rounds these alike)
        Fo[0] = fma(wb, Fo[0], we * out_rho);
#pragma unroll
        for (int k = 1; k < NFC; ++k) Fo[k] = wb * Fo[k];
        Go[0] = fma(wb, Go[0], we * (Cvf - R(0.5 * D)) * out_rho * out_T);
#pragma unroll
        for (int k = 1; k < NGC; ++k) Go[k] = wb * Go[k];
        orient<D, 3, R>(Fo, o.F, swap);
        orient<D, 2, R>(Go, o.G, swap);
        if constexpr (D == 2) {
            const R dn = keep_dl[0] + out_du[0], dt = keep_dl[1] + out_du[1];
            o.du[0] = na ? dt : dn;
            o.du[1] = na ? dn : dt;
        } else {
            o.du[0] = keep_dl[0] + out_du[0];
        }
        o.T = out_T;
    }
}

// Tiles of the learned predictor: 16 x 4 faces of each axis (the 128 rows of one MLP tile)
constexpr int kPredTileX = 16, kPredTileY = 4;
template <int D, typename R>
__host__ __device__ __forceinline__ long long pred_tiles(const Params<D, R> &P)
{
    return ((P.nx + 1 + kPredTileX - 1) / kPredTileX) * ((P.ny + 1 + kPredTileY - 1) / kPredTileY);
}

// Tile variants of the face kernel: TX x TY cells per CTA (one thread per x face and one
// per y face in 2D, one per face in 1D) and MINB CTAs per SM for the register budget.  The
// autotuner picks one per problem.
template <int D, int TX_, int TY_, int MINB_, int SCR_ = 0, bool TMA_ = false>
struct FaceVariant {
    static constexpr int TX = TX_, TY = D == 2 ? TY_ : 1, MINB = MINB_;
    static constexpr int THREADS = D == 2 ? 2 * TX_ * TY_ : TX_;
    static constexpr int SCR = SCR_;   // shared scratch level of the corrector (FP32 2D, not EQUIL)
    // interior tiles stage their box from tensor-map copies (FP32 2D with a scratch level;
    // the copies land in the corrector's scratch before the corrector uses it)
    static constexpr bool TMA = TMA_;
};

// Instantiations (MODE): FACE_PLAIN; FACE_COLLECT also writes (features, converged frame)
// pairs of sampled converged faces for the learned predictor; FACE_LEARNED starts each face
// from the learned prediction when there is one; FACE_EQUIL moves the stencil cells into
// the corrector frame by the equilibration alternative of Sec. II.C (an ablation).
// Separate instantiations, so the plain kernel carries none of them (and keeps its
// register budget).
enum { FACE_PLAIN = 0, FACE_COLLECT = 1, FACE_LEARNED = 2, FACE_EQUIL = 3 };

// one tensor-map copy of a three-dimensional box into shared memory, completing on mbar
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(tc::smem_addr(dst)), "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z),
        "r"(tc::smem_addr(mbar))
        : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *mbar, unsigned int bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_addr(mbar)), "r"(bytes) : "memory");
}

// The face kernel's body; maps (the TMA variants' tensor maps, in kernel-parameter space)
// is null for the plain launches.
template <int D, typename R, int MODE, typename V>
__device__ __forceinline__ void face_body(const Params<D, R> &P, const StageMaps *maps)
{
    constexpr bool COLLECT = MODE == FACE_COLLECT, LEARNED = MODE == FACE_LEARNED, EQUIL = MODE == FACE_EQUIL;
    constexpr int TX = V::TX, TY = V::TY;
    constexpr int BX = TX + 3, BY = D == 2 ? TY + 3 : 1;
    constexpr int NFC = NCoef<D, 3>::value, NGC = NCoef<D, 2>::value;
    using W = typename FrameWords<R>::word;
    // the staged box, and (2D) its transpose for the y-face threads: there a cell sits at
    // [x][y] with its coefficient orders and velocity components swapped, so every face
    // reads its stencil in face axes (normal first) and no transformation reorders anything
    __shared__ StagedCell<D, R> tile[BY * BX];
    __shared__ StagedCell<D, R> tileT[D == 2 ? BY * BX : 1];
    __shared__ W utile[D];
    constexpr int SCR = D == 2 && sizeof(R) == 4 && MODE != FACE_EQUIL ? V::SCR : 0;
    // TMA staging: the copied planes land in the scratch, which the corrector takes over
    // after the staging barrier
    constexpr bool TMA = V::TMA && D == 2 && sizeof(R) == 4 && SCR > 0;
    __shared__ alignas(TMA ? 128 : 16) float4 scratch[SCR ? face_scratch_slots(SCR) * V::THREADS : 1];

    const Clock &K = *P.clock;
    // t_end reached (dt = 0): the step is a no-op; tested after the staging loads, so that
    // this load's latency overlaps theirs
    const double step_dt = K.dt;
    const StepC<R> &KC = step_c<R>(K);
    const R cp = KC.cp, ce = KC.ce;

    const long long i0 = (long long)blockIdx.x * TX, j0 = (long long)blockIdx.y * TY;

    // face of this thread
    int dir = 0, tx = threadIdx.x, ty = 0;
    if (D == 2) {
        dir = threadIdx.x >= TX * TY ? 1 : 0;
        const int t = threadIdx.x - dir * TX * TY;
        tx = t % TX;
        ty = t / TX;
    }
    const long long fi = i0 + tx, fj = j0 + ty;
    bool active;
    long long fidx;
    if (dir == 0) { active = fi <= P.nx && fj < P.ny; fidx = fj * (P.nx + 1) + fi; }
    else { active = fi < P.nx && fj <= P.ny; fidx = fj * P.nx + fi; }
    W *Frm = dir == 0 ? P.xfr : P.yfr;
    const long long nf = dir == 0 ? P.nxf() : P.nyf();
    // the face's predictor frame, loaded before the staging so that the loads overlap
    W uref[D], Tpw;
#pragma unroll
    for (int a = 0; a < D; ++a) uref[a] = active ? Frm[a * nf + fidx] : fr_word(R(0));
    Tpw = active ? Frm[D * nf + fidx] : fr_word(R(1));

    // reference velocity of the tile (staged velocities are differences from it): every
    // thread reads it (the same words), so the staging needs no barrier before it
    W ut[D];
    cell_velocity<D, R>(P, i0, j0, ut);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int a = 0; a < D; ++a) utile[a] = ut[a];
    }
    // a staged cell into the box and (2D) its transpose
    auto put_staged = [&](int t, const StagedCell<D, R> &c) {
        tile[t] = c;
        if constexpr (D == 2) {
            const int bx = t % BX, by = t / BX;
            StagedCell<D, R> ct;
            orient<D, 3, R>(c.A, ct.A, true);
            orient<D, 2, R>(c.B, ct.B, true);
            ct.du[0] = c.du[1];
            ct.du[1] = c.du[0];
            ct.T = c.T;
            tileT[bx * BY + by] = ct;
        }
    };
    bool staged = false;
    if constexpr (TMA) {
        // Interior tile (the box [i0-2, i0+TX] x [j0-2, j0+TY] inside the grid, so no ghost
        // rule applies): one elected thread copies the f, g and frame planes of the box
        // [i0-4, i0+11] x [j0-2, j0+TY] (x rounded down to a 16-byte boundary) with three
        // tensor-map loads; the threads then form phi-bar-plus from shared memory, with the
        // arithmetic of the per-thread staging.  The wait is bounded: on time-out the tile
        // is flagged, the copies in flight are waited for once more, and the tile is staged
        // per thread.
        __shared__ uint64_t tma_bar;
        if (maps && i0 >= 2 && i0 + TX <= P.nx - 1 && j0 >= 2 && j0 + TY <= P.ny - 1) {
            static_assert(TX % 4 == 0 && BX + 2 <= kTmaBoxX, "the copied box covers the staged one");
            constexpr int NFS = NFC - D, PL = BY * kTmaBoxX;
            constexpr unsigned int BYTES = unsigned(PL * (NFS + NGC) * sizeof(R) + PL * (D + 1) * sizeof(W));
            static_assert(BYTES <= sizeof(float4) * face_scratch_slots(SCR) * V::THREADS, "the copies fit the scratch");
            R *raw_f = reinterpret_cast<R *>(scratch);   // [NFS][BY][kTmaBoxX]
            R *raw_g = raw_f + NFS * PL;                 // [NGC][BY][kTmaBoxX]
            W *raw_w = reinterpret_cast<W *>(raw_g + NGC * PL);   // [D+1][BY][kTmaBoxX]
            if (threadIdx.x == 0) {
                tc::mbar_init(&tma_bar, 1);
                mbar_expect_tx(&tma_bar, BYTES);
                const int x = int(i0) - 4, y = int(j0) - 2;
                tma_load_3d(raw_f, &maps->sf, x, y, 0, &tma_bar);
                tma_load_3d(raw_g, &maps->sg, x, y, 0, &tma_bar);
                tma_load_3d(raw_w, &maps->sfr, x, y, 0, &tma_bar);
            }
            __syncthreads();   // the barrier is initialised before any thread waits on it
            const bool ok = __syncthreads_and(tc::mbar_wait(&tma_bar, 0, mlp::kPolls)) != 0;
            if (ok) {
                for (int t = threadIdx.x; t < BX * BY; t += blockDim.x) {
                    const int o = (t / BX) * kTmaBoxX + t % BX + 2;
                    StagedCell<D, R> c;
#pragma unroll
                    for (int k = 0; k < NFC; ++k) {
                        const int pl = fplane<D>(k);
                        c.A[k] = pl < 0 ? R(0) : raw_f[pl * PL + o];
                    }
#pragma unroll
                    for (int k = 0; k < NGC; ++k) c.B[k] = raw_g[k * PL + o];
                    W u[D];
#pragma unroll
                    for (int a = 0; a < D; ++a) u[a] = raw_w[a * PL + o];
                    const R T = R(fr_lead(raw_w[D * PL + o]));
                    finish_bar_plus<D, R>(P, cp, ce, ut, u, T, c);
                    put_staged(t, c);
                }
                if (threadIdx.x == 0) atomicAdd(&P.diag->tma_tiles, 1ull);
                staged = true;
            } else {
                if (threadIdx.x == 0) atomicOr(&P.diag->flags, FLAG_TIMEOUT);
                tc::mbar_wait(&tma_bar, 0, mlp::kPolls);
            }
        }
    }
    // stage phi-bar-plus of the box [i0-2, i0+TX] x [j0-2, j0+TY] (1D: [i0-2, i0+TX])
    if (!staged) {
        for (int t = threadIdx.x; t < BX * BY; t += blockDim.x) {
            const int bx = t % BX, by = t / BX;
            const long long ci = i0 - 2 + bx, cj = D == 2 ? j0 - 2 + by : 0;
            StagedCell<D, R> c;
            load_cell_bar_plus<D, R>(P, ci, cj, cp, ce, ut, c);
            put_staged(t, c);
        }
    }
    if (!(step_dt > 0.0)) return;   // the same value in every thread
    __syncthreads();

    unsigned long long my_iters = 0, my_nonconv = 0, my_fallbacks = 0, my_nonphys = 0;
    if (active) {
        // stencil slots in the staged box (box coords of cell (i, j) = (i - i0 + 2, j - j0 + 2))
        const bool swap = dir == 1;
        // the face's stencil in the staged box (box coords of cell (i, j) = (i - i0 + 2, j - j0 + 2))
        Stencil<D, R> cells;
        if (swap) {   // transposed copy: the normal (y) runs along its rows
            cells.base = &tileT[int(fi - i0 + 2) * BY + int(fj - j0 + 2)];
            cells.sn = 1;
            cells.st = BY;
        } else {
            cells.base = &tile[(D == 2 ? int(fj - j0 + 2) * BX : 0) + int(fi - i0 + 2)];
            cells.sn = 1;
            cells.st = D == 2 ? BX : 0;
        }
        R *Fout = dir == 0 ? P.xf : P.yf;
        R *Gout = dir == 0 ? P.xg : P.yg;
        FaceOut<D, R> o;
        FaceCfg<R> cfg;
        cfg.h_dn = swap ? KC.h_dy : KC.h_dx;
        cfg.h_dt = D == 2 ? (swap ? KC.h_dx : KC.h_dy) : R(0);
        cfg.Cv = P.Cv_r; cfg.tol = P.tol_r; cfg.wb = KC.wb; cfg.we = KC.we;
        cfg.limiter = P.limiter; cfg.max_iter = P.max_iter; cfg.fixed_iters = P.fixed_iters;
        const R Tp = R(fr_lead(Tpw));
        const int na = swap ? 1 : 0, ta = 1 - na;
        R dref[D], uabs[D];
        dref[0] = R(fr_rel(sel(uref, na), utile[na]));
        uabs[0] = R(fr_lead(sel(uref, na)));
        if constexpr (D == 2) {
            dref[1] = R(fr_rel(sel(uref, ta), utile[ta]));
            uabs[1] = R(fr_lead(sel(uref, ta)));
        }
        // With the learned predictor on, the corrector starts from the network's prediction
        // and keeps that result only if it converges without a restart; otherwise the face
        // is solved again from the previous half step's frame, exactly as without the
        // network.  The corrector and its convergence test alone decide the result.
        W base[D];
#pragma unroll
        for (int a = 0; a < D; ++a) base[a] = uref[a];
        bool learned_first = false;
        W lrn[D + 1];
        long long ptile = 0;
        if constexpr (D == 2 && LEARNED) {
            // the predictor's tile of this face and whether the predictor ran there
            const long long pnbx = (P.nx + 1 + kPredTileX - 1) / kPredTileX;
            ptile = (fj / kPredTileY) * pnbx + fi / kPredTileX;
            const unsigned int step = (unsigned int)K.steps;
            if (P.use_learned && P.pred_active[(step & 1u) * pred_tiles(P) + ptile] == step) {
                const W *Lrm = dir == 0 ? P.xlr : P.ylr;
#pragma unroll
                for (int a = 0; a <= D; ++a) lrn[a] = Lrm[a * nf + fidx];
                const R Tl = R(fr_lead(lrn[D]));
                learned_first = Tl > R(0) && isfinite(Tl);
            }
        }
        int tot_iters = 0, tot_fallbacks = 0;
        for (int attempt = learned_first ? 0 : 1; attempt < 2; ++attempt) {
            const bool from_learned = attempt == 0;
            R dw[D], uw[D], Tw = Tp;
#pragma unroll
            for (int a = 0; a < D; ++a) { dw[a] = dref[a]; uw[a] = uabs[a]; }
            if (from_learned) {
                dw[0] = R(fr_rel(sel(lrn, na), utile[na]));
                uw[0] = R(fr_lead(sel(lrn, na)));
                if constexpr (D == 2) {
                    dw[1] = R(fr_rel(sel(lrn, ta), utile[ta]));
                    uw[1] = R(fr_lead(sel(lrn, ta)));
                }
                Tw = R(fr_lead(lrn[D]));
            }
            solve_face<D, R, EQUIL, SCR>(cells, swap, dw, uw, Tw, cfg, o,
                                         FaceScratch{scratch + (SCR ? threadIdx.x : 0), int(V::THREADS)});
            tot_iters += o.iters;
            tot_fallbacks += o.fallbacks;
            if (from_learned && o.have && o.done && o.fallbacks == 0) {
#pragma unroll
                for (int a = 0; a < D; ++a) base[a] = lrn[a];
                break;
            }
        }
        my_iters = tot_iters; my_nonconv = o.done ? 0 : 1; my_fallbacks = tot_fallbacks;
        if constexpr (D == 2 && LEARNED) {
            if (P.use_learned && (tot_iters > 1 || learned_first)) {
                const unsigned int next = (unsigned int)K.steps + 1u;
                P.pred_active[(next & 1u) * pred_tiles(P) + ptile] = next;
            }
        }
        if constexpr (COLLECT && D == 2) {
            const unsigned long long hsh = (unsigned long long)(fidx * 2 + dir + 1) * 0x9E3779B97F4A7C15ull ^
                                           (unsigned long long)(K.steps + 1) * 0xBF58476D1CE4E5B9ull;
            if (o.have && o.done && Tp > R(0) && ((hsh >> 33) % (unsigned long long)P.pair_every) == 0) {
                const float dn = float(dref[0]), dt_ = float(dref[D - 1]);
                mlp::SlotPrim sp[8];
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    sp[q] = {float(cells[q]->A[0]), float(cells[q]->du[0]) - dn, float(cells[q]->du[1]) - dt_,
                             float(cells[q]->T)};   // stencil cells are in face axes
                float f[mlp::kIn];
                mlp::features(sp, float(Tp), float(cfg.h_dn), f);
                const unsigned long long slot = atomicAdd(P.pair_count, 1ull);
                if (slot < (unsigned long long)P.pair_cap) {
                    float *row = P.pairs + slot * mlp::kPairStride;
#pragma unroll
                    for (int q = 0; q < mlp::kIn; ++q) row[q] = f[q];
                    const double rs = 1.0 / sqrt(double(Tp));
                    row[mlp::kIn + 0] = float(double(sel(o.du, na)) * rs);
                    row[mlp::kIn + 1] = float(double(sel(o.du, ta)) * rs);
                    row[mlp::kIn + 2] = float(log(double(o.T) / double(Tp)));
                    row[mlp::kIn + 3] = float(o.iters);
                }
            }
        }
        if (o.have) {
#pragma unroll
            for (int k = 0; k < NFC; ++k) Fout[k * nf + fidx] = o.F[k];
#pragma unroll
            for (int k = 0; k < NGC; ++k) Gout[k * nf + fidx] = o.G[k];
#pragma unroll
            for (int a = 0; a < D; ++a) Frm[a * nf + fidx] = fr_add(base[a], o.du[a]);
            Frm[D * nf + fidx] = fr_word(o.T);
        } else {
            ++my_nonphys;
            const R nan = R(__longlong_as_double(0x7ff8000000000000ll));
#pragma unroll
            for (int k = 0; k < NFC; ++k) Fout[k * nf + fidx] = nan;
#pragma unroll
            for (int k = 0; k < NGC; ++k) Gout[k * nf + fidx] = nan;
            fr_store(Frm[D * nf + fidx], double(nan));
        }
    }
    // warp-aggregated diagnostics
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

template <int D, typename R, int MODE, typename V>
__global__ void __launch_bounds__(V::THREADS, V::MINB)
face_kernel(const Params<D, R> P)
{
    face_body<D, R, MODE, V>(P, nullptr);
}

// the TMA-staged face variants: the tensor maps travel as a grid-constant kernel parameter,
// whose address the copies take
template <int D, typename R, int MODE, typename V>
__global__ void __launch_bounds__(V::THREADS, V::MINB)
face_tma_kernel(const Params<D, R> P, const __grid_constant__ StageMaps maps)
{
    face_body<D, R, MODE, V>(P, &maps);
}

// ---------------------------------------------------------------- cell update

// Adds -scale * H[v_n phi] for one face to the f (H) and g (G) Hermite moments of the
// cell, phi given by face coefficients in the face frame.  The face populations are first
// re-expressed in the cell frame (Eq. fluxEq), then multiplied by v_n = sqrt(T) c_n + u_n
// using c He_r(c) = He_{r+1}(c) + r He_{r-1}(c); He_4 vanishes on the D1Q4 nodes and the
// Grad forms have no moments above their order, so the product closes on the same orders.
// invTc, rsqTc: 1/T and 1/sqrt(T) of the cell frame.
template <int D, typename R, bool EQ = false>
__device__ __forceinline__ void add_face_flux(const R *Fc, const R *Gc, const R *dv, R Tbr, R Tcr, R invTc, R rsqTc,
                                              int axis, R scale, R sqTc, R un, R *H, R *G)
{
    constexpr int NFC = NCoef<D, 3>::value, NGC = NCoef<D, 2>::value;
    const R s = w_sqrt<R>(Tbr * invTc), e = (Tbr - Tcr) * invTc;
    Map1<R> X(s, e, dv[0] * rsqTc);
    Map1<R> Y = X;
    if constexpr (D == 2) Y = Map1<R>(s, e, dv[1] * rsqTc);
    R Fp[NFC], Gp[NGC];
    shift_scale<D, 3, R>(Fc, X, Y, Fp);
    shift_scale<D, 2, R>(Gc, X, Y, Gp);
    // EQ: the face populations moved into the cell frame by the equilibration alternative
    // carry fast components; the product with v_n lowers one order of them into the slow
    // orders (c He_r = He_{r+1} + r He_{r-1})
    FastEq<R> qf{}, qg{};
    if constexpr (EQ) {
        qf = fast_eq<D, 3, R>(Fp);
        qg = fast_eq<D, 2, R>(Gp);
    }
    if constexpr (D == 1) {
#pragma unroll
        for (int r = 0; r <= 3; ++r) {
            R v = un * Fp[r];
            if (r + 1 <= 3) v += sqTc * Fp[r + 1];
            if (r >= 1) v += sqTc * R(r) * Fp[r - 1];
            H[r] -= scale * v;
        }
#pragma unroll
        for (int r = 0; r <= 2; ++r) {
            R v = un * Gp[r];
            if (r + 1 <= 2) v += sqTc * Gp[r + 1];
            else if (EQ) v += sqTc * qg.at(r + 1, 0);
            if (r >= 1) v += sqTc * R(r) * Gp[r - 1];
            G[r] -= scale * v;
        }
    } else {
#pragma unroll
        for (int r = 0; r <= 3; ++r)
#pragma unroll
            for (int q = 0; q + r <= 3; ++q) {
                const int k = hidx(r, q);
                R v = un * Fp[k];
                if (axis == 0) {
                    if (r + q + 1 <= 3) v += sqTc * Fp[hidx(r + 1, q)];
                    else if (EQ && r + 1 <= 3) v += sqTc * qf.at(r + 1, q);
                    if (r >= 1) v += sqTc * R(r) * Fp[hidx(r - 1, q)];
                } else {
                    if (r + q + 1 <= 3) v += sqTc * Fp[hidx(r, q + 1)];
                    else if (EQ && q + 1 <= 3) v += sqTc * qf.at(r, q + 1);
                    if (q >= 1) v += sqTc * R(q) * Fp[hidx(r, q - 1)];
                }
                H[k] -= scale * v;
            }
#pragma unroll
        for (int r = 0; r <= 2; ++r)
#pragma unroll
            for (int q = 0; q + r <= 2; ++q) {
                const int k = hidx(r, q);
                R v = un * Gp[k];
                if (axis == 0) {
                    if (r + q + 1 <= 2) v += sqTc * Gp[hidx(r + 1, q)];
                    else if (EQ) v += sqTc * qg.at(r + 1, q);
                    if (r >= 1) v += sqTc * R(r) * Gp[hidx(r - 1, q)];
                } else {
                    if (r + q + 1 <= 2) v += sqTc * Gp[hidx(r, q + 1)];
                    else if (EQ) v += sqTc * qg.at(r, q + 1);
                    if (q >= 1) v += sqTc * R(q) * Gp[hidx(r, q - 1)];
                }
                G[k] -= scale * v;
            }
    }
}


// CFL rate of a cell frame: max over axes of (|u_a| + sqrt(T/T_L) max|c|)/dx_a, in the
// working precision (FP32 populations: the rate in FP32 is enough)
// v through a volatile move: the compiler treats the result as unknown at every use, so
// nothing derived from it is hoisted out of a loop
__device__ __forceinline__ long long opaque(long long v)
{
    long long r;
    asm volatile("mov.b64 %0, %1;" : "=l"(r) : "l"(v));
    return r;
}

template <typename R>
__device__ __forceinline__ R cell_rate_r(const R *u, R T, R inv_dx, R inv_dy, int D)
{
    const R c = sqrt(T) * R(kCHi);
    R r = (fabs(u[0]) + c) * inv_dx;
    if (D == 2) r = max(r, (fabs(u[1]) + c) * inv_dy);
    return r;
}
template <typename R>
__device__ __forceinline__ double cell_rate(const R *u, R T, R inv_dx, R inv_dy, int D)
{
    return double(cell_rate_r<R>(u, T, inv_dx, inv_dy, D));
}

// block max of a non-negative double, then the last block turns the grid max into the
// next time step (CFL condition, clipped to t_end) and advances the clock
// Non-negative doubles order like their bit patterns, so the maximum is taken on the
// patterns with integer operations (no FP64 instructions).  Only thread 0 waits for the
// grid-wide atomics; the other warps leave after the block's maximum is formed.
__device__ __forceinline__ unsigned long long warp_max_bits(unsigned long long b)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long x = __shfl_down_sync(0xffffffffu, b, o);
        b = x > b ? x : b;
    }
    return b;
}
__device__ __forceinline__ void reduce_rate_and_advance(Clock *clock, double rate, bool advance)
{
    __shared__ unsigned long long red[32];
    unsigned long long b = (unsigned long long)__double_as_longlong(rate);
    if (b > 0x7ff0000000000000ull) b = 0ull;   // a NaN (or a negative) rate counts as none
    b = warp_max_bits(b);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = b;
    __syncthreads();
    if (threadIdx.x >= 32) return;
    const int nw = (blockDim.x + 31) >> 5;
    b = warp_max_bits(threadIdx.x < nw ? red[threadIdx.x] : 0ull);
    bool last = false;
    if (threadIdx.x == 0) {
        atomicMax(&clock->rate_bits, b);
        __threadfence();
        const unsigned int nb = gridDim.x * gridDim.y * gridDim.z;
        last = atomicAdd(&clock->blocks_done, 1u) == nb - 1;
    }
    if (last) {
        __threadfence();
        const double rmax = __longlong_as_double((long long)atomicAdd(&clock->rate_bits, 0ull));
        double t = clock->t;
        if (advance) {
            t += clock->dt;
            clock->t = t;
            clock->steps += 1;
        }
        double dt = clock->cfl / rmax;
        if (clock->t_end > 0.0) {
            if (t >= clock->t_end) dt = 0.0;
            else if (t + dt > clock->t_end) dt = clock->t_end - t;
        }
        set_step_constants(*clock, dt);
        clock->rate_bits = 0ull;
        clock->blocks_done = 0u;
    }
}

// Step 1 of the next step after the update: the new co-moving frame from the conserved
// moments (H: f, G: g Hermite moments in the old cell frame) and the Grad projection into
// it (f third order, g second order).  The frame changes by increments formed relative to
// the old frame, du and dT (T' = T (1 + dT)), which the caller applies to its own
// representation of the frame.
template <int D, typename R>
__device__ __forceinline__ bool cell_finish(const R *H, const R *G, R invTc, R sqTc, R Cv, R *Ho, R *Go, R *du, R &dT)
{
    const R rsqTc = invTc * sqTc;
    const R rn = H[0];
    const R irn = w_rcp<R>(rn);
    R k2 = R(0), trH;
    if constexpr (D == 1) {
        du[0] = sqTc * H[1] * irn;
        k2 = du[0] * du[0];
        trH = H[2];
    } else {
        du[0] = sqTc * H[hidx(1, 0)] * irn;
        du[1] = sqTc * H[hidx(0, 1)] * irn;
        k2 = du[0] * du[0] + du[1] * du[1];
        trH = H[hidx(2, 0)] + H[hidx(0, 2)];
    }
    // T'/T - 1 = (1/2 tr H + G0/T - (Cv - D/2) rho' - rho' |du|^2/(2T)) / (Cv rho')
    dT = w_div<R>(R(0.5) * trH + G[0] * invTc - (Cv - R(0.5 * D)) * rn - R(0.5) * rn * k2 * invTc, Cv * rn);
    const bool ok = rn > R(0) && R(1) + dT > R(0) && isfinite(rn) && isfinite(dT);
    // s^2 = T/T' = 1/(1 + dT/T), e = s^2 - 1, d = -du/sqrt(T')
    const R s2 = w_rcp<R>(R(1) + dT);
    const R sc = w_sqrt<R>(s2), e = -dT * s2;
    const R rsqn = rsqTc * sc;
    Map1<R> X(sc, e, -du[0] * rsqn);
    Map1<R> Y = X;
    if constexpr (D == 2) Y = Map1<R>(sc, e, -du[1] * rsqn);
    shift_scale<D, 3, R>(H, X, Y, Ho);
    shift_scale<D, 2, R>(G, X, Y, Go);
    return ok;
}

// Step 3 of Sec. III.B.4 (flux into the cell frame, Eq. fluxEq; update, Eqs.
// FinalUpdateDUGKS) fused with step 1 of the next step (re-expression in the new co-moving
// frame from the conserved moments) and the CFL reduction.  The frame (u, T) advances by
// increments formed from the Hermite moments relative to the old frame (u' = u + du,
// T' = T (1 + dT/T)), so no kinetic energy of the frame enters.
// EQ: the face populations enter the cell frame by the equilibration alternative (Sec. II.C).
template <int D, typename R, int THREADS, int MINB = 1, bool EQ = false, bool GS = false>
__global__ void __launch_bounds__(THREADS, MINB)
cell_kernel(const Params<D, R> P)
{
    constexpr int NFC = NCoef<D, 3>::value, NGC = NCoef<D, 2>::value;
    const Clock &K = *P.clock;
    if (!(K.dt > 0.0)) return;
    const long long n = P.ncell();
    R rate = R(0);
    using W = typename FrameWords<R>::word;
    const StepC<R> &KC = step_c<R>(K);
    auto update = [&](const long long c) {
        // GS: the plane strides pass through an opaque copy, so that the compiler forms the
        // planes' offsets per cell instead of holding them all in registers across cells
        const long long n = GS ? opaque(P.ncell()) : P.ncell();
        const long long i = c % P.nx, j = c / P.nx;
        W uc[D];
#pragma unroll
        for (int a = 0; a < D; ++a) uc[a] = P.sfr[a * n + c];
        const W Tc = P.sfr[D * n + c];
        const R rho = P.sf[c];
        const R ca = KC.ca, cb = KC.cb, Cv = P.Cv_r;
        const R Tcr = R(fr_lead(Tc));
        const R invTc = w_rcp<R>(Tcr), rsqTc = w_sqrt<R>(invTc), sqTc = Tcr * rsqTc;
        // collision part of Eqs. (FinalUpdateDUGKS) in Hermite moments of the cell frame
        R H[NFC], G[NGC];
#pragma unroll
        for (int k = 0; k < NFC; ++k) {
            const int pl = fplane<D>(k);
            H[k] = pl < 0 ? R(0) : ca * P.sf[pl * n + c];
        }
        H[0] += cb * rho;
#pragma unroll
        for (int k = 0; k < NGC; ++k) G[k] = ca * P.sg[k * n + c];
        G[0] += cb * (Cv - R(0.5 * D)) * rho * Tcr;
        // fluxes through the 2D faces
        const long long nxf = GS ? opaque(P.nxf()) : P.nxf();
        const R sx = KC.dt_dx;
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const long long f = j * (P.nx + 1) + i + side;
            R Fc[NFC], Gc[NGC], dv[D];
#pragma unroll
            for (int k = 0; k < NFC; ++k) Fc[k] = P.xf[k * nxf + f];
#pragma unroll
            for (int k = 0; k < NGC; ++k) Gc[k] = P.xg[k * nxf + f];
#pragma unroll
            for (int a = 0; a < D; ++a) dv[a] = R(fr_rel(P.xfr[a * nxf + f], uc[a]));
            const R Tb = R(fr_lead(P.xfr[D * nxf + f]));
            add_face_flux<D, R, EQ>(Fc, Gc, dv, Tb, Tcr, invTc, rsqTc, 0, side ? sx : -sx, sqTc, R(fr_lead(uc[0])), H, G);
        }
        if constexpr (D == 2) {
            const long long nyf = GS ? opaque(P.nyf()) : P.nyf();
            const R sy = KC.dt_dy;
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const long long f = (j + side) * P.nx + i;
                R Fc[NFC], Gc[NGC], dv[D];
#pragma unroll
                for (int k = 0; k < NFC; ++k) Fc[k] = P.yf[k * nyf + f];
#pragma unroll
                for (int k = 0; k < NGC; ++k) Gc[k] = P.yg[k * nyf + f];
#pragma unroll
                for (int a = 0; a < D; ++a) dv[a] = R(fr_rel(P.yfr[a * nyf + f], uc[a]));
                const R Tb = R(fr_lead(P.yfr[D * nyf + f]));
                add_face_flux<D, R, EQ>(Fc, Gc, dv, Tb, Tcr, invTc, rsqTc, 1, side ? sy : -sy, sqTc, R(fr_lead(uc[1])), H, G);
            }
        }
        R Ho[NFC], Go[NGC], du[D], dT;
        bool ok = cell_finish<D, R>(H, G, invTc, sqTc, Cv, Ho, Go, du, dT);
        W un[D];
        R unr[D];
#pragma unroll
        for (int a = 0; a < D; ++a) {
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
        for (int k = 0; k < NFC; ++k) {
            const int pl = fplane<D>(k);
            if (pl >= 0) P.sf[pl * n + c] = Ho[k];
        }
#pragma unroll
        for (int k = 0; k < NGC; ++k) P.sg[k * n + c] = Go[k];
#pragma unroll
        for (int a = 0; a < D; ++a) P.sfr[a * n + c] = un[a];
        P.sfr[D * n + c] = Tn;
        if (ok) rate = max(rate, cell_rate_r<R>(unr, Tnr, KC.inv_dx, KC.inv_dy, D));
    };
    const long long c0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if constexpr (GS) {
        // grid-stride over the cells (the launch caps the grid), so that the block's rate
        // reduction and the time-step atomics serve several cells per thread
        for (long long c = c0; c < n; c += (long long)gridDim.x * blockDim.x) update(c);
    } else if (c0 < n) {
        update(c0);
    }
    reduce_rate_and_advance(P.clock, double(rate), true);
}

// ------------------------------------------------------------ fused step

// Tile variants of the fused step: TX x TY cells per CTA, whose faces (TX+1) x TY along x
// and TX x (TY+1) along y are all solved in the CTA (the faces on the tile's far edges are
// also solved by the neighbouring tile), one thread per face; MINB CTAs per SM.
template <int D, int TX_, int TY_, int MINB_>
struct StepVariant {
    static constexpr int TX = TX_, TY = D == 2 ? TY_ : 1, MINB = MINB_;
    static constexpr int NXF = (TX + 1) * TY, NYF = D == 2 ? TX * (TY + 1) : 0, NF = NXF + NYF;
    static constexpr int THREADS = ((NF + 31) / 32) * 32;
};

// the faces' populations (coefficients in the face frame, x, y order) and frames in shared
// memory, one array per component (NF faces each), so that neighbouring threads touch
// neighbouring words
template <int D, typename R, int NF>
struct FaceRecs {
    R F[NCoef<D, 3>::value][NF];
    R G[NCoef<D, 2>::value][NF];
    typename FrameWords<R>::word fr[D + 1][NF];
};

// One whole step (Sec. III.B.4) of a tile in one kernel: the CTA stages phi-bar-plus of the
// box [i0-2, i0+TX+1] x [j0-2, j0+TY+1] (steps 1 and 2a), solves every face of its cells by
// the predictor-corrector (step 2b) into shared memory, and updates its cells from those
// faces (step 3, with step 1 of the next step and the CFL rate, as cell_kernel).  The state
// and the face frames are read from sf, sg, sfr, xfr, yfr and written to their *_n copies,
// so no CTA sees another's new values; faces on a tile's far edges are solved twice (by
// both tiles) and written by their owner only.  Face populations never reach global memory.
template <int D, typename R, typename V>
__global__ void __launch_bounds__(V::THREADS, V::MINB)
step_kernel(const Params<D, R> P)
{
    constexpr int TX = V::TX, TY = V::TY;
    constexpr int BX = TX + 4, BY = D == 2 ? TY + 4 : 1;
    constexpr int NFC = NCoef<D, 3>::value, NGC = NCoef<D, 2>::value;
    using W = typename FrameWords<R>::word;
    __shared__ StagedCell<D, R> tile[BY * BX];
    __shared__ StagedCell<D, R> tileT[D == 2 ? BY * BX : 1];
    __shared__ FaceRecs<D, R, V::NF> frec;
    __shared__ W utile[D];

    const Clock &K = *P.clock;
    if (!(K.dt > 0.0)) return;  // t_end reached: the step is a no-op
    const StepC<R> &KC = step_c<R>(K);
    const R cp = KC.cp, ce = KC.ce;
    const long long i0 = (long long)blockIdx.x * TX, j0 = (long long)blockIdx.y * TY;
    if (threadIdx.x == 0) cell_velocity<D, R>(P, i0, j0, utile);
    __syncthreads();
    for (int t = threadIdx.x; t < BX * BY; t += blockDim.x) {
        const int bx = t % BX, by = t / BX;
        const long long ci = i0 - 2 + bx, cj = D == 2 ? j0 - 2 + by : 0;
        if constexpr (D == 2) {
            StagedCell<D, R> c;
            load_cell_bar_plus<D, R>(P, ci, cj, cp, ce, utile, c);
            tile[t] = c;
            StagedCell<D, R> ct;
            orient<D, 3, R>(c.A, ct.A, true);
            orient<D, 2, R>(c.B, ct.B, true);
            ct.du[0] = c.du[1];
            ct.du[1] = c.du[0];
            ct.T = c.T;
            tileT[bx * BY + by] = ct;
        } else {
            load_cell_bar_plus<D, R>(P, ci, cj, cp, ce, utile, tile[t]);
        }
    }
    __syncthreads();

    // ---- the faces of the tile's cells
    static_assert(V::THREADS >= V::NF && V::THREADS >= TX * TY, "one face and at most one cell per thread");
    unsigned long long my_iters = 0, my_faces = 0, my_nonconv = 0, my_fallbacks = 0, my_nonphys = 0;
    const int f = threadIdx.x;
    if (f < V::NF) do {
        const int dir = f >= V::NXF ? 1 : 0;
        int tx, ty;
        if (dir == 0) { tx = f % (TX + 1); ty = f / (TX + 1); }
        else { tx = (f - V::NXF) % TX; ty = (f - V::NXF) / TX; }
        const long long fi = i0 + tx, fj = j0 + ty;
        bool active, owned;
        long long fidx;
        if (dir == 0) {
            active = fi <= P.nx && fj < P.ny;
            owned = tx < TX || fi == P.nx;
            fidx = fj * (P.nx + 1) + fi;
        } else {
            active = fi < P.nx && fj <= P.ny;
            owned = ty < TY || fj == P.ny;
            fidx = fj * P.nx + fi;
        }
        if (!active) break;
        const bool swap = dir == 1;
        Stencil<D, R> cells;
        if (swap) {
            cells.base = &tileT[int(fi - i0 + 2) * BY + int(fj - j0 + 2)];
            cells.sn = 1;
            cells.st = BY;
        } else {
            cells.base = &tile[(D == 2 ? int(fj - j0 + 2) * BX : 0) + int(fi - i0 + 2)];
            cells.sn = 1;
            cells.st = D == 2 ? BX : 0;
        }
        const W *Frm = dir == 0 ? P.xfr : P.yfr;
        W *Frm_n = dir == 0 ? P.xfr_n : P.yfr_n;
        const long long nf = dir == 0 ? P.nxf() : P.nyf();
        W uref[D];
#pragma unroll
        for (int a = 0; a < D; ++a) uref[a] = Frm[a * nf + fidx];
        FaceCfg<R> cfg;
        cfg.h_dn = swap ? KC.h_dy : KC.h_dx;
        cfg.h_dt = D == 2 ? (swap ? KC.h_dx : KC.h_dy) : R(0);
        cfg.Cv = P.Cv_r; cfg.tol = P.tol_r; cfg.wb = KC.wb; cfg.we = KC.we;
        cfg.limiter = P.limiter; cfg.max_iter = P.max_iter; cfg.fixed_iters = P.fixed_iters;
        const R Tp = R(fr_lead(Frm[D * nf + fidx]));
        const int na = swap ? 1 : 0, ta = 1 - na;
        R dref[D], uabs[D];
        dref[0] = R(fr_rel(sel(uref, na), utile[na]));
        uabs[0] = R(fr_lead(sel(uref, na)));
        if constexpr (D == 2) {
            dref[1] = R(fr_rel(sel(uref, ta), utile[ta]));
            uabs[1] = R(fr_lead(sel(uref, ta)));
        }
        FaceOut<D, R> o;
        solve_face<D, R, false, 0, sizeof(R) == 4>(cells, swap, dref, uabs, Tp, cfg, o);
        if (owned) {
            my_iters += o.iters;
            my_faces += 1;
            my_fallbacks += o.fallbacks;
            if (!o.done) ++my_nonconv;
        }
        W frw[D + 1];
        if (o.have) {
#pragma unroll
            for (int k = 0; k < NFC; ++k) frec.F[k][f] = o.F[k];
#pragma unroll
            for (int k = 0; k < NGC; ++k) frec.G[k][f] = o.G[k];
#pragma unroll
            for (int a = 0; a < D; ++a) frw[a] = fr_add(uref[a], o.du[a]);
            frw[D] = fr_word(o.T);
        } else {
            if (owned) ++my_nonphys;
            const R nan = R(__longlong_as_double(0x7ff8000000000000ll));
#pragma unroll
            for (int k = 0; k < NFC; ++k) frec.F[k][f] = nan;
#pragma unroll
            for (int k = 0; k < NGC; ++k) frec.G[k][f] = nan;
#pragma unroll
            for (int a = 0; a < D; ++a) frw[a] = uref[a];
            fr_store(frw[D], double(nan));
        }
#pragma unroll
        for (int a = 0; a <= D; ++a) frec.fr[a][f] = frw[a];
        if (owned) {
#pragma unroll
            for (int a = 0; a <= D; ++a) Frm_n[a * nf + fidx] = frw[a];
        }
    } while (false);
    __syncthreads();

    // ---- the tile's cells: Eqs. (fluxEq), (FinalUpdateDUGKS), the new frame and the CFL rate
    double rate = 0.0;
    const long long n = P.ncell();
    const int t = threadIdx.x;
    if (t < TX * TY) do {
        const int tx = t % TX, ty = t / TX;
        const long long i = i0 + tx, j = j0 + ty;
        if (i >= P.nx || (D == 2 && j >= P.ny)) break;
        const long long c = j * P.nx + i;
        W uc[D];
#pragma unroll
        for (int a = 0; a < D; ++a) uc[a] = P.sfr[a * n + c];
        const W Tc = P.sfr[D * n + c];
        const R rho = P.sf[c];
        const R ca = KC.ca, cb = KC.cb, Cv = P.Cv_r;
        const R Tcr = R(fr_lead(Tc));
        const R invTc = w_rcp<R>(Tcr), rsqTc = w_sqrt<R>(invTc), sqTc = Tcr * rsqTc;
        R H[NFC], G[NGC];
#pragma unroll
        for (int k = 0; k < NFC; ++k) {
            const int pl = fplane<D>(k);
            H[k] = pl < 0 ? R(0) : ca * P.sf[pl * n + c];
        }
        H[0] += cb * rho;
#pragma unroll
        for (int k = 0; k < NGC; ++k) G[k] = ca * P.sg[k * n + c];
        G[0] += cb * (Cv - R(0.5 * D)) * rho * Tcr;
        auto face_flux = [&](int f, int axis, R scale, R un) {
            R Fc[NFC], Gc[NGC], dv[D];
#pragma unroll
            for (int k = 0; k < NFC; ++k) Fc[k] = frec.F[k][f];
#pragma unroll
            for (int k = 0; k < NGC; ++k) Gc[k] = frec.G[k][f];
#pragma unroll
            for (int a = 0; a < D; ++a) dv[a] = R(fr_rel(frec.fr[a][f], uc[a]));
            add_face_flux<D, R>(Fc, Gc, dv, R(fr_lead(frec.fr[D][f])), Tcr, invTc, rsqTc, axis, scale, sqTc, un, H, G);
        };
        const R sx = KC.dt_dx;
        face_flux(ty * (TX + 1) + tx, 0, -sx, R(fr_lead(uc[0])));
        face_flux(ty * (TX + 1) + tx + 1, 0, sx, R(fr_lead(uc[0])));
        if constexpr (D == 2) {
            const R sy = KC.dt_dy;
            face_flux(V::NXF + ty * TX + tx, 1, -sy, R(fr_lead(uc[1])));
            face_flux(V::NXF + (ty + 1) * TX + tx, 1, sy, R(fr_lead(uc[1])));
        }
        R Ho[NFC], Go[NGC], du[D], dT;
        bool ok = cell_finish<D, R>(H, G, invTc, sqTc, Cv, Ho, Go, du, dT);
        W un[D];
        R unr[D];
#pragma unroll
        for (int a = 0; a < D; ++a) {
            un[a] = fr_add(uc[a], du[a]);
            unr[a] = R(fr_lead(un[a]));
        }
        const W Tn = fr_add(Tc, Tcr * dT);
        const R Tnr = R(fr_lead(Tn));
        ok = ok && Tnr > R(0) && isfinite(Tnr);
        if (!ok) {
            ++my_nonphys;
            atomicCAS((unsigned long long *)&P.diag->first_bad, (unsigned long long)-1ll, (unsigned long long)c);
        }
#pragma unroll
        for (int k = 0; k < NFC; ++k) {
            const int pl = fplane<D>(k);
            if (pl >= 0) P.sf_n[pl * n + c] = Ho[k];
        }
#pragma unroll
        for (int k = 0; k < NGC; ++k) P.sg_n[k * n + c] = Go[k];
#pragma unroll
        for (int a = 0; a < D; ++a) P.sfr_n[a * n + c] = un[a];
        P.sfr_n[D * n + c] = Tn;
        if (ok) rate = cell_rate<R>(unr, Tnr, KC.inv_dx, KC.inv_dy, D);
    } while (false);
    // warp-aggregated diagnostics
    my_iters = warp_sum_count(my_iters);
    my_faces = warp_sum_count(my_faces);
    my_nonconv = warp_sum_count(my_nonconv);
    my_fallbacks = warp_sum_count(my_fallbacks);
    my_nonphys = warp_sum_count(my_nonphys);
    if ((threadIdx.x & 31) == 0) {
        if (my_faces) { atomicAdd(&P.diag->face_iters, my_iters); atomicAdd(&P.diag->face_solves, my_faces); }
        if (my_nonconv) { atomicAdd(&P.diag->nonconv, my_nonconv); atomicOr(&P.diag->flags, FLAG_NOT_CONVERGED); }
        if (my_fallbacks) atomicAdd(&P.diag->fallbacks, my_fallbacks);
        if (my_nonphys) { atomicAdd(&P.diag->nonphys, my_nonphys); atomicOr(&P.diag->flags, FLAG_NONPHYSICAL); }
    }
    reduce_rate_and_advance(P.clock, rate, true);
}

// ------------------------------------------------------------ initial condition

// Equilibria of Eqs. (feqPond), (geqPond) in each cell's frame from primitive fields.
template <int D, typename R>
__global__ void init_cells_kernel(const Params<D, R> P, const double *rho, const double *ux, const double *uy, const double *p)
{
    constexpr int NFS = Params<D, R>::NFS, NGC = NCoef<D, 2>::value;
    const long long n = P.ncell();
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double rate = 0.0;
    if (c < n) {
        const double r = rho[c], T = p[c] / r;
        double u[2] = {ux[c], (D == 2 && uy) ? uy[c] : 0.0};
        P.sf[c] = R(r);
#pragma unroll
        for (int k = 1; k < NFS; ++k) P.sf[k * n + c] = R(0);
        P.sg[c] = R((P.Cv - 0.5 * D) * r * T);
#pragma unroll
        for (int k = 1; k < NGC; ++k) P.sg[k * n + c] = R(0);
#pragma unroll
        for (int a = 0; a < D; ++a) fr_store(P.sfr[a * n + c], u[a]);
        fr_store(P.sfr[D * n + c], T);
        const bool ok = r > 0.0 && T > 0.0 && isfinite(r) && isfinite(T);
        if (!ok) {
            atomicOr(&P.diag->flags, FLAG_NONPHYSICAL);
            atomicAdd(&P.diag->nonphys, 1ull);
            atomicCAS((unsigned long long *)&P.diag->first_bad, (unsigned long long)-1ll, (unsigned long long)c);
        }
        const R ur[2] = {R(u[0]), R(u[1])};
        rate = ok ? cell_rate<R>(ur, R(T), R(1.0 / P.dx), R(1.0 / P.dy), D) : 0.0;
    }
    reduce_rate_and_advance(P.clock, rate, false);
}

// conserved moments (rho, rho u, rho E) of a resolved cell, from its stored state
template <int D, typename R>
__device__ __forceinline__ void cell_conserved(const Params<D, R> &P, long long i, long long j, double &r, double *m, double &E)
{
    long long idx = 0;
    int flip = 0;
    const int side = resolve(P, i, j, &idx, &flip);
    double u[2] = {0.0, 0.0}, T;
    if (side >= 0) {
        r = P.inflow[side][0];
        T = P.inflow[side][3] / r;
        u[0] = P.inflow[side][1];
        u[1] = P.inflow[side][2];
    } else {
        const long long n = P.ncell();
        r = double(P.sf[idx]);
#pragma unroll
        for (int a = 0; a < D; ++a) u[a] = fr_value(P.sfr[a * n + idx]);
        T = fr_value(P.sfr[D * n + idx]);
    }
    if (flip & 1) u[0] = -u[0];
    if (flip & 2) u[1] = -u[1];
    double k2 = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a) { m[a] = r * u[a]; k2 += u[a] * u[a]; }
    E = r * (P.Cv * T + 0.5 * k2);
}

// face predictor before the first step: frame of the pooled moments of the two cells
template <int D, typename R>
__global__ void init_faces_kernel(const Params<D, R> P)
{
    const long long nxf = P.nxf(), nyf = D == 2 ? P.nyf() : 0;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nxf + nyf) return;
    const bool xdir = t < nxf;
    const long long f = xdir ? t : t - nxf;
    long long ai, aj, bi, bj;
    if (xdir) { const long long i = f % (P.nx + 1), j = f / (P.nx + 1); ai = i - 1; aj = j; bi = i; bj = j; }
    else { const long long i = f % P.nx, j = f / P.nx; ai = i; aj = j - 1; bi = i; bj = j; }
    double ra, ma[2] = {0, 0}, Ea, rb, mb[2] = {0, 0}, Eb;
    cell_conserved<D, R>(P, ai, aj, ra, ma, Ea);
    cell_conserved<D, R>(P, bi, bj, rb, mb, Eb);
    const double r = 0.5 * (ra + rb), E = 0.5 * (Ea + Eb);
    double k2 = 0.0, u[2];
#pragma unroll
    for (int a = 0; a < D; ++a) { const double m = 0.5 * (ma[a] + mb[a]); u[a] = m / r; k2 += m * m; }
    typename FrameWords<R>::word *Frm = xdir ? P.xfr : P.yfr;
    const long long nf = xdir ? nxf : nyf;
#pragma unroll
    for (int a = 0; a < D; ++a) fr_store(Frm[a * nf + f], u[a]);
    fr_store(Frm[D * nf + f], (E - 0.5 * k2 / r) / (P.Cv * r));
}

// ------------------------------------------------------- learned gauge predictor

// Before the face corrector of a step: the learned prediction of the converged frame of
// every face of the active tiles (features as in mlp::features), written beside the
// previous half step's frame.
// Persistent CTAs (mlp::kInferCtasPerSm per SM) stage the network once and loop over tiles
// of 16 x 4 cells: the 64 x-faces and 64 y-faces of a tile are the 128 rows of one MLP tile
// (the face kernel's mapping), and the (16+3) x (4+3) cells they read are staged once in
// shared memory as (rho, velocity relative to the tile's reference, T) in FP32.
constexpr int kPredTX = kPredTileX, kPredTY = kPredTileY;
static_assert(2 * kPredTX * kPredTY == mlp::kRows, "one face per MLP row");

template <typename R>
__global__ void __launch_bounds__(mlp::kThreads, mlp::kInferCtasPerSm)
gauge_predict_kernel(const Params<2, R> P)
{
    using W = typename FrameWords<R>::word;
    constexpr int BX = kPredTX + 3, BY = kPredTY + 3;
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ float4 box[BY * BX];   // rho, u - u_ref, v - v_ref, T
    __shared__ W uref_tile[2];
    const Clock &K = *P.clock;
    if (!(K.dt > 0.0)) return;
    const long long nxf = P.nxf(), nyf = P.nyf(), n = P.ncell();
    if (threadIdx.x < 32) tc::tmem_alloc(&tmem_base, mlp::kInferTmemCols);
    if (threadIdx.x == 0) tc::mbar_init(&mbar, 1);
    mlp::stage_infer(P.mlp, sm);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    uint32_t phase = 0;
    bool ok = true;
    const int nbx = int((P.nx + 1 + kPredTX - 1) / kPredTX), nby = int((P.ny + 1 + kPredTY - 1) / kPredTY);
    const int ntiles = nbx * nby;
    // this thread's face within a tile
    const int dir = threadIdx.x >= kPredTX * kPredTY ? 1 : 0;
    const int tl = threadIdx.x - dir * kPredTX * kPredTY, tx = tl % kPredTX, ty = tl / kPredTX;
    const int na = dir, ta = 1 - dir;
    const unsigned int step = (unsigned int)K.steps;
    const unsigned int *active = P.pred_active + (step & 1u) * (unsigned)ntiles;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        // only tiles where a face needed more than one pass (or used a prediction) in the
        // previous step: elsewhere the previous half step's frame is already converged
        if (active[tile] != step) continue;
        const long long i0 = (long long)(tile % nbx) * kPredTX, j0 = (long long)(tile / nbx) * kPredTY;
        if (threadIdx.x == 0) cell_velocity<2, R>(P, i0, j0, uref_tile);
        __syncthreads();
        for (int t = threadIdx.x; t < BX * BY; t += blockDim.x) {
            const long long ci = i0 - 2 + t % BX, cj = j0 - 2 + t / BX;
            long long idx = 0;
            int flip = 0;
            const int side = resolve(P, ci, cj, &idx, &flip);
            W u[2];
            float rho, T;
            if (side >= 0) {
                rho = float(P.inflow[side][0]);
                fr_store(u[0], P.inflow[side][1]);
                fr_store(u[1], P.inflow[side][2]);
                T = float(P.inflow[side][3] / P.inflow[side][0]);
            } else {
                rho = float(P.sf[idx]);
                u[0] = P.sfr[idx];
                u[1] = P.sfr[n + idx];
                T = float(fr_lead(P.sfr[2 * n + idx]));
            }
            if (flip & 1) u[0] = fr_neg(u[0]);
            if (flip & 2) u[1] = fr_neg(u[1]);
            box[t] = make_float4(rho, float(fr_rel(u[0], uref_tile[0])), float(fr_rel(u[1], uref_tile[1])), T);
        }
        __syncthreads();
        const long long fi = i0 + tx, fj = j0 + ty;
        const bool valid = dir == 0 ? (fi <= P.nx && fj < P.ny) : (fi < P.nx && fj <= P.ny);
        const long long fidx = dir == 0 ? fj * (P.nx + 1) + fi : fj * P.nx + fi;
        const long long nfd = dir ? nyf : nxf;
        W *Frm = dir ? P.yfr : P.xfr;
        W uref[2];
        R Tp = R(0);
        float f[mlp::kIn];
        if (valid) {
            uref[0] = Frm[fidx];
            uref[1] = Frm[nfd + fidx];
            Tp = R(fr_lead(Frm[2 * nfd + fidx]));
            const float dref[2] = {float(fr_rel(uref[0], uref_tile[0])), float(fr_rel(uref[1], uref_tile[1]))};
            // stencil slots LL, L, R, RR, L-t, L+t, R-t, R+t in box coordinates (x, y)
            const int bx0 = tx + 2, by0 = ty + 2;
            int sx[8], sy[8];
            if (dir == 0) {
                const int ox[8] = {-2, -1, 0, 1, -1, -1, 0, 0}, oy[8] = {0, 0, 0, 0, -1, 1, -1, 1};
#pragma unroll
                for (int q = 0; q < 8; ++q) { sx[q] = bx0 + ox[q]; sy[q] = by0 + oy[q]; }
            } else {
                const int ox[8] = {0, 0, 0, 0, -1, 1, -1, 1}, oy[8] = {-2, -1, 0, 1, -1, -1, 0, 0};
#pragma unroll
                for (int q = 0; q < 8; ++q) { sx[q] = bx0 + ox[q]; sy[q] = by0 + oy[q]; }
            }
            mlp::SlotPrim sp[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float4 c = box[sy[q] * BX + sx[q]];
                const float du[2] = {c.y - dref[0], c.z - dref[1]};
                sp[q] = {c.x, du[na], du[ta], c.w};
            }
            mlp::features(sp, float(Tp), dir ? K.kf.h_dy : K.kf.h_dx, f);
        } else {
#pragma unroll
            for (int q = 0; q < mlp::kIn; ++q) f[q] = 0.f;
        }
#pragma unroll
        for (int k0 = 0; k0 < mlp::kIn; k0 += 8) mlp::put_bf16x8(sm + mlp::iX, threadIdx.x, k0, mlp::kIn, f + k0);
        float out[mlp::kOutP];
        ok = mlp::forward_infer(sm, tmem, &mbar, phase, out);
        if (ok && valid) {
            // the prediction for this step's corrector (T not finite: none, the gate or an
            // undefined predictor frame); the previous half step's frame stays in place
            const float y0 = fminf(fmaxf(out[0], -5.f), 5.f), y1 = fminf(fmaxf(out[1], -5.f), 5.f);
            const float y2 = fminf(fmaxf(out[2], -5.f), 5.f);
            const float ymax = fmaxf(fabsf(y0), fmaxf(fabsf(y1), fabsf(y2)));
            const bool use = Tp > R(0) && ymax > P.gauge_gate && ymax <= P.gauge_trust;
            W *Lrm = dir ? P.ylr : P.xlr;
            if (use) {
                const R sq = sqrt(Tp);
                Lrm[na * nfd + fidx] = fr_add(uref[na], sq * R(y0));
                Lrm[ta * nfd + fidx] = fr_add(uref[ta], sq * R(y1));
                Lrm[2 * nfd + fidx] = fr_word(R(Tp * R(__expf(y2))));
            } else {
                Lrm[2 * nfd + fidx] = fr_word(R(__int_as_float(0x7fc00000)));
            }
        }
    }
    if (!ok && threadIdx.x == 0) atomicOr(P.mlp_err, 1u);
    mlp::drain(&mbar, phase, ok);
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) tc::tmem_free(tmem, mlp::kInferTmemCols);
}

// ---------------------------------------------------------------- read-back kernels

// conserved fields per cell (lab frame, FP64)
template <int D, typename R>
__global__ void conserved_kernel(const Params<D, R> P, double *rho, double *mx, double *my, double *E)
{
    const long long n = P.ncell();
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    double r, m[2] = {0, 0}, e;
    cell_conserved<D, R>(P, c % P.nx, c / P.nx, r, m, e);
    if (rho) rho[c] = r;
    if (mx) mx[c] = m[0];
    if (my) my[c] = D == 2 ? m[1] : 0.0;
    if (E) E[c] = e;
}

// stored state as full coefficient arrays [cells][NFC], [cells][NGC] and frames [cells][D+1]
template <int D, typename R>
__global__ void export_state_kernel(const Params<D, R> P, double *cf, double *cg, double *fr)
{
    constexpr int NFC = NCoef<D, 3>::value, NGC = NCoef<D, 2>::value;
    const long long n = P.ncell();
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    if (cf)
#pragma unroll
        for (int k = 0; k < NFC; ++k) {
            const int pl = fplane<D>(k);
            cf[c * NFC + k] = pl < 0 ? 0.0 : double(P.sf[pl * n + c]);
        }
    if (cg)
#pragma unroll
        for (int k = 0; k < NGC; ++k) cg[c * NGC + k] = double(P.sg[k * n + c]);
    if (fr)
#pragma unroll
        for (int a = 0; a <= D; ++a) fr[c * (D + 1) + a] = fr_value(P.sfr[a * n + c]);
}

}  // namespace pond
