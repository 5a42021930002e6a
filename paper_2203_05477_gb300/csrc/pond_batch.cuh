// pond_batch.cuh -- many independent 1D shock tubes (D1Q4) advanced in one persistent launch.
//
// Each CTA owns one tube for the whole run and loops over the time steps itself: the
// tube's time step comes from its own CFL maximum (a CTA reduction), so tubes never wait
// on one another and no inter-CTA synchronization exists.  Per step every warp streams its
// own chunks of 30 cells (chunk w, w + warps, ...): the chunk and a halo of two cells on
// each side are staged in the warp's part of shared memory (phi-bar-plus, Eq. Fbarplus),
// each lane solves one of the chunk's 31 faces (Sec. III.B.3) into shared memory, and the
// lane that staged a cell of the chunk then updates it from the state it still holds
// (Eqs. fluxEq, FinalUpdateDUGKS, with the re-expression in the new co-moving frame).  Warps meet only at the end of a step (the CFL reduction), so a
// warp whose faces need more corrector passes holds up no other.  The state and the face
// predictors are read from one of two buffers and written to the other, so a chunk never
// sees a neighbouring chunk's new values.  Face populations never reach global memory; per
// cell and step the traffic is the state read and written once and the face predictor
// read and written once.
//
// Frames.  The FP64 kernel holds each frame as doubles.  The FP32 kernel holds a cell frame
// (u, T) as a float-float pair and the face predictor as plain floats, so its inner loops
// issue no FP64 instruction: a face frame and the cells it reads are handled as FP32
// offsets from one reference velocity per chunk.
#pragma once

#include "pond_kernels.cuh"

namespace pond {

constexpr int kTubeThreads = 256;  // CTA size of the per-tube set-up and read-back kernels

template <typename R>
struct TubeParams {
    int n_tubes;
    const long long *cell_off;    // first cell of tube k in the concatenated arrays
    const long long *face_off;    // first face of tube k (a tube of L cells has L + 1 faces)
    const int *len;
    const int *order;             // CTA b processes tube order[b] (longest first)
    const double *Cv;            // per tube: 1/(gamma - 1)
    const double *dx;            // per tube
    using CellW = typename FrameWords<R>::word;
    using FaceW = typename FrameWords<R>::pred;
    double tau, cfl;
    int limiter;
    double tol;
    int max_iter, fixed_iters;
    long long ncell, nface;
    R *sf[2];                     // [3][ncell] rho, a2, a3  (two buffers)
    R *sg[2];                     // [3][ncell] b0, b1, b2
    CellW *sfr[2];                // [2][ncell] u, T
    FaceW *fu[2], *fT[2];         // face predictors [nface] (two buffers, paired with the state's)
    double *t, *dt;               // per tube
    double *totals;               // per tube [4]: rho, rho u, 0, rho E summed times dx
    int *status;                  // per tube: 0 running, 1 stopped after a non-physical state
    long long *steps_done;        // per tube: steps taken
    Diag *diag;
};

template <typename R>
__device__ __forceinline__ void tube_stage(const TubeParams<R> &P, int cur, long long c, R Cvh, R cp, R ce,
                                           typename FrameWords<R>::word uref, StagedCell<1, R> &o)
{
    const long long n = P.ncell;
    const R rho = P.sf[cur][c];
    o.A[0] = cp * rho + ce * rho;
    o.A[1] = R(0);
    o.A[2] = cp * P.sf[cur][n + c];
    o.A[3] = cp * P.sf[cur][2 * n + c];
    const R T = fr_lead(P.sfr[cur][n + c]);
    o.B[0] = cp * P.sg[cur][c] + ce * Cvh * rho * T;
    o.B[1] = cp * P.sg[cur][n + c];
    o.B[2] = cp * P.sg[cur][2 * n + c];
    o.du[0] = R(fr_rel(P.sfr[cur][c], uref));
    o.T = T;
}

// volatile reads of a parked value (the compiler may not forward the stored registers)
template <typename R>
__device__ __forceinline__ R vload(const R *p) { return *reinterpret_cast<const volatile R *>(p); }
__device__ __forceinline__ double vload_word(const double *p) { return vload(p); }
__device__ __forceinline__ ffloat vload_word(const ffloat *p)
{
    const volatile float *q = reinterpret_cast<const volatile float *>(p);
    return ffloat{q[0], q[1]};
}

// per-step constants of one tube (Eqs. FinalUpdateDUGKS, Fbarplus, FluxTransf), formed in
// FP64 by one thread and kept in the working precision
template <typename R>
struct TubeStep {
    double dt;
    R cp, ce, wb, we, ca, cb, h_dx, dt_dx, inv_dx;
};

// THREADS threads per tube (THREADS / 32 warps, each streaming its own chunks of kTubeChunk
// cells), MINB CTAs per SM for the register budget; the autotuner picks the variant
constexpr int kTubeChunk = 30;  // cells per warp chunk: 31 faces and 34 staged cells

template <typename R, int THREADS, int MINB>
__global__ void __launch_bounds__(THREADS, MINB)
tube_kernel(const TubeParams<R> P, int steps, int cur0)
{
    constexpr int NW = THREADS / 32;
    constexpr int kStage = kTubeChunk + 4;
    using CellW = typename FrameWords<R>::word;
    __shared__ StagedCell<1, R> tile[NW][kStage];
    __shared__ R faceF[NW][kTubeChunk + 1][4];
    __shared__ R faceG[NW][kTubeChunk + 1][3];
    __shared__ R faceU[NW][kTubeChunk + 1], faceT[NW][kTubeChunk + 1];  // face frame: velocity relative to the chunk reference, T
    __shared__ TubeStep<R> ks;
    // the raw state of the cell each lane stages and later updates, parked here across the
    // face solves (read back with volatile loads) instead of held in registers
    __shared__ R raw[NW][6][32];
    __shared__ CellW raww[NW][2][32];
    __shared__ R red[NW];
    __shared__ int tube_bad;
    __shared__ int next_chunk;   // the next chunk of the step that no warp has taken yet
    // FP32: per-thread scratch of the face solve (the last valid pass's frames), thread-minor
    __shared__ float4 kept[sizeof(R) == 4 ? 2 * THREADS : 1];

    const int tube = P.order[blockIdx.x];
    if (P.status[tube] != 0) return;  // stopped earlier: its state is not advanced any more
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) tube_bad = 0;
    const long long c_off = P.cell_off[tube], f_off = P.face_off[tube];
    const int L = P.len[tube];
    const double Cv = P.Cv[tube], dx = P.dx[tube];
    const double tau = P.tau;
    const R CvR = R(Cv), tolR = R(P.tol);
    // per-thread counts (32-bit: a thread's counts over a call stay far below 2^32 / 32)
    unsigned int my_iters = 0, my_faces = 0, my_nonconv = 0, my_fallbacks = 0, my_nonphys = 0;
    StagedCell<1, R> *wt = tile[warp];

    for (int step = 0; step < steps; ++step) {
        const int cur = (cur0 + step) & 1, nxt = cur ^ 1;
        if (threadIdx.x < 32) {
            // the nine quotients side by side, one per lane of warp 0 (one FP64 division
            // instead of nine in a row on the step's critical path)
            const double dt = P.dt[tube], h = 0.5 * dt;
            double num = 1.0, den = dx;   // lane 8 (and idle lanes): 1/dx
            if (lane == 0) { num = 2.0 * tau - dt; den = 2.0 * tau + dt; }
            if (lane == 1) { num = 2.0 * dt; den = 2.0 * tau + dt; }
            if (lane == 2) { num = 2.0 * tau - h; den = 2.0 * tau + dt; }
            if (lane == 3) { num = 3.0 * h; den = 2.0 * tau + dt; }
            if (lane == 4) { num = 2.0 * tau; den = 2.0 * tau + h; }
            if (lane == 5) { num = h; den = 2.0 * tau + h; }
            if (lane == 6) { num = h; den = dx; }
            if (lane == 7) { num = dt; den = dx; }
            const R q = R(num / den);
            if (lane == 0) { ks.dt = dt; ks.ca = q; }
            if (lane == 1) ks.cb = q;
            if (lane == 2) ks.cp = q;
            if (lane == 3) ks.ce = q;
            if (lane == 4) ks.wb = q;
            if (lane == 5) ks.we = q;
            if (lane == 6) ks.h_dx = q;
            if (lane == 7) ks.dt_dx = q;
            if (lane == 8) ks.inv_dx = q;
            if (lane == 9) next_chunk = NW;   // chunks 0 .. NW-1 go to warps 0 .. NW-1
        }
        __syncthreads();
        const R cp = ks.cp, ce = ks.ce, ca = ks.ca, cb = ks.cb;
        FaceCfg<R> cfg;
        cfg.h_dn = ks.h_dx;
        cfg.h_dt = R(0);
        cfg.Cv = CvR;
        cfg.tol = tolR;
        cfg.wb = ks.wb;
        cfg.we = ks.we;
        cfg.limiter = P.limiter;
        cfg.max_iter = P.max_iter;
        cfg.fixed_iters = P.fixed_iters;
        const typename TubeParams<R>::FaceW *fu_in = P.fu[cur], *fT_in = P.fT[cur];
        typename TubeParams<R>::FaceW *fu_out = P.fu[nxt], *fT_out = P.fT[nxt];
        R rate = R(0);
        const long long n = P.ncell;
        const R Cvh = CvR - R(0.5);
        // chunks are dealt dynamically: a warp that finishes one takes the next free one, so
        // a warp held up by a chunk whose faces need many corrector passes does fewer chunks
        // (the state and predictors are double-buffered, so the order does not matter)
        for (int ci = warp; ci * kTubeChunk < L;) {
            const int c0 = ci * kTubeChunk;
            const int nc = min(kTubeChunk, L - c0);
            // reference velocity of the chunk: its first cell's frame velocity
            const CellW utile = P.sfr[cur][c_off + c0];
            // lane l stages cell c0 - 2 + l (zero-gradient ends) and keeps its state for the
            // update below; lanes 0 and 1 also stage the right halo c0 + 30, c0 + 31
            const long long c = c_off + min(max(c0 - 2 + lane, 0), L - 1);
            const R rho = P.sf[cur][c], a2 = P.sf[cur][n + c], a3 = P.sf[cur][2 * n + c];
            const R b0 = P.sg[cur][c], b1 = P.sg[cur][n + c], b2 = P.sg[cur][2 * n + c];
            const CellW uc = P.sfr[cur][c], Tc = P.sfr[cur][n + c];
            const R Tcr = R(fr_lead(Tc));
            {
                StagedCell<1, R> &o = wt[lane];
                o.A[0] = cp * rho + ce * rho;
                o.A[1] = R(0);
                o.A[2] = cp * a2;
                o.A[3] = cp * a3;
                o.B[0] = cp * b0 + ce * Cvh * rho * Tcr;
                o.B[1] = cp * b1;
                o.B[2] = cp * b2;
                o.du[0] = R(fr_rel(uc, utile));
                o.T = Tcr;
            }
            raw[warp][0][lane] = rho; raw[warp][1][lane] = a2; raw[warp][2][lane] = a3;
            raw[warp][3][lane] = b0; raw[warp][4][lane] = b1; raw[warp][5][lane] = b2;
            raww[warp][0][lane] = uc; raww[warp][1][lane] = Tc;
            if (lane < 2) tube_stage<R>(P, cur, c_off + min(c0 + kTubeChunk + lane, L - 1), Cvh, cp, ce, utile, wt[32 + lane]);
            __syncwarp();
            // faces c0 .. c0+nc: face k lies between cells k-1 and k; the last one is also the
            // next chunk's first face, which that chunk owns (except at the tube's end)
            if (lane <= nc) {
                const int f = lane;
                const long long k = c0 + f;
                Stencil<1, R> cells;   // LL, L, R, RR at wt[f .. f+3]
                cells.base = &wt[f + 2];
                cells.sn = 1;
                cells.st = 0;
                const R dref[1] = {R(fr_rel(fu_in[f_off + k], utile))};
                const R uabs[1] = {R(fr_lead(fu_in[f_off + k]))};
                FaceOut<1, R> o;
                solve_face<1, R, false, 0, false, sizeof(R) == 4 ? 1 : 0>(cells, false, dref, uabs, R(fT_in[f_off + k]), cfg, o,
                                                               FaceScratch{kept + (sizeof(R) == 4 ? threadIdx.x : 0), THREADS});
                const bool owned = f < nc || k == L;
                if (owned) {
                    my_iters += o.iters;
                    my_faces += 1;
                    my_fallbacks += o.fallbacks;
                    if (!o.done) ++my_nonconv;
                }
                if (o.have) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) faceF[warp][f][q] = o.F[q];
#pragma unroll
                    for (int q = 0; q < 3; ++q) faceG[warp][f][q] = o.G[q];
                    const R fdu = dref[0] + o.du[0];
                    faceU[warp][f] = fdu;
                    faceT[warp][f] = o.T;
                    if (owned) {
                        fu_out[f_off + k] = fr_face(utile, fdu);
                        fT_out[f_off + k] = o.T;
                    }
                } else {
                    if (owned) ++my_nonphys;
                    tube_bad = 1;
                    const R nan = R(__int_as_float(0x7fc00000));
#pragma unroll
                    for (int q = 0; q < 4; ++q) faceF[warp][f][q] = nan;
#pragma unroll
                    for (int q = 0; q < 3; ++q) faceG[warp][f][q] = nan;
                    faceU[warp][f] = dref[0];
                    faceT[warp][f] = nan;
                    if (owned) {
                        fu_out[f_off + k] = fu_in[f_off + k];
                        fT_out[f_off + k] = nan;
                    }
                }
            }
            __syncwarp();
            // lane l = 2 .. nc+1 updates the cell it staged, c0 + l - 2, between faces l-2 and l-1
            if (lane >= 2 && lane < nc + 2) {
                const int t = lane - 2;
                const R rho = vload(&raw[warp][0][lane]), a2 = vload(&raw[warp][1][lane]), a3 = vload(&raw[warp][2][lane]);
                const R b0 = vload(&raw[warp][3][lane]), b1 = vload(&raw[warp][4][lane]), b2 = vload(&raw[warp][5][lane]);
                const CellW uc = vload_word(&raww[warp][0][lane]), Tc = vload_word(&raww[warp][1][lane]);
                const R Tcr = R(fr_lead(Tc));
                const long long c = c_off + min(max(c0 - 2 + lane, 0), L - 1);
                const R duc = wt[lane].du[0];
                const R invTc = w_rcp<R>(Tcr), rsqTc = w_sqrt<R>(invTc), sqTc = Tcr * rsqTc;
                R H[4], G[3];
                H[0] = ca * rho + cb * rho;
                H[1] = R(0);
                H[2] = ca * a2;
                H[3] = ca * a3;
                G[0] = ca * b0 + cb * Cvh * rho * Tcr;
                G[1] = ca * b1;
                G[2] = ca * b2;
                const R sx = ks.dt_dx;
                const R ucr = R(fr_lead(uc));
#pragma unroll
                for (int side = 0; side < 2; ++side) {
                    const int f = t + side;
                    const R dv[1] = {faceU[warp][f] - duc};
                    add_face_flux<1, R>(faceF[warp][f], faceG[warp][f], dv, faceT[warp][f], Tcr, invTc, rsqTc, 0,
                                        side ? sx : -sx, sqTc, ucr, H, G);
                }
                R Ho[4], Go[3], du[1], dT;
                bool ok = cell_finish<1, R>(H, G, invTc, sqTc, CvR, Ho, Go, du, dT);
                const CellW un = fr_add(uc, du[0]);
                const CellW Tn = fr_add(Tc, Tcr * dT);
                const R unr = R(fr_lead(un)), Tnr = R(fr_lead(Tn));
                ok = ok && Tnr > R(0) && isfinite(Tnr);
                if (!ok) {
                    ++my_nonphys;
                    tube_bad = 1;
                    atomicCAS((unsigned long long *)&P.diag->first_bad, (unsigned long long)-1ll, (unsigned long long)c);
                }
                P.sf[nxt][c] = Ho[0];
                P.sf[nxt][n + c] = Ho[2];
                P.sf[nxt][2 * n + c] = Ho[3];
                P.sg[nxt][c] = Go[0];
                P.sg[nxt][n + c] = Go[1];
                P.sg[nxt][2 * n + c] = Go[2];
                P.sfr[nxt][c] = un;
                P.sfr[nxt][n + c] = Tn;
                if (ok) {
                    if constexpr (sizeof(R) == 8) rate = fmax(rate, (fabs(unr) + sqrt(Tnr) * kCHi) / dx);
                    else rate = fmaxf(rate, (fabsf(unr) + sqrtf(Tnr) * float(kCHi)) * ks.inv_dx);
                }
            }
            __syncwarp();   // the chunk's shared records are read before the next chunk restages them
            int nxt_c = 0;
            if (lane == 0) nxt_c = atomicAdd(&next_chunk, 1);
            ci = __shfl_sync(0xffffffffu, nxt_c, 0);
        }
        // the tube's next time step from its CFL maximum (Sec. IV)
        R r = rate;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r = max(r, __shfl_down_sync(0xffffffffu, r, o));
        if (lane == 0) red[warp] = r;
        __syncthreads();
        if (threadIdx.x == 0) {
            R rm = R(0);
            for (int w = 0; w < NW; ++w) rm = max(rm, red[w]);
            P.t[tube] += ks.dt;
            P.dt[tube] = P.cfl / double(rm);
            P.steps_done[tube] += 1;
            if (tube_bad) P.status[tube] = 1;
        }
        __syncthreads();
        if (tube_bad) break;  // a non-physical tube stops; pond_sync reports it
    }
    // warp-aggregated diagnostics
    my_iters = warp_sum_count(my_iters);
    my_faces = warp_sum_count(my_faces);
    my_nonconv = warp_sum_count(my_nonconv);
    my_fallbacks = warp_sum_count(my_fallbacks);
    my_nonphys = warp_sum_count(my_nonphys);
    if (lane == 0) {
        using U = unsigned long long;
        if (my_faces) { atomicAdd(&P.diag->face_iters, U(my_iters)); atomicAdd(&P.diag->face_solves, U(my_faces)); }
        if (my_nonconv) { atomicAdd(&P.diag->nonconv, U(my_nonconv)); atomicOr(&P.diag->flags, FLAG_NOT_CONVERGED); }
        if (my_fallbacks) atomicAdd(&P.diag->fallbacks, U(my_fallbacks));
        if (my_nonphys) { atomicAdd(&P.diag->nonphys, U(my_nonphys)); atomicOr(&P.diag->flags, FLAG_NONPHYSICAL); }
    }
}

// initial condition of every tube: co-moving equilibria (Eqs. feqPond, geqPond), the face
// predictors (pooled moments of the two adjacent cells, zero-gradient ends), t = 0 and the
// first time step
template <typename R>
__global__ void __launch_bounds__(kTubeThreads)
tube_init_kernel(const TubeParams<R> P, int cur, const double *rho, const double *ux, const double *p)
{
    __shared__ double red[kTubeThreads / 32];
    __shared__ int any_bad;
    const int tube = blockIdx.x;
    const long long c_off = P.cell_off[tube], f_off = P.face_off[tube];
    const int L = P.len[tube];
    const double Cv = P.Cv[tube], dx = P.dx[tube];
    const long long n = P.ncell;
    double rate = 0.0;
    unsigned long long bad = 0;
    if (threadIdx.x == 0) any_bad = 0;
    __syncthreads();
    for (int k = threadIdx.x; k < L; k += blockDim.x) {
        const long long c = c_off + k;
        const double r = rho[c], T = p[c] / r, u = ux[c];
        P.sf[cur][c] = R(r);
        P.sf[cur][n + c] = R(0);
        P.sf[cur][2 * n + c] = R(0);
        P.sg[cur][c] = R((Cv - 0.5) * r * T);
        P.sg[cur][n + c] = R(0);
        P.sg[cur][2 * n + c] = R(0);
        fr_store(P.sfr[cur][c], u);
        fr_store(P.sfr[cur][n + c], T);
        if (r > 0.0 && T > 0.0 && isfinite(r) && isfinite(T)) {
            rate = fmax(rate, (fabs(u) + sqrt(T) * kCHi) / dx);
        } else {
            ++bad;
            atomicCAS((unsigned long long *)&P.diag->first_bad, (unsigned long long)-1ll, (unsigned long long)c);
        }
    }
    for (int k = threadIdx.x; k <= L; k += blockDim.x) {
        const long long a = c_off + max(k - 1, 0), b = c_off + min(k, L - 1);
        const double ra = rho[a], rb = rho[b], ua = ux[a], ub = ux[b];
        const double Ea = p[a] * Cv + 0.5 * ra * ua * ua, Eb = p[b] * Cv + 0.5 * rb * ub * ub;
        const double r = 0.5 * (ra + rb), m = 0.5 * (ra * ua + rb * ub), E = 0.5 * (Ea + Eb);
        fr_store(P.fu[cur][f_off + k], m / r);
        fr_store(P.fT[cur][f_off + k], (E - 0.5 * m * m / r) / (Cv * r));
    }
    if (bad) { atomicAdd(&P.diag->nonphys, bad); atomicOr(&P.diag->flags, FLAG_NONPHYSICAL); any_bad = 1; }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rate = fmax(rate, __shfl_down_sync(0xffffffffu, rate, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = rate;
    __syncthreads();
    if (threadIdx.x == 0) {
        double rm = 0.0;
        for (int w = 0; w < kTubeThreads / 32; ++w) rm = fmax(rm, red[w]);
        P.t[tube] = 0.0;
        P.dt[tube] = P.cfl / rm;
        P.steps_done[tube] = 0;
        P.status[tube] = any_bad;
    }
}

// conserved fields of every tube (lab frame, FP64) and the per-tube sums times dx
template <typename R>
__global__ void __launch_bounds__(kTubeThreads)
tube_conserved_kernel(const TubeParams<R> P, int cur, double *rho, double *mx, double *E)
{
    __shared__ double red[3][kTubeThreads / 32];
    const int tube = blockIdx.x;
    const long long c_off = P.cell_off[tube];
    const int L = P.len[tube];
    const double Cv = P.Cv[tube], dx = P.dx[tube];
    const long long n = P.ncell;
    double s[3] = {0, 0, 0};
    for (int k = threadIdx.x; k < L; k += blockDim.x) {
        const long long c = c_off + k;
        const double r = double(P.sf[cur][c]), u = fr_value(P.sfr[cur][c]), T = fr_value(P.sfr[cur][n + c]);
        const double v[3] = {r, r * u, r * (Cv * T + 0.5 * u * u)};
        if (rho) rho[c] = v[0];
        if (mx) mx[c] = v[1];
        if (E) E[c] = v[2];
#pragma unroll
        for (int q = 0; q < 3; ++q) s[q] += v[q];
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s[q] += __shfl_down_sync(0xffffffffu, s[q], o);
        if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = s[q];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot[3] = {0, 0, 0};
        for (int w = 0; w < kTubeThreads / 32; ++w)
            for (int q = 0; q < 3; ++q) tot[q] += red[q][w];
        P.totals[4 * tube + 0] = tot[0] * dx;
        P.totals[4 * tube + 1] = tot[1] * dx;
        P.totals[4 * tube + 2] = 0.0;
        P.totals[4 * tube + 3] = tot[2] * dx;
    }
}

// stored state as full coefficient arrays [cells][4], [cells][3] and frames [cells][2]
template <typename R>
__global__ void tube_export_kernel(const TubeParams<R> P, int cur, double *cf, double *cg, double *fr)
{
    const long long n = P.ncell;
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    if (cf) {
        cf[4 * c] = double(P.sf[cur][c]);
        cf[4 * c + 1] = 0.0;
        cf[4 * c + 2] = double(P.sf[cur][n + c]);
        cf[4 * c + 3] = double(P.sf[cur][2 * n + c]);
    }
    if (cg)
        for (int q = 0; q < 3; ++q) cg[3 * c + q] = double(P.sg[cur][q * n + c]);
    if (fr) {
        fr[2 * c] = fr_value(P.sfr[cur][c]);
        fr[2 * c + 1] = fr_value(P.sfr[cur][n + c]);
    }
}

}  // namespace pond
