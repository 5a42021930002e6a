// pond_sl.cuh -- the semi-Lagrangian realization of Sec. III.A on D1Q4 grids (D2Q16: pond_sl2.cuh).
//
// One thread per node.  A CTA stages its TX nodes and a halo of two on each side (the raw
// populations in each node's own frame, as Hermite coefficients).  Each thread then runs
// the node's predictor-corrector: every pass re-expresses the five stencil nodes in the
// pass's frame (the regularized transformation of Sec. II.C, as 1D lower-triangular maps),
// advects each of the four populations from its departure point x - v_i dt by the limited
// 4-point Lagrange interpolation, and takes the moments that define the next frame.  The
// converged populations are projected into the frame of their own moments, relaxed by the
// BGK collision with beta = dt / (2 tau + dt), and written to the other state buffer.  The
// CFL reduction of the new frames sets the next time step, as in the cell kernel.
#pragma once

#include "pond_kernels.cuh"

namespace pond {

// limited 4-point Lagrange interpolation at th in [0, 1] of values at offsets -1, 0, 1, 2:
// the cubic interpolant, or the linear one when the cubic leaves the bracket [v1, v2]
template <typename R>
__device__ __forceinline__ R sl_interp(R v0, R v1, R v2, R v3, R th)
{
    const R tm = th - R(1), t2 = th - R(2), tp = th + R(1);
    const R w0 = -th * tm * t2 * R(1.0 / 6.0);
    const R w1 = tp * tm * t2 * R(0.5);
    const R w2 = -tp * th * t2 * R(0.5);
    const R w3 = tp * th * tm * R(1.0 / 6.0);
    R p = w0 * v0 + w1 * v1 + w2 * v2 + w3 * v3;
    const R lo = min(v1, v2), hi = max(v1, v2);
    if (p < lo || p > hi) p = v1 + th * (v2 - v1);
    return p;
}

// warp-aggregated node diagnostics (passes, non-converged, restarts, non-physical), then
// the CFL reduction that sets the next step; every thread of the block calls it
template <typename R>
__device__ __forceinline__ void sl_diag_and_advance(Diag *diag, Clock *clock, bool active, unsigned long long my_iters,
                                                    unsigned long long my_nonconv, unsigned long long my_fallbacks,
                                                    unsigned long long my_nonphys, double rate)
{
    unsigned long long n_act = active ? 1ull : 0ull;
    my_iters = warp_sum_count(my_iters);
    my_nonconv = warp_sum_count(my_nonconv);
    my_fallbacks = warp_sum_count(my_fallbacks);
    my_nonphys = warp_sum_count(my_nonphys);
    n_act = warp_sum_count(n_act);
    if ((threadIdx.x & 31) == 0 && n_act) {
        atomicAdd(&diag->face_iters, my_iters);
        atomicAdd(&diag->face_solves, n_act);
        if (my_nonconv) { atomicAdd(&diag->nonconv, my_nonconv); atomicOr(&diag->flags, FLAG_NOT_CONVERGED); }
        if (my_fallbacks) atomicAdd(&diag->fallbacks, my_fallbacks);
        if (my_nonphys) { atomicAdd(&diag->nonphys, my_nonphys); atomicOr(&diag->flags, FLAG_NONPHYSICAL); }
    }
    reduce_rate_and_advance(clock, rate, true);
}

// a staged D1Q4 node without padding: nine words, so that neighbouring threads' scalar
// loads (this kernel reads fields one at a time) fall in distinct banks
template <typename R>
struct SlCell1 {
    R A[4];
    R B[3];
    R du[1];
    R T;
};

template <typename R, int TX>
__global__ void __launch_bounds__(TX, sizeof(R) == 4 ? 8 : 1)   // FP32: 64 registers, 8 CTAs per SM
sl_kernel(const Params<1, R> P)
{
    using W = typename FrameWords<R>::word;
    constexpr int BX = TX + 4;
    __shared__ SlCell1<R> tile[BX];
    __shared__ W utile[1];
    const Clock &K = *P.clock;
    if (!(K.dt > 0.0)) return;
    const StepC<R> &KC = step_c<R>(K);
    const long long n = P.ncell();
    const long long i0 = (long long)blockIdx.x * TX;
    if (threadIdx.x == 0) cell_velocity<1, R>(P, i0, 0, utile);
    __syncthreads();
    for (int t = threadIdx.x; t < BX; t += blockDim.x) {
        StagedCell<1, R> c;
        load_cell_bar_plus<1, R>(P, i0 - 2 + t, 0, R(1), R(0), utile, c);
        SlCell1<R> &o = tile[t];
#pragma unroll
        for (int k = 0; k < 4; ++k) o.A[k] = c.A[k];
#pragma unroll
        for (int k = 0; k < 3; ++k) o.B[k] = c.B[k];
        o.du[0] = c.du[0];
        o.T = c.T;
    }
    __syncthreads();

    const long long i = i0 + threadIdx.x;
    double rate = 0.0;
    unsigned long long my_iters = 0, my_nonconv = 0, my_fallbacks = 0, my_nonphys = 0;
    const bool active = i < P.nx;
    if (active) {
        const SlCell1<R> *cells[5];
#pragma unroll
        for (int s = 0; s < 5; ++s) cells[s] = &tile[threadIdx.x + s];
        const R dt_dx = KC.dt_dx;
        const R Cv = P.Cv_r, tolR = P.tol_r;
        const R uref = R(fr_lead(utile[0]));
        const NodeTab<R> &tab = node_tab<R>();
        R dl = cells[2]->du[0], Tl = cells[2]->T;   // predictor: the node's own frame
        R keep_dl = R(0), keep_T = R(0), out_du = R(0), out_T = R(0), out_rho = R(0);
        R Phi[4], Psi[3];
        bool have = false, done = false, restarted = false, last_valid = false;
        int iters = 0, fallbacks = 0;
        auto pass = [&](R dlp, R Tlp) {
            const R invTl = R(1) / Tlp, rsqTl = sqrt(invTl), sqTl = Tlp * rsqTl;
            R F[5][4], G[5][3];
#pragma unroll
            for (int s = 0; s < 5; ++s) {
                const R sc = sqrt(cells[s]->T * invTl), e = (cells[s]->T - Tlp) * invTl;
                Map1<R> X(sc, e, (cells[s]->du[0] - dlp) * rsqTl);
                shift_scale_1d<3, R, true>(cells[s]->A, X, F[s]);   // staged f: zero first order
                shift_scale_1d<2, R>(cells[s]->B, X, G[s]);
            }
            // The node's own coefficients enter the moments directly and only the differences
            // of the neighbours from the node are interpolated: the same result (the
            // interpolation and its limiter commute with adding a constant, and the D1Q4
            // quadrature maps coefficients to populations and back exactly), but a uniform
            // state is reproduced without the round-off of the quadrature, so FP32 runs do not
            // drift in mass where nothing moves.
#pragma unroll
            for (int k = 0; k < 4; ++k) Phi[k] = F[2][k];
#pragma unroll
            for (int k = 0; k < 3; ++k) Psi[k] = G[2][k];
#pragma unroll
            for (int s = 0; s < 5; ++s) {
                if (s == 2) continue;
#pragma unroll
                for (int k = 0; k < 4; ++k) F[s][k] -= F[2][k];
#pragma unroll
                for (int k = 0; k < 3; ++k) G[s][k] -= G[2][k];
            }
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const R d = (sqTl * tab.c[m] + uref + dlp) * dt_dx;   // departure distance in cells
                const bool right = d > R(0);                          // departure point left of the node
                const R th = right ? R(1) - d : -d;
                // population m (unweighted) of the five stencil nodes, minus the node's own
                R fv[5], gv[5];
#pragma unroll
                for (int s = 0; s < 5; ++s) {
                    if (s == 2) {
                        fv[s] = gv[s] = R(0);
                        continue;
                    }
                    fv[s] = F[s][0] * tab.hen[m][0] + F[s][1] * tab.hen[m][1] + F[s][2] * tab.hen[m][2] +
                            F[s][3] * tab.hen[m][3];
                    gv[s] = G[s][0] * tab.hen[m][0] + G[s][1] * tab.hen[m][1] + G[s][2] * tab.hen[m][2];
                }
                const R fb = right ? sl_interp<R>(fv[0], fv[1], fv[2], fv[3], th) : sl_interp<R>(fv[1], fv[2], fv[3], fv[4], th);
                const R gb = right ? sl_interp<R>(gv[0], gv[1], gv[2], gv[3], th) : sl_interp<R>(gv[1], gv[2], gv[3], gv[4], th);
#pragma unroll
                for (int a = 0; a < 4; ++a) Phi[a] += tab.whe[m][a] * fb;
#pragma unroll
                for (int a = 0; a < 3; ++a) Psi[a] += tab.whe[m][a] * gb;
            }
        };
        for (int k = 0; k < P.max_iter && !done; ++k) {
            pass(dl, Tl);
            R rho1, du[1], T1;
            const bool ok = pass_frame<1, R>(Phi, Psi, Tl, Cv, rho1, du, T1);
            iters = k + 1;
            if (!ok) {
                ++fallbacks;
                last_valid = false;
                if (!restarted) {
                    // restart once from the frame of the pooled conserved moments of the stencil
                    restarted = true;
                    R r = R(0), mo = R(0), e = R(0);
#pragma unroll
                    for (int s = 0; s < 5; ++s) {
                        const R rc = cells[s]->A[0], us = cells[s]->du[0];
                        r += rc;
                        mo += rc * us;
                        e += rc * (Cv * cells[s]->T + R(0.5) * us * us);
                    }
                    r *= R(0.2); mo *= R(0.2); e *= R(0.2);
                    dl = mo / r;
                    Tl = (e - R(0.5) * mo * mo / r) / (Cv * r);
                    continue;
                }
                break;
            }
            have = true;
            last_valid = true;
            keep_dl = dl; keep_T = Tl; out_du = du[0]; out_T = T1; out_rho = rho1;
            if (P.fixed_iters > 0) done = iters >= P.fixed_iters;
            else done = fabs(T1 - Tl) <= tolR * Tl && fabs(du[0]) <= tolR * sqrt(Tl);
            dl += du[0];
            Tl = T1;
        }
        my_iters = iters;
        my_nonconv = done ? 0 : 1;
        my_fallbacks = fallbacks;
        W un = utile[0], Tn;
        R A[4], B[3];
        bool ok = have;
        if (have) {
            if (!last_valid) pass(keep_dl, keep_T);
            // the pre-collision populations in the frame of their own moments, then BGK
            const R invT = R(1) / out_T;
            Map1<R> X(sqrt(keep_T * invT), (keep_T - out_T) * invT, -out_du * sqrt(invT));
            shift_scale_1d<3, R>(Phi, X, A);
            shift_scale_1d<2, R>(Psi, X, B);
            const R twob = KC.cb;  // 2 beta = 2 dt / (2 tau + dt)
            const R keep = R(1) - twob;
            A[0] = keep * A[0] + twob * out_rho;
            A[2] = keep * A[2];
            A[3] = keep * A[3];
            B[0] = keep * B[0] + twob * P.Cvh_r * out_rho * out_T;
            B[1] = keep * B[1];
            B[2] = keep * B[2];
            un = fr_add(utile[0], keep_dl + out_du);
            Tn = fr_word(out_T);
            ok = out_rho > R(0) && out_T > R(0) && isfinite(out_rho) && isfinite(out_T);
        }
        if (!ok) {
            ++my_nonphys;
            const R nan = R(__int_as_float(0x7fc00000));
            A[0] = A[2] = A[3] = B[0] = B[1] = B[2] = nan;
            Tn = fr_word(nan);
            atomicCAS((unsigned long long *)&P.diag->first_bad, (unsigned long long)-1ll, (unsigned long long)i);
        }
        // the new state goes to the other buffer (held in the face planes, plane stride n)
        P.xf[i] = A[0];
        P.xf[n + i] = A[2];
        P.xf[2 * n + i] = A[3];
        P.xg[i] = B[0];
        P.xg[n + i] = B[1];
        P.xg[2 * n + i] = B[2];
        P.xfr[i] = un;
        P.xfr[n + i] = Tn;
        if (ok) {
            const R unr = R(fr_lead(un));
            rate = cell_rate<R>(&unr, out_T, KC.inv_dx, KC.inv_dx, 1);
        }
    }
    sl_diag_and_advance<R>(P.diag, P.clock, active, my_iters, my_nonconv, my_fallbacks, my_nonphys, rate);
}

}  // namespace pond
