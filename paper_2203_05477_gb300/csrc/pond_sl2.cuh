// pond_sl2.cuh -- the semi-Lagrangian realization of Sec. III.A on D2Q16 grids.
//
// One thread per node; a CTA stages its TX x TY nodes and a halo of two (raw populations in
// each node's frame, as Hermite coefficients).  A corrector pass in frame lambda takes, for
// each of the four x-nodes m of the lattice, the 5 x 4 stencil nodes that the departure
// points of the populations (m, n) can reach (the x base depends only on m), re-expresses
// each in lambda (the regularized transformation, Sec. II.C), collapses it along x at c_m
// and keeps the 7 collapsed coefficients in a per-thread shared-memory scratch.  Each
// population (m, n) then evaluates its 4 x 4 box from the scratch (the y base depends only
// on n) and interpolates it with the limited bicubic of the reading in Sec. III.A.  As in
// the D1Q4 kernel, the node's own coefficients enter the moments directly and only the
// differences of the neighbours from the node are interpolated (the same result in exact
// arithmetic).  The converged populations are projected into the frame of their own
// moments, relaxed by BGK, and written to the other state buffer.
#pragma once

#include "pond_sl.cuh"

namespace pond {

// limited bicubic at (thx, thy) in [0, 1]^2 of v[row y][column x] at offsets -1..2: the
// tensor-product Lagrange interpolant, or the bilinear one of the 2 x 2 nearest values when
// it leaves their range
template <typename R>
__device__ __forceinline__ R sl_interp2(const R (&v)[4][4], R thx, R thy)
{
    auto weights = [](R th, R *w) {
        const R tm = th - R(1), t2 = th - R(2), tp = th + R(1);
        w[0] = -th * tm * t2 * R(1.0 / 6.0);
        w[1] = tp * tm * t2 * R(0.5);
        w[2] = -tp * th * t2 * R(0.5);
        w[3] = tp * th * tm * R(1.0 / 6.0);
    };
    R wx[4], wy[4];
    weights(thx, wx);
    weights(thy, wy);
    R p = R(0);
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int m = 0; m < 4; ++m) p += wy[r] * wx[m] * v[r][m];
    const R lo = min(min(v[1][1], v[1][2]), min(v[2][1], v[2][2]));
    const R hi = max(max(v[1][1], v[1][2]), max(v[2][1], v[2][2]));
    if (p < lo || p > hi)
        p = (R(1) - thy) * ((R(1) - thx) * v[1][1] + thx * v[1][2]) + thy * ((R(1) - thx) * v[2][1] + thx * v[2][2]);
    return p;
}

template <typename R>
__device__ __forceinline__ void sl2_transform(const StagedCell<2, R> *cp, const R *dl, R Tl, R invTl, R rsqTl, R *F, R *G)
{
    const StagedCell<2, R> c = fetch<2, R>(cp);   // 16-byte loads of the staged record
    Map1<R> X(R(1), R(0), R(0)), Y(R(1), R(0), R(0));
    cell_maps<2, R>(c.T, c.du, Tl, invTl, rsqTl, dl, X, Y);
    shift_scale<2, 3, R, true>(c.A, X, Y, F);   // staged f: zero first order
    shift_scale<2, 2, R>(c.B, X, Y, G);
}

// per-thread scratch: [row 0..4][column 0..3][7 collapsed coefficients], thread-minor
template <int NT>
__device__ __forceinline__ int sl2_scr(int row, int col, int q) { return ((row * 4 + col) * 7 + q) * NT; }

template <typename R, int TX, int TY>
__global__ void __launch_bounds__(TX * TY)
sl2_kernel(const Params<2, R> P)
{
    using W = typename FrameWords<R>::word;
    constexpr int NT = TX * TY, BX = TX + 4, BY = TY + 4;
    constexpr int NFC = NCoef<2, 3>::value, NGC = NCoef<2, 2>::value;
    __shared__ StagedCell<2, R> tile[BX * BY];
    __shared__ W utile[2];
    extern __shared__ __align__(16) unsigned char sl2_dyn[];
    R *scr = reinterpret_cast<R *>(sl2_dyn) + threadIdx.x;
    const Clock &K = *P.clock;
    if (!(K.dt > 0.0)) return;
    const StepC<R> &KC = step_c<R>(K);
    const long long n = P.ncell();
    const long long i0 = (long long)blockIdx.x * TX, j0 = (long long)blockIdx.y * TY;
    if (threadIdx.x == 0) cell_velocity<2, R>(P, i0, j0, utile);
    __syncthreads();
    for (int t = threadIdx.x; t < BX * BY; t += blockDim.x)
        load_cell_bar_plus<2, R>(P, i0 - 2 + t % BX, j0 - 2 + t / BX, R(1), R(0), utile, tile[t]);
    __syncthreads();

    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const long long i = i0 + tx, j = j0 + ty, c = j * P.nx + i;
    double rate = 0.0;
    unsigned long long my_iters = 0, my_nonconv = 0, my_fallbacks = 0, my_nonphys = 0;
    const bool active = i < P.nx && j < P.ny;
    if (active) {
        auto cell = [&](int r, int col) -> const StagedCell<2, R> * { return &tile[(ty + r) * BX + tx + col]; };
        const R dt_dx = KC.dt_dx, dt_dy = KC.dt_dy;
        const R Cv = P.Cv_r, tolR = P.tol_r;
        const R uref[2] = {R(fr_lead(utile[0])), R(fr_lead(utile[1]))};
        const NodeTab<R> &tab = node_tab<R>();
        R dl[2] = {cell(2, 2)->du[0], cell(2, 2)->du[1]}, Tl = cell(2, 2)->T;   // the node's own frame
        R keep_dl[2] = {R(0), R(0)}, keep_T = R(0), out_du[2] = {R(0), R(0)}, out_T = R(0), out_rho = R(0);
        R Phi[NFC], Psi[NGC];
        bool have = false, done = false, restarted = false, last_valid = false;
        int iters = 0, fallbacks = 0;
        auto pass = [&](const R *dlp, R Tlp) {
            const R invTl = R(1) / Tlp, rsqTl = sqrt(invTl), sqTl = Tlp * rsqTl;
            R Fc[NFC], Gc[NGC];
            sl2_transform<R>(cell(2, 2), dlp, Tlp, invTl, rsqTl, Fc, Gc);
#pragma unroll
            for (int k = 0; k < NFC; ++k) Phi[k] = Fc[k];
#pragma unroll
            for (int k = 0; k < NGC; ++k) Psi[k] = Gc[k];
#pragma unroll 1
            for (int m = 0; m < 4; ++m) {
                const R dx = (sqTl * tab.c[m] + uref[0] + dlp[0]) * dt_dx;   // departure distance in cells
                const bool rx = dx > R(0);
                const R thx = rx ? R(1) - dx : -dx;
                const int cx0 = rx ? 0 : 1;
                // the node's own coefficients collapsed along x at c_m, to be subtracted
                R Cc[4], Dc[3];
#pragma unroll
                for (int s = 0; s <= 3; ++s) {
                    R acc = R(0);
#pragma unroll
                    for (int r = 0; r + s <= 3; ++r) acc += Fc[hidx(r, s)] * tab.hen[m][r];
                    Cc[s] = acc;
                }
#pragma unroll
                for (int s = 0; s <= 2; ++s) {
                    R acc = R(0);
#pragma unroll
                    for (int r = 0; r + s <= 2; ++r) acc += Gc[hidx(r, s)] * tab.hen[m][r];
                    Dc[s] = acc;
                }
#pragma unroll 1
                for (int row = 0; row < 5; ++row)
#pragma unroll 1
                    for (int k = 0; k < 4; ++k) {
                        R F[NFC], G[NGC];
                        sl2_transform<R>(cell(row, cx0 + k), dlp, Tlp, invTl, rsqTl, F, G);
#pragma unroll
                        for (int s = 0; s <= 3; ++s) {
                            R acc = R(0);
#pragma unroll
                            for (int r = 0; r + s <= 3; ++r) acc += F[hidx(r, s)] * tab.hen[m][r];
                            scr[sl2_scr<NT>(row, k, s)] = acc - Cc[s];
                        }
#pragma unroll
                        for (int s = 0; s <= 2; ++s) {
                            R acc = R(0);
#pragma unroll
                            for (int r = 0; r + s <= 2; ++r) acc += G[hidx(r, s)] * tab.hen[m][r];
                            scr[sl2_scr<NT>(row, k, 4 + s)] = acc - Dc[s];
                        }
                    }
                R S[4] = {R(0), R(0), R(0), R(0)}, SG[3] = {R(0), R(0), R(0)};
#pragma unroll
                for (int nn = 0; nn < 4; ++nn) {
                    const R dy = (sqTl * R(node_c(nn)) + uref[1] + dlp[1]) * dt_dy;
                    const bool ry = dy > R(0);
                    const R thy = ry ? R(1) - dy : -dy;
                    const int ry0 = ry ? 0 : 1;
                    R fv[4][4], gv[4][4];
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) {
                            R f = R(0), g = R(0);
#pragma unroll
                            for (int s = 0; s <= 3; ++s) f += scr[sl2_scr<NT>(ry0 + a, b, s)] * R(hen(s, nn));
#pragma unroll
                            for (int s = 0; s <= 2; ++s) g += scr[sl2_scr<NT>(ry0 + a, b, 4 + s)] * R(hen(s, nn));
                            fv[a][b] = f;
                            gv[a][b] = g;
                        }
                    const R fb = sl_interp2<R>(fv, thx, thy), gb = sl_interp2<R>(gv, thx, thy);
#pragma unroll
                    for (int s = 0; s <= 3; ++s) S[s] += R(node_w(nn) * he(s, nn)) * fb;
#pragma unroll
                    for (int s = 0; s <= 2; ++s) SG[s] += R(node_w(nn) * he(s, nn)) * gb;
                }
#pragma unroll
                for (int r = 0; r <= 3; ++r)
#pragma unroll
                    for (int s = 0; r + s <= 3; ++s) Phi[hidx(r, s)] += tab.whe[m][r] * S[s];
#pragma unroll
                for (int r = 0; r <= 2; ++r)
#pragma unroll
                    for (int s = 0; r + s <= 2; ++s) Psi[hidx(r, s)] += tab.whe[m][r] * SG[s];
            }
        };
        for (int k = 0; k < P.max_iter && !done; ++k) {
            pass(dl, Tl);
            R rho1, du[2], T1;
            const bool ok = pass_frame<2, R>(Phi, Psi, Tl, Cv, rho1, du, T1);
            iters = k + 1;
            if (!ok) {
                ++fallbacks;
                last_valid = false;
                if (!restarted) {
                    // restart once from the frame of the pooled conserved moments of the stencil
                    restarted = true;
                    R r = R(0), mo[2] = {R(0), R(0)}, e = R(0);
#pragma unroll 1
                    for (int q = 0; q < 25; ++q) {
                        const StagedCell<2, R> *sc = cell(q / 5, q % 5);
                        const R rc = sc->A[0];
                        r += rc;
                        mo[0] += rc * sc->du[0];
                        mo[1] += rc * sc->du[1];
                        e += rc * (Cv * sc->T + R(0.5) * (sc->du[0] * sc->du[0] + sc->du[1] * sc->du[1]));
                    }
                    r *= R(1.0 / 25.0); mo[0] *= R(1.0 / 25.0); mo[1] *= R(1.0 / 25.0); e *= R(1.0 / 25.0);
                    dl[0] = mo[0] / r;
                    dl[1] = mo[1] / r;
                    Tl = (e - R(0.5) * (mo[0] * mo[0] + mo[1] * mo[1]) / r) / (Cv * r);
                    continue;
                }
                break;
            }
            have = true;
            last_valid = true;
            keep_dl[0] = dl[0]; keep_dl[1] = dl[1]; keep_T = Tl;
            out_du[0] = du[0]; out_du[1] = du[1]; out_T = T1; out_rho = rho1;
            if (P.fixed_iters > 0) done = iters >= P.fixed_iters;
            else done = fabs(T1 - Tl) <= tolR * Tl && fabs(du[0]) <= tolR * sqrt(Tl) && fabs(du[1]) <= tolR * sqrt(Tl);
            dl[0] += du[0];
            dl[1] += du[1];
            Tl = T1;
        }
        my_iters = iters;
        my_nonconv = done ? 0 : 1;
        my_fallbacks = fallbacks;
        W un[2] = {utile[0], utile[1]}, Tn;
        R A[NFC], B[NGC];
        bool ok = have;
        if (have) {
            if (!last_valid) pass(keep_dl, keep_T);
            // the pre-collision populations in the frame of their own moments, then BGK
            const R invT = R(1) / out_T, sc = sqrt(keep_T * invT), e = (keep_T - out_T) * invT, rs = sqrt(invT);
            Map1<R> X(sc, e, -out_du[0] * rs), Y(sc, e, -out_du[1] * rs);
            shift_scale<2, 3, R>(Phi, X, Y, A);
            shift_scale<2, 2, R>(Psi, X, Y, B);
            const R twob = KC.cb;  // 2 beta = 2 dt / (2 tau + dt)
            const R keep = R(1) - twob;
#pragma unroll
            for (int k = 0; k < NFC; ++k) A[k] = keep * A[k];
#pragma unroll
            for (int k = 0; k < NGC; ++k) B[k] = keep * B[k];
            A[0] += twob * out_rho;
            B[0] += twob * P.Cvh_r * out_rho * out_T;
#pragma unroll
            for (int a = 0; a < 2; ++a) un[a] = fr_add(utile[a], keep_dl[a] + out_du[a]);
            Tn = fr_word(out_T);
            ok = out_rho > R(0) && out_T > R(0) && isfinite(out_rho) && isfinite(out_T);
        }
        if (!ok) {
            ++my_nonphys;
            const R nan = R(__int_as_float(0x7fc00000));
#pragma unroll
            for (int k = 0; k < NFC; ++k) A[k] = nan;
#pragma unroll
            for (int k = 0; k < NGC; ++k) B[k] = nan;
            Tn = fr_word(nan);
            atomicCAS((unsigned long long *)&P.diag->first_bad, (unsigned long long)-1ll, (unsigned long long)c);
        }
        // the new state goes to the other buffer (held in the face planes, plane stride n)
#pragma unroll
        for (int k = 0; k < NFC; ++k) {
            const int pl = fplane<2>(k);
            if (pl >= 0) P.xf[pl * n + c] = A[k];
        }
#pragma unroll
        for (int k = 0; k < NGC; ++k) P.xg[k * n + c] = B[k];
        P.xfr[c] = un[0];
        P.xfr[n + c] = un[1];
        P.xfr[2 * n + c] = Tn;
        if (ok) {
            const R unr[2] = {R(fr_lead(un[0])), R(fr_lead(un[1]))};
            rate = cell_rate<R>(unr, out_T, KC.inv_dx, KC.inv_dy, 2);
        }
    }
    sl_diag_and_advance<R>(P.diag, P.clock, active, my_iters, my_nonconv, my_fallbacks, my_nonphys, rate);
}

}  // namespace pond
