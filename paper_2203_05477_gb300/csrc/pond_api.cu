// pond_api.cu -- host side of the C ABI declared in include/pond.h.
//
// A pond_state owns one device allocation holding the cell planes, the face planes, the
// device clock (time, time step, CFL reduction) and the diagnostics; every step is two
// kernel launches (face corrector, cell update) that read the time step from the device,
// so runs of steps are captured once into a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <type_traits>
#include <new>
#include <vector>

#include "../../include/pond.h"
#include "pond_kernels.cuh"

namespace {

thread_local char g_err[512] = "";

pond_status fail(pond_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

#define CUDA_TRY(call)                                                                          \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) return fail(POND_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

constexpr int kGraphSteps = 32;   // steps per captured graph
constexpr int kReduceBlocks = 1024;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

struct pond_state {
    int D = 1, prec = POND_FP64;
    pond_grid grid{};
    pond_options opts{};
    double gamma = 1.4, tau = 1e-5;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    char *base = nullptr;
    size_t bytes = 0;
    pond::Clock *clock = nullptr;
    pond::Diag *diag = nullptr;
    double *stage = nullptr;      // staging for host transfers and reductions
    size_t stage_doubles = 0;
    alignas(16) unsigned char params[sizeof(pond::Params<2, double>)];
    int64_t launches = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
};

namespace {

template <int D, typename R>
pond::Params<D, R> &params_of(pond_state *s) { return *reinterpret_cast<pond::Params<D, R> *>(s->params); }

void *dev_alloc(pond_state *s, size_t bytes)
{
    if (s->opts.alloc) return s->opts.alloc(bytes, s->opts.alloc_ctx);
    void *p = nullptr;
    return cudaMalloc(&p, bytes) == cudaSuccess ? p : nullptr;
}

void dev_free(pond_state *s, void *p)
{
    if (!p) return;
    if (s->opts.free) s->opts.free(p, s->opts.alloc_ctx);
    else cudaFree(p);
}

template <int D, typename R>
pond_status setup(pond_state *s)
{
    using P_t = pond::Params<D, R>;
    P_t P{};
    const pond_grid &g = s->grid;
    P.nx = g.nx;
    P.ny = D == 2 ? g.ny : 1;
    P.dx = (g.x1 - g.x0) / double(g.nx);
    P.dy = D == 2 ? (g.y1 - g.y0) / double(g.ny) : 1.0;
    for (int k = 0; k < 4; ++k) {
        P.bc[k] = g.bc[k];
        P.lo[k] = g.inflow_lo[k];
        P.hi[k] = g.inflow_hi[k];
        for (int q = 0; q < 4; ++q) P.inflow[k][q] = g.inflow[k][q];
    }
    P.gamma = s->gamma;
    P.Cv = 1.0 / (s->gamma - 1.0);
    P.tau = s->tau;
    P.limiter = s->opts.limiter;
    P.tol = s->opts.tol;
    P.max_iter = s->opts.max_iter;
    P.fixed_iters = s->opts.fixed_iters;
    const long long n = P.ncell(), nxf = P.nxf(), nyf = D == 2 ? P.nyf() : 0;
    constexpr int NFC = P_t::NFC, NGC = P_t::NGC, NFS = P_t::NFS;
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off = align_up(off + b, 256); return o; };
    const size_t o_sf = take(sizeof(R) * NFS * n), o_sg = take(sizeof(R) * NGC * n), o_sfr = take(8 * (D + 1) * n);
    const size_t o_xf = take(sizeof(R) * NFC * nxf), o_xg = take(sizeof(R) * NGC * nxf), o_xfr = take(8 * (D + 1) * nxf);
    size_t o_yf = 0, o_yg = 0, o_yfr = 0;
    if (D == 2) { o_yf = take(sizeof(R) * NFC * nyf); o_yg = take(sizeof(R) * NGC * nyf); o_yfr = take(8 * (D + 1) * nyf); }
    const size_t o_clock = take(sizeof(pond::Clock)), o_diag = take(sizeof(pond::Diag));
    size_t stage = 4 * size_t(n);
    stage = std::max<size_t>(stage, size_t(NFC + NGC + D + 1) * size_t(n));
    stage = std::max<size_t>(stage, size_t(D + 1) * size_t(nxf + nyf));
    stage += size_t(kReduceBlocks) * 8 + 8;
    const size_t o_stage = take(8 * stage);
    s->bytes = off;
    s->base = static_cast<char *>(dev_alloc(s, off));
    if (!s->base) return fail(POND_ERR_OOM, "device allocation of %zu bytes failed", off);
    P.sf = reinterpret_cast<R *>(s->base + o_sf);
    P.sg = reinterpret_cast<R *>(s->base + o_sg);
    P.sfr = reinterpret_cast<double *>(s->base + o_sfr);
    P.xf = reinterpret_cast<R *>(s->base + o_xf);
    P.xg = reinterpret_cast<R *>(s->base + o_xg);
    P.xfr = reinterpret_cast<double *>(s->base + o_xfr);
    if (D == 2) {
        P.yf = reinterpret_cast<R *>(s->base + o_yf);
        P.yg = reinterpret_cast<R *>(s->base + o_yg);
        P.yfr = reinterpret_cast<double *>(s->base + o_yfr);
    }
    P.clock = reinterpret_cast<pond::Clock *>(s->base + o_clock);
    P.diag = reinterpret_cast<pond::Diag *>(s->base + o_diag);
    s->clock = P.clock;
    s->diag = P.diag;
    s->stage = reinterpret_cast<double *>(s->base + o_stage);
    s->stage_doubles = stage;
    CUDA_TRY(cudaMemsetAsync(s->base, 0, off, s->stream));
    new (s->params) P_t(P);
    return POND_OK;
}

pond_status reset_clock(pond_state *s)
{
    pond::Clock c{};
    c.t = 0.0;
    c.dt = 0.0;
    c.t_end = s->opts.t_end;
    c.cfl = s->opts.cfl;
    c.tau = s->tau;
    c.dx = (s->grid.x1 - s->grid.x0) / double(s->grid.nx);
    c.dy = s->D == 2 ? (s->grid.y1 - s->grid.y0) / double(s->grid.ny) : 1.0;
    pond::Diag d{};
    d.first_bad = -1;
    CUDA_TRY(cudaMemcpyAsync(s->clock, &c, sizeof(c), cudaMemcpyHostToDevice, s->stream));
    CUDA_TRY(cudaMemcpyAsync(s->diag, &d, sizeof(d), cudaMemcpyHostToDevice, s->stream));
    // the copies read host stack memory: complete them before returning
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    return POND_OK;
}

unsigned blocks_for(long long n, int threads) { return unsigned((n + threads - 1) / threads); }

template <int D, typename R>
pond_status set_primitive_impl(pond_state *s, const double *rho, const double *ux, const double *uy, const double *p, int on_device)
{
    auto &P = params_of<D, R>(s);
    const long long n = P.ncell();
    const double *dr = rho, *dux = ux, *duy = uy, *dp = p;
    if (!on_device) {
        double *st = s->stage;
        CUDA_TRY(cudaMemcpyAsync(st, rho, 8 * n, cudaMemcpyHostToDevice, s->stream));
        CUDA_TRY(cudaMemcpyAsync(st + n, ux, 8 * n, cudaMemcpyHostToDevice, s->stream));
        if (D == 2 && uy) CUDA_TRY(cudaMemcpyAsync(st + 2 * n, uy, 8 * n, cudaMemcpyHostToDevice, s->stream));
        CUDA_TRY(cudaMemcpyAsync(st + 3 * n, p, 8 * n, cudaMemcpyHostToDevice, s->stream));
        dr = st; dux = st + n; duy = (D == 2 && uy) ? st + 2 * n : nullptr; dp = st + 3 * n;
    }
    pond_status r = reset_clock(s);
    if (r != POND_OK) return r;
    pond::init_cells_kernel<D, R><<<blocks_for(n, 256), 256, 0, s->stream>>>(P, dr, dux, duy, dp);
    const long long nf = P.nxf() + (D == 2 ? P.nyf() : 0);
    pond::init_faces_kernel<D, R><<<blocks_for(nf, 256), 256, 0, s->stream>>>(P);
    s->launches += 2;
    CUDA_TRY(cudaGetLastError());
    if (!on_device) CUDA_TRY(cudaStreamSynchronize(s->stream));
    return POND_OK;
}

template <int D, typename R>
void launch_step(pond_state *s)
{
    auto &P = params_of<D, R>(s);
    using FT = pond::FaceTile<D>;
    dim3 fg(unsigned((P.nx + 1 + FT::TX - 1) / FT::TX), D == 2 ? unsigned((P.ny + 1 + FT::TY - 1) / FT::TY) : 1u);
    pond::face_kernel<D, R><<<fg, FT::THREADS, 0, s->stream>>>(P);
    pond::cell_kernel<D, R><<<blocks_for(P.ncell(), pond::CellBlock<D>::THREADS), pond::CellBlock<D>::THREADS, 0, s->stream>>>(P);
}

template <int D, typename R>
pond_status step_impl(pond_state *s, int64_t n_steps)
{
    int64_t left = n_steps;
    if (left >= kGraphSteps) {
        if (!s->graph_exec) {
            CUDA_TRY(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
            for (int k = 0; k < kGraphSteps; ++k) launch_step<D, R>(s);
            cudaGraph_t g = nullptr;
            CUDA_TRY(cudaStreamEndCapture(s->stream, &g));
            s->graph = g;
            CUDA_TRY(cudaGraphInstantiate(&s->graph_exec, g, 0));
        }
        while (left >= kGraphSteps) {
            CUDA_TRY(cudaGraphLaunch(s->graph_exec, s->stream));
            s->launches += 2 * kGraphSteps;
            left -= kGraphSteps;
        }
    }
    for (; left > 0; --left) {
        launch_step<D, R>(s);
        s->launches += 2;
    }
    CUDA_TRY(cudaGetLastError());
    return POND_OK;
}

template <int D, typename R>
pond_status step_timed_impl(pond_state *s, int64_t n_steps, double *ms)
{
    auto &P = params_of<D, R>(s);
    using FT = pond::FaceTile<D>;
    dim3 fg(unsigned((P.nx + 1 + FT::TX - 1) / FT::TX), D == 2 ? unsigned((P.ny + 1 + FT::TY - 1) / FT::TY) : 1u);
    const unsigned cb = blocks_for(P.ncell(), pond::CellBlock<D>::THREADS);
    std::vector<cudaEvent_t> ev(size_t(2 * n_steps + 1));
    for (auto &e : ev) CUDA_TRY(cudaEventCreate(&e));
    CUDA_TRY(cudaEventRecord(ev[0], s->stream));
    for (int64_t k = 0; k < n_steps; ++k) {
        pond::face_kernel<D, R><<<fg, FT::THREADS, 0, s->stream>>>(P);
        CUDA_TRY(cudaEventRecord(ev[2 * k + 1], s->stream));
        pond::cell_kernel<D, R><<<cb, pond::CellBlock<D>::THREADS, 0, s->stream>>>(P);
        CUDA_TRY(cudaEventRecord(ev[2 * k + 2], s->stream));
    }
    s->launches += 2 * n_steps;
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaEventSynchronize(ev.back()));
    for (int64_t k = 0; k < n_steps; ++k) {
        float a = 0.f, b = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&a, ev[2 * k], ev[2 * k + 1]));
        CUDA_TRY(cudaEventElapsedTime(&b, ev[2 * k + 1], ev[2 * k + 2]));
        ms[0] += a;
        ms[1] += b;
    }
    for (auto &e : ev) cudaEventDestroy(e);
    return POND_OK;
}

template <int D, typename R>
pond_status moments_impl(pond_state *s, double *rho, double *mx, double *my, double *E, double *totals, int on_device)
{
    auto &P = params_of<D, R>(s);
    const long long n = P.ncell();
    const bool need_stage = !on_device || totals;
    double *st = s->stage;
    double *o[4] = {rho, mx, my, E};
    double *d[4];
    for (int k = 0; k < 4; ++k) d[k] = (on_device && o[k]) ? o[k] : (need_stage ? st + k * n : nullptr);
    if (!need_stage && !rho && !mx && !my && !E) return POND_OK;
    pond::conserved_kernel<D, R><<<blocks_for(n, 256), 256, 0, s->stream>>>(P, d[0], d[1], d[2], d[3]);
    s->launches += 1;
    if (totals) {
        double *part = s->stage + (s->stage_doubles - (kReduceBlocks * 8 + 8));
        // the reduction staging sits at the end of the staging area, after 4n doubles only
        // when there is room; otherwise it reuses the front (fields are then copied first)
        const bool room = s->stage_doubles >= size_t(4 * n) + kReduceBlocks * 8 + 8;
        if (!room) {
            for (int k = 0; k < 4; ++k)
                if (o[k] && !on_device) CUDA_TRY(cudaMemcpyAsync(o[k], d[k], 8 * n, cudaMemcpyDeviceToHost, s->stream));
        }
        int nb = int(std::min<long long>(kReduceBlocks, (n + 255) / 256));
        pond::dd_partial_kernel<<<nb, 256, 0, s->stream>>>(d[0], d[1], d[2], d[3], n, part);
        const double vol = P.dx * P.dy;
        pond::dd_final_kernel<<<1, 32, 0, s->stream>>>(part, nb, vol, part + kReduceBlocks * 8);
        s->launches += 2;
        CUDA_TRY(cudaMemcpyAsync(totals, part + kReduceBlocks * 8, 4 * 8, cudaMemcpyDeviceToHost, s->stream));
        if (room && !on_device)
            for (int k = 0; k < 4; ++k)
                if (o[k]) CUDA_TRY(cudaMemcpyAsync(o[k], d[k], 8 * n, cudaMemcpyDeviceToHost, s->stream));
    } else if (!on_device) {
        for (int k = 0; k < 4; ++k)
            if (o[k]) CUDA_TRY(cudaMemcpyAsync(o[k], d[k], 8 * n, cudaMemcpyDeviceToHost, s->stream));
    }
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    return POND_OK;
}

template <int D, typename R>
pond_status get_state_impl(pond_state *s, double *cf, double *cg, double *fr)
{
    auto &P = params_of<D, R>(s);
    using P_t = pond::Params<D, R>;
    const long long n = P.ncell();
    double *st = s->stage;
    double *dcf = st, *dcg = st + P_t::NFC * n, *dfr = st + (P_t::NFC + P_t::NGC) * n;
    pond::export_state_kernel<D, R><<<blocks_for(n, 256), 256, 0, s->stream>>>(P, dcf, dcg, dfr);
    s->launches += 1;
    CUDA_TRY(cudaGetLastError());
    if (cf) CUDA_TRY(cudaMemcpyAsync(cf, dcf, 8 * P_t::NFC * n, cudaMemcpyDeviceToHost, s->stream));
    if (cg) CUDA_TRY(cudaMemcpyAsync(cg, dcg, 8 * P_t::NGC * n, cudaMemcpyDeviceToHost, s->stream));
    if (fr) CUDA_TRY(cudaMemcpyAsync(fr, dfr, 8 * (D + 1) * n, cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    return POND_OK;
}

// face frames are stored plane-major [D+1][nf]; the ABI exchanges [nf][D+1]
template <int D, typename R>
pond_status face_gauges_impl(pond_state *s, double *xg, double *yg, const double *xin, const double *yin)
{
    auto &P = params_of<D, R>(s);
    const long long nxf = P.nxf(), nyf = D == 2 ? P.nyf() : 0;
    const int w = D + 1;
    for (int dir = 0; dir < D; ++dir) {
        const long long nf = dir == 0 ? nxf : nyf;
        double *dev = dir == 0 ? P.xfr : P.yfr;
        std::vector<double> h(size_t(w) * nf);
        if (xin || yin) {
            const double *src = dir == 0 ? xin : yin;
            if (!src) continue;
            for (long long f = 0; f < nf; ++f)
                for (int a = 0; a < w; ++a) h[size_t(a) * nf + f] = src[f * w + a];
            CUDA_TRY(cudaMemcpyAsync(dev, h.data(), 8 * w * nf, cudaMemcpyHostToDevice, s->stream));
            CUDA_TRY(cudaStreamSynchronize(s->stream));
        } else {
            double *dst = dir == 0 ? xg : yg;
            if (!dst) continue;
            CUDA_TRY(cudaMemcpyAsync(h.data(), dev, 8 * w * nf, cudaMemcpyDeviceToHost, s->stream));
            CUDA_TRY(cudaStreamSynchronize(s->stream));
            for (long long f = 0; f < nf; ++f)
                for (int a = 0; a < w; ++a) dst[f * w + a] = h[size_t(a) * nf + f];
        }
    }
    return POND_OK;
}

template <typename Fn>
pond_status dispatch(pond_state *s, Fn &&fn)
{
    if (s->D == 1) return s->prec == POND_FP32 ? fn(std::integral_constant<int, 1>{}, float{}) : fn(std::integral_constant<int, 1>{}, double{});
    return s->prec == POND_FP32 ? fn(std::integral_constant<int, 2>{}, float{}) : fn(std::integral_constant<int, 2>{}, double{});
}

pond_status check_state(const pond_state *s)
{
    if (!s) return fail(POND_ERR_INVALID_ARG, "state is NULL");
    return POND_OK;
}

}  // namespace

extern "C" {

pond_status pond_init(const pond_grid *grid, pond_velset velset, double gamma, double tau, const pond_options *opts,
                      pond_state **out)
{
    if (!grid || !opts || !out) return fail(POND_ERR_INVALID_ARG, "grid, opts and out must not be NULL");
    *out = nullptr;
    if (velset == POND_D1Q3 || velset == POND_D2Q9)
        return fail(POND_ERR_UNSUPPORTED, "D1Q3/D2Q9 cannot carry the third-order Grad projection");
    if (velset != POND_D1Q4 && velset != POND_D2Q16) return fail(POND_ERR_INVALID_ARG, "unknown velocity set %d", int(velset));
    const int D = velset == POND_D1Q4 ? 1 : 2;
    if (grid->dim != D) return fail(POND_ERR_INVALID_ARG, "grid dim %d does not match the velocity set", grid->dim);
    if (grid->nx < 1 || (D == 2 && grid->ny < 1)) return fail(POND_ERR_INVALID_ARG, "grid must have at least one cell");
    if (!(grid->x1 > grid->x0) || (D == 2 && !(grid->y1 > grid->y0))) return fail(POND_ERR_INVALID_ARG, "empty domain");
    if (!(gamma > 1.0)) return fail(POND_ERR_INVALID_ARG, "gamma must exceed 1");
    if (1.0 / (gamma - 1.0) < 0.5 * D) return fail(POND_ERR_UNSUPPORTED, "gamma > 1 + 2/D makes Cv - D/2 negative");
    if (!(tau > 0.0)) return fail(POND_ERR_INVALID_ARG, "tau must be positive");
    if (opts->precision != POND_FP32 && opts->precision != POND_FP64) return fail(POND_ERR_INVALID_ARG, "bad precision");
    if (opts->limiter != POND_VANLEER && opts->limiter != POND_MINMOD) return fail(POND_ERR_INVALID_ARG, "bad limiter");
    if (!(opts->cfl > 0.0) || opts->max_iter < 1 || opts->fixed_iters < 0) return fail(POND_ERR_INVALID_ARG, "bad cfl/max_iter/fixed_iters");
    for (int k = 0; k < 4; ++k)
        if (grid->bc[k] < 0 || grid->bc[k] > 2) return fail(POND_ERR_INVALID_ARG, "bad boundary condition on side %d", k);
    if ((grid->bc[0] == POND_BC_PERIODIC) != (grid->bc[1] == POND_BC_PERIODIC) ||
        (D == 2 && (grid->bc[2] == POND_BC_PERIODIC) != (grid->bc[3] == POND_BC_PERIODIC)))
        return fail(POND_ERR_INVALID_ARG, "periodic sides must come in pairs");
    pond_state *s = new (std::nothrow) pond_state();
    if (!s) return fail(POND_ERR_OOM, "host allocation failed");
    s->D = D;
    s->prec = opts->precision;
    s->grid = *grid;
    if (D == 1) s->grid.ny = 1;
    s->opts = *opts;
    s->gamma = gamma;
    s->tau = tau;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e != cudaSuccess) { delete s; return fail(POND_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e)); }
    if (opts->stream) {
        s->stream = static_cast<cudaStream_t>(opts->stream);
    } else {
        e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete s; return fail(POND_ERR_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(e)); }
        s->own_stream = true;
    }
    pond_status st = dispatch(s, [&](auto d, auto r) { return setup<decltype(d)::value, decltype(r)>(s); });
    if (st == POND_OK) st = reset_clock(s);
    if (st != POND_OK) { pond_destroy(s); return st; }
    *out = s;
    return POND_OK;
}

pond_status pond_set_primitive(pond_state *s, const double *rho, const double *ux, const double *uy, const double *p, int on_device)
{
    if (pond_status st = check_state(s)) return st;
    if (!rho || !ux || !p || (s->D == 2 && !uy)) return fail(POND_ERR_INVALID_ARG, "rho, ux, p (and uy in 2D) must not be NULL");
    return dispatch(s, [&](auto d, auto r) { return set_primitive_impl<decltype(d)::value, decltype(r)>(s, rho, ux, uy, p, on_device); });
}

pond_status pond_step(pond_state *s, int64_t n_steps)
{
    if (pond_status st = check_state(s)) return st;
    if (n_steps < 0) return fail(POND_ERR_INVALID_ARG, "n_steps must be >= 0");
    return dispatch(s, [&](auto d, auto r) { return step_impl<decltype(d)::value, decltype(r)>(s, n_steps); });
}

pond_status pond_step_timed(pond_state *s, int64_t n_steps, double ms[2])
{
    if (pond_status st = check_state(s)) return st;
    if (n_steps < 0 || !ms) return fail(POND_ERR_INVALID_ARG, "n_steps must be >= 0 and ms not NULL");
    return dispatch(s, [&](auto d, auto r) { return step_timed_impl<decltype(d)::value, decltype(r)>(s, n_steps, ms); });
}

pond_status pond_moments(pond_state *s, double *rho, double *mx, double *my, double *E, double totals[4], int on_device)
{
    if (pond_status st = check_state(s)) return st;
    return dispatch(s, [&](auto d, auto r) { return moments_impl<decltype(d)::value, decltype(r)>(s, rho, mx, my, E, totals, on_device); });
}

pond_status pond_get_state(pond_state *s, double *coef_f, double *coef_g, double *frame)
{
    if (pond_status st = check_state(s)) return st;
    return dispatch(s, [&](auto d, auto r) { return get_state_impl<decltype(d)::value, decltype(r)>(s, coef_f, coef_g, frame); });
}

pond_status pond_get_face_gauges(pond_state *s, double *xg, double *yg)
{
    if (pond_status st = check_state(s)) return st;
    if (!xg && !yg) return POND_OK;
    return dispatch(s, [&](auto d, auto r) { return face_gauges_impl<decltype(d)::value, decltype(r)>(s, xg, yg, nullptr, nullptr); });
}

pond_status pond_set_face_gauges(pond_state *s, const double *xg, const double *yg)
{
    if (pond_status st = check_state(s)) return st;
    if (!xg && !yg) return POND_OK;
    return dispatch(s, [&](auto d, auto r) { return face_gauges_impl<decltype(d)::value, decltype(r)>(s, nullptr, nullptr, xg, yg); });
}

pond_status pond_sync(pond_state *s, pond_diag *diag)
{
    if (pond_status st = check_state(s)) return st;
    pond::Clock c{};
    pond::Diag d{};
    CUDA_TRY(cudaMemcpyAsync(&c, s->clock, sizeof(c), cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaMemcpyAsync(&d, s->diag, sizeof(d), cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    CUDA_TRY(cudaGetLastError());
    if (diag) {
        diag->t = c.t;
        diag->dt = c.dt;
        diag->steps = c.steps;
        diag->face_solves = (int64_t)d.face_solves;
        diag->face_iters = (int64_t)d.face_iters;
        diag->nonconverged = (int64_t)d.nonconv;
        diag->fallbacks = (int64_t)d.fallbacks;
        diag->nonphysical = (int64_t)d.nonphys;
        diag->first_bad_cell = d.first_bad;
        diag->flags = d.flags;
    }
    if (d.flags & pond::FLAG_NONPHYSICAL) return fail(POND_ERR_NONPHYSICAL, "non-physical state: %llu cells/faces, first cell %lld",
                                                      (unsigned long long)d.nonphys, (long long)d.first_bad);
    if (s->opts.strict_convergence && (d.flags & pond::FLAG_NOT_CONVERGED))
        return fail(POND_ERR_NOT_CONVERGED, "%llu faces stopped at max_iter", (unsigned long long)d.nonconv);
    return POND_OK;
}

int64_t pond_launch_count(const pond_state *s) { return s ? s->launches : 0; }

void pond_destroy(pond_state *s)
{
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->graph_exec) cudaGraphExecDestroy(s->graph_exec);
    if (s->graph) cudaGraphDestroy(s->graph);
    dev_free(s, s->base);
    if (s->own_stream) cudaStreamDestroy(s->stream);
    delete s;
}

const char *pond_last_error(void) { return g_err; }

}  // extern "C"
