// pond_api.cu -- host side of the C ABI declared in include/pond.h.
//
// A pond_state owns one device allocation holding the cell planes, the face planes, the
// device clock (time, time step, CFL reduction) and the diagnostics; every step is two
// kernel launches (face corrector, cell update) that read the time step from the device,
// so runs of steps are captured once into a CUDA graph and replayed.
#include <cuda_runtime.h>
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <new>
#include <utility>
#include <vector>
#include <mutex>
#include <string>

#include "../../include/pond.h"
#include "pond_launch.cuh"
#include "pond_sl2.cuh"
#include "pond3_launch.cuh"
#include "pond_mlp_train.cuh"
#include "pond_reduce.cuh"
#include <cuda_bf16.h>

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

constexpr size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// The CUDA events of one timed run, destroyed on every return path.
struct Events {
    std::vector<cudaEvent_t> ev;
    explicit Events(size_t n) : ev(n, nullptr) {}
    Events(const Events &) = delete;
    Events &operator=(const Events &) = delete;
    ~Events()
    {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    }
    cudaError_t create()
    {
        for (cudaEvent_t &e : ev) {
            const cudaError_t r = cudaEventCreate(&e);
            if (r != cudaSuccess) return r;
        }
        return cudaSuccess;
    }
    cudaEvent_t &operator[](size_t i) { return ev[i]; }
    cudaEvent_t back() const { return ev.back(); }
};

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
    // D3Q64 grids
    pond_grid3 grid3{};
    alignas(16) unsigned char params3[sizeof(pond::Params3<double>)];
    int64_t launches = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    // learned face-gauge predictor
    float *mlp = nullptr, *mlp_m = nullptr, *mlp_v = nullptr, *mlp_grad = nullptr, *mlp_loss = nullptr;
    unsigned int *mlp_err = nullptr;
    unsigned long long *pair_count = nullptr;
    char *mlp_block = nullptr;
    char *train_scratch = nullptr;
    int64_t train_rows = 0;
    bool learned = false;
    bool equilibrate = false;     // the equilibration alternative of Sec. II.C (an ablation)
    int adam_t = 0;
    int sms = 152;
    // kernel variants in use (indices into the lists of pond_launch.cuh), set by the autotuner;
    // on grids tube_v selects the step: 0 the face and cell kernels, k + 1 fused variant k
    int face_v = 0, cell_v = 0, tube_v = 0;
    // tensor maps of the two state buffers for the TMA-staged face variant (D2Q16, FP32)
    pond::StageMaps stage_maps[2] = {};
    // semi-Lagrangian scheme and fused steps: the state alternates between two sets of
    // planes; sl_parity counts the swaps, graph_parity is the parity a captured graph starts at
    int scheme = POND_FV;
    int sl_parity = 0, graph_parity = 0;
    // batched tubes
    bool batch = false;
    int64_t n_tubes = 0, ncell = 0, nface = 0, steps_taken = 0;
    int cur = 0;
    alignas(16) unsigned char tparams[sizeof(pond::TubeParams<double>)];
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

// cuTensorMapEncodeTiled from the driver, through the runtime (no link against libcuda)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// Tensor maps of the state planes (f: NFS planes, g: NGC planes, frame words: D + 1 planes)
// of both state buffers, as [planes][ny][nx] tensors copied in boxes of kTmaBoxX x (TY + 3)
// x planes for the 8 x 8 TMA face variant.  They need rows that are multiples of 16 bytes
// (nx a multiple of 4); false (no maps, the variant stages per thread) otherwise or when the
// driver refuses a map.
template <typename R>
bool encode_stage_maps(pond_state *s, long long nx, long long ny, const R *sf0, const R *sg0, const void *sfr0,
                       const R *sf1, const R *sg1, const void *sfr1)
{
    constexpr int NFS = pond::Params<2, R>::NFS, NGC = pond::Params<2, R>::NGC, BY = 8 + 3;
    if (nx % 4 != 0 || nx < 16 || ny < BY || nx > (1ll << 31) || ny > (1ll << 31)) return false;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    auto one = [&](CUtensorMap *m, const void *ptr, int planes, size_t es, CUtensorMapDataType ty) {
        const cuuint64_t dims[3] = {cuuint64_t(nx), cuuint64_t(ny), cuuint64_t(planes)};
        const cuuint64_t strides[2] = {cuuint64_t(nx) * es, cuuint64_t(nx) * cuuint64_t(ny) * es};
        const cuuint32_t box[3] = {cuuint32_t(pond::kTmaBoxX), cuuint32_t(BY), cuuint32_t(planes)};
        const cuuint32_t estr[3] = {1, 1, 1};
        return enc(m, ty, 3, const_cast<void *>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    const R *sf[2] = {sf0, sf1}, *sg[2] = {sg0, sg1};
    const void *sfr[2] = {sfr0, sfr1};
    for (int b = 0; b < 2; ++b) {
        pond::StageMaps &m = s->stage_maps[b];
        if (!one(&m.sf, sf[b], NFS, sizeof(R), CU_TENSOR_MAP_DATA_TYPE_FLOAT32) ||
            !one(&m.sg, sg[b], NGC, sizeof(R), CU_TENSOR_MAP_DATA_TYPE_FLOAT32) ||
            !one(&m.sfr, sfr[b], 3, 8, CU_TENSOR_MAP_DATA_TYPE_FLOAT64))
            return false;
        m.key = sf[b];
    }
    return true;
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
    P.Cv_r = R(P.Cv);
    P.Cvh_r = R(P.Cv - 0.5 * D);
    P.tol_r = R(P.tol);
    P.max_iter = s->opts.max_iter;
    P.fixed_iters = s->opts.fixed_iters;
    P.sms = s->sms;
    const long long n = P.ncell(), nxf = P.nxf(), nyf = D == 2 ? P.nyf() : 0;
    using W = typename P_t::W;
    constexpr int NFC = P_t::NFC, NGC = P_t::NGC, NFS = P_t::NFS;
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off = align_up(off + b, 256); return o; };
    const size_t o_sf = take(sizeof(R) * NFS * n), o_sg = take(sizeof(R) * NGC * n), o_sfr = take(sizeof(W) * (D + 1) * n);
    const size_t o_xf = take(sizeof(R) * NFC * nxf), o_xg = take(sizeof(R) * NGC * nxf), o_xfr = take(sizeof(W) * (D + 1) * nxf);
    size_t o_yf = 0, o_yg = 0, o_yfr = 0;
    size_t o_xlr = 0, o_ylr = 0;
    if (D == 2) {
        o_yf = take(sizeof(R) * NFC * nyf); o_yg = take(sizeof(R) * NGC * nyf); o_yfr = take(sizeof(W) * (D + 1) * nyf);
        o_xlr = take(sizeof(W) * (D + 1) * nxf); o_ylr = take(sizeof(W) * (D + 1) * nyf);  // learned predictions
    }
    size_t o_pact = 0;
    if (D == 2) o_pact = take(sizeof(unsigned int) * 2 * size_t(pond::pred_tiles(P)));
    // the fused step's second state and face-frame buffers
    const size_t o_sf2 = take(sizeof(R) * NFS * n), o_sg2 = take(sizeof(R) * NGC * n), o_sfr2 = take(sizeof(W) * (D + 1) * n);
    const size_t o_xfr2 = take(sizeof(W) * (D + 1) * nxf);
    const size_t o_yfr2 = D == 2 ? take(sizeof(W) * (D + 1) * nyf) : 0;
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
    P.sfr = reinterpret_cast<W *>(s->base + o_sfr);
    P.xf = reinterpret_cast<R *>(s->base + o_xf);
    P.xg = reinterpret_cast<R *>(s->base + o_xg);
    P.xfr = reinterpret_cast<W *>(s->base + o_xfr);
    if (D == 2) {
        P.yf = reinterpret_cast<R *>(s->base + o_yf);
        P.yg = reinterpret_cast<R *>(s->base + o_yg);
        P.yfr = reinterpret_cast<W *>(s->base + o_yfr);
        P.xlr = reinterpret_cast<W *>(s->base + o_xlr);
        P.pred_active = reinterpret_cast<unsigned int *>(s->base + o_pact);
        P.ylr = reinterpret_cast<W *>(s->base + o_ylr);
    }
    P.sf_n = reinterpret_cast<R *>(s->base + o_sf2);
    P.sg_n = reinterpret_cast<R *>(s->base + o_sg2);
    P.sfr_n = reinterpret_cast<W *>(s->base + o_sfr2);
    P.xfr_n = reinterpret_cast<W *>(s->base + o_xfr2);
    P.yfr_n = D == 2 ? reinterpret_cast<W *>(s->base + o_yfr2) : nullptr;
    P.clock = reinterpret_cast<pond::Clock *>(s->base + o_clock);
    P.diag = reinterpret_cast<pond::Diag *>(s->base + o_diag);
    s->clock = P.clock;
    s->diag = P.diag;
    s->stage = reinterpret_cast<double *>(s->base + o_stage);
    s->stage_doubles = stage;
    CUDA_TRY(cudaMemsetAsync(s->base, 0, off, s->stream));
    P.stage_maps = nullptr;
    if constexpr (D == 2 && sizeof(R) == 4) {
        if (encode_stage_maps<R>(s, P.nx, P.ny, P.sf, P.sg, P.sfr, P.sf_n, P.sg_n, P.sfr_n)) P.stage_maps = s->stage_maps;
    }
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
    c.dz = 1.0;
    if (s->D == 3) {
        c.dy = (s->grid3.y1 - s->grid3.y0) / double(s->grid3.ny);
        c.dz = (s->grid3.z1 - s->grid3.z0) / double(s->grid3.nz);
        c.dx = (s->grid3.x1 - s->grid3.x0) / double(s->grid3.nx);
    }
    pond::Diag d{};
    d.first_bad = -1;
    CUDA_TRY(cudaMemcpyAsync(s->clock, &c, sizeof(c), cudaMemcpyHostToDevice, s->stream));
    CUDA_TRY(cudaMemcpyAsync(s->diag, &d, sizeof(d), cudaMemcpyHostToDevice, s->stream));
    // the copies read host stack memory: complete them before returning
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    return POND_OK;
}

unsigned blocks_for(long long n, int threads) { return unsigned((n + threads - 1) / threads); }

// persistent CTAs of the learned predictor: kInferCtasPerSm per SM, at most one per tile
unsigned predict_blocks(const pond_state *s)
{
    const long long nbx = (s->grid.nx + 1 + pond::kPredTX - 1) / pond::kPredTX;
    const long long nby = (s->grid.ny + 1 + pond::kPredTY - 1) / pond::kPredTY;
    return unsigned(std::min<long long>(nbx * nby, (long long)pond::mlp::kInferCtasPerSm * s->sms));
}

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

// network parameters: seeded Xavier-uniform W1, W2; zero W3 and biases (the untrained
// predictor returns the previous half step's frame)
void mlp_default_params(std::vector<float> &p)
{
    namespace M = pond::mlp;
    p.assign(M::kParams, 0.f);
    uint64_t st = 0x243F6A8885A308D3ull;
    auto uni = [&]() {
        st = st * 6364136223846793005ull + 1442695040888963407ull;
        return float((st >> 40) & 0xFFFFFF) / float(1 << 24) * 2.f - 1.f;
    };
    const float a1 = std::sqrt(6.f / float(M::kUsed + M::kHid)), a2 = std::sqrt(6.f / float(2 * M::kHid));
    for (int o = 0; o < M::kHid; ++o)
        for (int i = 0; i < M::kUsed; ++i) p[M::oW1 + o * M::kIn + i] = a1 * uni();
    for (int e = 0; e < M::kHid * M::kHid; ++e) p[M::oW2 + e] = a2 * uni();
}

pond_status mlp_setup(pond_state *s)
{
    namespace M = pond::mlp;
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off = align_up(off + b, 256); return o; };
    const size_t o_p = take(4 * M::kParams), o_m = take(4 * M::kParams), o_v = take(4 * M::kParams),
                 o_g = take(4 * M::kParams), o_l = take(64), o_e = take(64), o_c = take(64);
    s->mlp_block = static_cast<char *>(dev_alloc(s, off));
    if (!s->mlp_block) return fail(POND_ERR_OOM, "device allocation of %zu bytes failed", off);
    CUDA_TRY(cudaMemsetAsync(s->mlp_block, 0, off, s->stream));
    s->mlp = reinterpret_cast<float *>(s->mlp_block + o_p);
    s->mlp_m = reinterpret_cast<float *>(s->mlp_block + o_m);
    s->mlp_v = reinterpret_cast<float *>(s->mlp_block + o_v);
    s->mlp_grad = reinterpret_cast<float *>(s->mlp_block + o_g);
    s->mlp_loss = reinterpret_cast<float *>(s->mlp_block + o_l);
    s->mlp_err = reinterpret_cast<unsigned int *>(s->mlp_block + o_e);
    s->pair_count = reinterpret_cast<unsigned long long *>(s->mlp_block + o_c);
    std::vector<float> p;
    mlp_default_params(p);
    CUDA_TRY(cudaMemcpyAsync(s->mlp, p.data(), 4 * M::kParams, cudaMemcpyHostToDevice, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    CUDA_TRY(cudaFuncSetAttribute(pond::mlp::tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, M::kTileSmem));
    CUDA_TRY(cudaFuncSetAttribute(pond::gauge_predict_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, M::kInferSmem));
    CUDA_TRY(cudaFuncSetAttribute(pond::gauge_predict_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, M::kInferSmem));
    int sms = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device));
    s->sms = sms;
    return POND_OK;
}

// one semi-Lagrangian step: the kernel reads the cell planes and writes the face planes,
// which then become the state (the swap is on the host copy of the parameters, so a
// captured graph holds both orders alternately)
constexpr int kSlThreads = 128;

// D2Q16: tiles of 8 x 8 nodes (FP32) or 8 x 4 (FP64), the per-thread scratch of 140
// collapsed coefficients in dynamic shared memory
template <typename R>
struct Sl2Tile {
    static constexpr int TX = 8, TY = sizeof(R) == 4 ? 8 : 4;
    static constexpr size_t scratch = size_t(TX) * TY * 140 * sizeof(R);
};

template <int D, typename R>
void launch_sl(pond_state *s, pond::Params<D, R> &P)
{
    if constexpr (D == 1) {
        pond::sl_kernel<R, kSlThreads><<<blocks_for(P.nx, kSlThreads), kSlThreads, 0, s->stream>>>(P);
    } else {
        using T = Sl2Tile<R>;
        const dim3 g(unsigned((P.nx + T::TX - 1) / T::TX), unsigned((P.ny + T::TY - 1) / T::TY));
        pond::sl2_kernel<R, T::TX, T::TY><<<g, T::TX * T::TY, T::scratch, s->stream>>>(P);
    }
    std::swap(P.sf, P.xf);
    std::swap(P.sg, P.xg);
    std::swap(P.sfr, P.xfr);
    s->sl_parity ^= 1;
}

// one fused step (face and cell work of a tile in one kernel): it writes the other set of
// state and face-frame planes, which then become the state (swapped on the host copy of the
// parameters, so a captured graph holds both orders alternately)
template <int D, typename R>
void launch_fused(pond_state *s, pond::Params<D, R> &P)
{
    pond::launch_step_fused<D, R>(s->tube_v - 1, P, s->stream);
    std::swap(P.sf, P.sf_n);
    std::swap(P.sg, P.sg_n);
    std::swap(P.sfr, P.sfr_n);
    std::swap(P.xfr, P.xfr_n);
    if constexpr (D == 2) std::swap(P.yfr, P.yfr_n);
    s->sl_parity ^= 1;
}

// the step runs fused: the tuner (or pond_set_variants) chose a fused variant and the step
// is the plain one (the learned predictor, pair collection and the equilibration ablation
// run the face and cell kernels)
template <int D, typename R>
bool fused_step(const pond_state *s, bool collect)
{
    return s->tube_v > 0 && !s->learned && !collect && !s->equilibrate && s->scheme == POND_FV;
}

template <int D, typename R>
void launch_step(pond_state *s, bool collect = false)
{
    auto &P = params_of<D, R>(s);
    if (s->scheme == POND_SL) {
        launch_sl<D, R>(s, P);
        return;
    }
    if (fused_step<D, R>(s, collect)) {
        launch_fused<D, R>(s, P);
        return;
    }
    if constexpr (D == 2) {
        if (s->learned) {
            pond::gauge_predict_kernel<R><<<predict_blocks(s), pond::mlp::kThreads, pond::mlp::kInferSmem, s->stream>>>(P);
            s->launches += 1;
        }
    }
    pond::launch_face<D, R>(s->face_v, D == 2 && collect, P, s->stream);
    pond::launch_cell_any<D, R>(s->cell_v, P, s->stream);
}

// Releases the captured step graph (it is captured again on the next long step).
void drop_graph(pond_state *s)
{
    if (s->graph_exec) cudaGraphExecDestroy(s->graph_exec);
    if (s->graph) cudaGraphDestroy(s->graph);
    s->graph_exec = nullptr;
    s->graph = nullptr;
}

// Instantiates a captured graph and keeps both on the state; on failure neither is kept.
pond_status keep_graph(pond_state *s, cudaGraph_t g)
{
    const cudaError_t e = cudaGraphInstantiate(&s->graph_exec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        s->graph_exec = nullptr;
        return fail(POND_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
    }
    s->graph = g;
    return POND_OK;
}

template <int D, typename R>
pond_status step_impl(pond_state *s, int64_t n_steps)
{
    int64_t left = n_steps;
    if (left >= kGraphSteps && s->graph_exec && s->graph_parity != s->sl_parity) {
        // the graph was captured starting from the other buffer
        drop_graph(s);
    }
    if (left >= kGraphSteps) {
        if (!s->graph_exec) {
            s->graph_parity = s->sl_parity;
            CUDA_TRY(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
            const int64_t before = s->launches;
            for (int k = 0; k < kGraphSteps; ++k) launch_step<D, R>(s);
            s->launches = before;
            cudaGraph_t g = nullptr;
            CUDA_TRY(cudaStreamEndCapture(s->stream, &g));
            if (pond_status st = keep_graph(s, g)) return st;
        }
        const int per_step = (s->scheme == POND_SL || fused_step<D, R>(s, false)) ? 1 : 2 + ((D == 2 && s->learned) ? 1 : 0);
        while (left >= kGraphSteps) {
            CUDA_TRY(cudaGraphLaunch(s->graph_exec, s->stream));
            s->launches += per_step * kGraphSteps;
            left -= kGraphSteps;
        }
    }
    for (; left > 0; --left) {
        const int64_t before = s->launches;
        launch_step<D, R>(s);
        s->launches = before + ((s->scheme == POND_SL || fused_step<D, R>(s, false)) ? 1 : 2 + ((D == 2 && s->learned) ? 1 : 0));
    }
    CUDA_TRY(cudaGetLastError());
    return POND_OK;
}

template <int D, typename R>
pond_status step_timed_impl(pond_state *s, int64_t n_steps, double *ms)
{
    auto &P = params_of<D, R>(s);
    Events ev(size_t(2 * n_steps + 1));
    CUDA_TRY(ev.create());
    CUDA_TRY(cudaEventRecord(ev[0], s->stream));
    for (int64_t k = 0; k < n_steps; ++k) {
        if constexpr (D == 2) {
            if (s->learned) {
                pond::gauge_predict_kernel<R><<<predict_blocks(s), pond::mlp::kThreads, pond::mlp::kInferSmem, s->stream>>>(P);
                s->launches += 1;
            }
        }
        if (s->scheme == POND_SL || fused_step<D, R>(s, false)) {
            // the whole step is one kernel (semi-Lagrangian or fused): it is timed as the first part
            if (s->scheme == POND_SL) launch_sl<D, R>(s, P);
            else launch_fused<D, R>(s, P);
            CUDA_TRY(cudaEventRecord(ev[2 * k + 1], s->stream));
            CUDA_TRY(cudaEventRecord(ev[2 * k + 2], s->stream));
            s->launches -= 1;
        } else {
            pond::launch_face<D, R>(s->face_v, false, P, s->stream);
            CUDA_TRY(cudaEventRecord(ev[2 * k + 1], s->stream));
            pond::launch_cell_any<D, R>(s->cell_v, P, s->stream);
            CUDA_TRY(cudaEventRecord(ev[2 * k + 2], s->stream));
        }
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
    using W = typename pond::Params<D, R>::W;
    const long long nxf = P.nxf(), nyf = D == 2 ? P.nyf() : 0;
    const int w = D + 1;
    for (int dir = 0; dir < D; ++dir) {
        const long long nf = dir == 0 ? nxf : nyf;
        W *dev = dir == 0 ? P.xfr : P.yfr;
        std::vector<W> h(size_t(w) * nf);
        if (xin || yin) {
            const double *src = dir == 0 ? xin : yin;
            if (!src) continue;
            for (long long f = 0; f < nf; ++f)
                for (int a = 0; a < w; ++a) pond::fr_store(h[size_t(a) * nf + f], src[f * w + a]);
            CUDA_TRY(cudaMemcpyAsync(dev, h.data(), sizeof(W) * w * nf, cudaMemcpyHostToDevice, s->stream));
            CUDA_TRY(cudaStreamSynchronize(s->stream));
        } else {
            double *dst = dir == 0 ? xg : yg;
            if (!dst) continue;
            CUDA_TRY(cudaMemcpyAsync(h.data(), dev, sizeof(W) * w * nf, cudaMemcpyDeviceToHost, s->stream));
            CUDA_TRY(cudaStreamSynchronize(s->stream));
            for (long long f = 0; f < nf; ++f)
                for (int a = 0; a < w; ++a) dst[f * w + a] = pond::fr_value(h[size_t(a) * nf + f]);
        }
    }
    return POND_OK;
}

// ------------------------------------------------------------------ batched tubes

template <typename R>
pond::TubeParams<R> &tparams_of(pond_state *s) { return *reinterpret_cast<pond::TubeParams<R> *>(s->tparams); }

template <typename R>
pond_status batch_setup(pond_state *s, const int64_t *lengths, const double *gammas, const double *dxs)
{
    using TP = pond::TubeParams<R>;
    TP P{};
    const int64_t nt = s->n_tubes;
    std::vector<long long> coff(nt), foff(nt);
    std::vector<int> len(nt), order(nt);
    std::vector<double> cv(nt), dx(nt);
    long long nc = 0, nf = 0;
    for (int64_t k = 0; k < nt; ++k) {
        coff[k] = nc;
        foff[k] = nf;
        len[k] = int(lengths[k]);
        nc += lengths[k];
        nf += lengths[k] + 1;
        cv[k] = 1.0 / (gammas[k] - 1.0);
        dx[k] = dxs ? dxs[k] : 1.0 / double(lengths[k]);
        order[k] = int(k);
    }
    // longest tubes first: the CTA scheduler then balances the rest
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return len[a] > len[b]; });
    s->ncell = nc;
    s->nface = nf;
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off = align_up(off + b, 256); return o; };
    const size_t o_coff = take(8 * nt), o_foff = take(8 * nt), o_len = take(4 * nt), o_ord = take(4 * nt);
    const size_t o_cv = take(8 * nt), o_dx = take(8 * nt), o_t = take(8 * nt), o_dt = take(8 * nt), o_tot = take(32 * nt);
    const size_t o_status = take(4 * nt), o_done = take(8 * nt);
    size_t o_sf[2], o_sg[2], o_sfr[2];
    for (int b = 0; b < 2; ++b) {
        o_sf[b] = take(sizeof(R) * 3 * nc);
        o_sg[b] = take(sizeof(R) * 3 * nc);
        o_sfr[b] = take(sizeof(typename TP::CellW) * 2 * nc);
    }
    size_t o_fu[2], o_fT[2];
    for (int b = 0; b < 2; ++b) {
        o_fu[b] = take(sizeof(typename TP::FaceW) * nf);
        o_fT[b] = take(sizeof(typename TP::FaceW) * nf);
    }
    const size_t o_diag = take(sizeof(pond::Diag)), o_clock = take(sizeof(pond::Clock));
    const size_t stage = std::max<size_t>(4 * size_t(nc), 7 * size_t(nc)) + 2 * size_t(nf) + 8;
    const size_t o_stage = take(8 * stage);
    s->bytes = off;
    s->base = static_cast<char *>(dev_alloc(s, off));
    if (!s->base) return fail(POND_ERR_OOM, "device allocation of %zu bytes failed", off);
    char *B = s->base;
    CUDA_TRY(cudaMemsetAsync(B, 0, off, s->stream));
    CUDA_TRY(cudaMemcpyAsync(B + o_coff, coff.data(), 8 * nt, cudaMemcpyHostToDevice, s->stream));
    CUDA_TRY(cudaMemcpyAsync(B + o_foff, foff.data(), 8 * nt, cudaMemcpyHostToDevice, s->stream));
    CUDA_TRY(cudaMemcpyAsync(B + o_len, len.data(), 4 * nt, cudaMemcpyHostToDevice, s->stream));
    CUDA_TRY(cudaMemcpyAsync(B + o_ord, order.data(), 4 * nt, cudaMemcpyHostToDevice, s->stream));
    CUDA_TRY(cudaMemcpyAsync(B + o_cv, cv.data(), 8 * nt, cudaMemcpyHostToDevice, s->stream));
    CUDA_TRY(cudaMemcpyAsync(B + o_dx, dx.data(), 8 * nt, cudaMemcpyHostToDevice, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));  // the host vectors go out of scope
    P.n_tubes = int(nt);
    P.cell_off = reinterpret_cast<const long long *>(B + o_coff);
    P.face_off = reinterpret_cast<const long long *>(B + o_foff);
    P.len = reinterpret_cast<const int *>(B + o_len);
    P.order = reinterpret_cast<const int *>(B + o_ord);
    P.Cv = reinterpret_cast<const double *>(B + o_cv);
    P.dx = reinterpret_cast<const double *>(B + o_dx);
    P.t = reinterpret_cast<double *>(B + o_t);
    P.dt = reinterpret_cast<double *>(B + o_dt);
    P.totals = reinterpret_cast<double *>(B + o_tot);
    P.status = reinterpret_cast<int *>(B + o_status);
    P.steps_done = reinterpret_cast<long long *>(B + o_done);
    for (int b = 0; b < 2; ++b) {
        P.sf[b] = reinterpret_cast<R *>(B + o_sf[b]);
        P.sg[b] = reinterpret_cast<R *>(B + o_sg[b]);
        P.sfr[b] = reinterpret_cast<typename TP::CellW *>(B + o_sfr[b]);
    }
    for (int b = 0; b < 2; ++b) {
        P.fu[b] = reinterpret_cast<typename TP::FaceW *>(B + o_fu[b]);
        P.fT[b] = reinterpret_cast<typename TP::FaceW *>(B + o_fT[b]);
    }
    P.diag = reinterpret_cast<pond::Diag *>(B + o_diag);
    P.tau = s->tau;
    P.cfl = s->opts.cfl;
    P.limiter = s->opts.limiter;
    P.tol = s->opts.tol;
    P.max_iter = s->opts.max_iter;
    P.fixed_iters = s->opts.fixed_iters;
    P.ncell = nc;
    P.nface = nf;
    s->diag = P.diag;
    s->clock = reinterpret_cast<pond::Clock *>(B + o_clock);
    s->stage = reinterpret_cast<double *>(B + o_stage);
    s->stage_doubles = stage;
    new (s->tparams) TP(P);
    return POND_OK;
}

template <typename R>
pond_status batch_set_primitive(pond_state *s, const double *rho, const double *ux, const double *p, int on_device)
{
    auto &P = tparams_of<R>(s);
    const long long n = s->ncell;
    const double *dr = rho, *du = ux, *dp = p;
    if (!on_device) {
        CUDA_TRY(cudaMemcpyAsync(s->stage, rho, 8 * n, cudaMemcpyHostToDevice, s->stream));
        CUDA_TRY(cudaMemcpyAsync(s->stage + n, ux, 8 * n, cudaMemcpyHostToDevice, s->stream));
        CUDA_TRY(cudaMemcpyAsync(s->stage + 2 * n, p, 8 * n, cudaMemcpyHostToDevice, s->stream));
        dr = s->stage; du = s->stage + n; dp = s->stage + 2 * n;
    }
    pond::Diag d{};
    d.first_bad = -1;
    CUDA_TRY(cudaMemcpyAsync(s->diag, &d, sizeof(d), cudaMemcpyHostToDevice, s->stream));
    s->cur = 0;
    s->steps_taken = 0;
    pond::tube_init_kernel<R><<<unsigned(s->n_tubes), pond::kTubeThreads, 0, s->stream>>>(P, 0, dr, du, dp);
    s->launches += 1;
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    return POND_OK;
}

template <typename R>
pond_status batch_step(pond_state *s, int64_t n_steps, double *ms)
{
    if (n_steps <= 0) return POND_OK;
    auto &P = tparams_of<R>(s);
    Events ev(ms ? 2 : 0);
    if (ms) {
        CUDA_TRY(ev.create());
        CUDA_TRY(cudaEventRecord(ev[0], s->stream));
    }
    pond::launch_tube<R>(s->tube_v, unsigned(s->n_tubes), P, int(n_steps), s->cur, s->stream);
    s->launches += 1;
    CUDA_TRY(cudaGetLastError());
    s->cur ^= int(n_steps & 1);
    s->steps_taken += n_steps;
    if (ms) {
        CUDA_TRY(cudaEventRecord(ev[1], s->stream));
        CUDA_TRY(cudaEventSynchronize(ev[1]));
        float a = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&a, ev[0], ev[1]));
        ms[0] += a;
    }
    return POND_OK;
}

template <typename R>
pond_status batch_moments(pond_state *s, double *rho, double *mx, double *my, double *E, double *totals, int on_device)
{
    auto &P = tparams_of<R>(s);
    const long long n = s->ncell;
    double *o[3] = {rho, mx, E};
    double *d[3];
    for (int k = 0; k < 3; ++k) d[k] = (on_device && o[k]) ? o[k] : (o[k] ? s->stage + k * n : nullptr);
    pond::tube_conserved_kernel<R><<<unsigned(s->n_tubes), pond::kTubeThreads, 0, s->stream>>>(P, s->cur, d[0], d[1], d[2]);
    s->launches += 1;
    CUDA_TRY(cudaGetLastError());
    if (my) {
        if (on_device) CUDA_TRY(cudaMemsetAsync(my, 0, 8 * n, s->stream));
        else std::memset(my, 0, 8 * n);
    }
    if (!on_device)
        for (int k = 0; k < 3; ++k)
            if (o[k]) CUDA_TRY(cudaMemcpyAsync(o[k], d[k], 8 * n, cudaMemcpyDeviceToHost, s->stream));
    if (totals) {
        std::vector<double> tt(size_t(4 * s->n_tubes));
        CUDA_TRY(cudaMemcpyAsync(tt.data(), P.totals, 32 * s->n_tubes, cudaMemcpyDeviceToHost, s->stream));
        CUDA_TRY(cudaStreamSynchronize(s->stream));
        for (int q = 0; q < 4; ++q) {  // Neumaier summation over tubes
            double sum = 0.0, comp = 0.0;
            for (int64_t k = 0; k < s->n_tubes; ++k) {
                const double v = tt[size_t(4 * k + q)], t2 = sum + v;
                comp += std::fabs(sum) >= std::fabs(v) ? (sum - t2) + v : (v - t2) + sum;
                sum = t2;
            }
            totals[q] = sum + comp;
        }
    }
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    return POND_OK;
}

template <typename R>
pond_status batch_get_state(pond_state *s, double *cf, double *cg, double *fr)
{
    auto &P = tparams_of<R>(s);
    const long long n = s->ncell;
    double *dcf = s->stage, *dcg = s->stage + 4 * n, *dfr = s->stage + 7 * n;
    if (s->stage_doubles < size_t(9 * n)) return fail(POND_ERR_OOM, "staging too small");
    pond::tube_export_kernel<R><<<unsigned((n + 255) / 256), 256, 0, s->stream>>>(P, s->cur, dcf, dcg, dfr);
    s->launches += 1;
    CUDA_TRY(cudaGetLastError());
    if (cf) CUDA_TRY(cudaMemcpyAsync(cf, dcf, 8 * 4 * n, cudaMemcpyDeviceToHost, s->stream));
    if (cg) CUDA_TRY(cudaMemcpyAsync(cg, dcg, 8 * 3 * n, cudaMemcpyDeviceToHost, s->stream));
    if (fr) CUDA_TRY(cudaMemcpyAsync(fr, dfr, 8 * 2 * n, cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    return POND_OK;
}

template <typename R>
pond_status batch_face_gauges(pond_state *s, double *out, const double *in)
{
    auto &P = tparams_of<R>(s);
    using W = typename pond::TubeParams<R>::FaceW;  // the face predictor's storage word
    const long long nf = s->nface;
    std::vector<W> u(nf), T(nf);
    if (in) {
        for (long long f = 0; f < nf; ++f) { u[f] = W(in[2 * f]); T[f] = W(in[2 * f + 1]); }
        CUDA_TRY(cudaMemcpyAsync(P.fu[s->cur], u.data(), sizeof(W) * nf, cudaMemcpyHostToDevice, s->stream));
        CUDA_TRY(cudaMemcpyAsync(P.fT[s->cur], T.data(), sizeof(W) * nf, cudaMemcpyHostToDevice, s->stream));
        CUDA_TRY(cudaStreamSynchronize(s->stream));
    } else {
        CUDA_TRY(cudaMemcpyAsync(u.data(), P.fu[s->cur], sizeof(W) * nf, cudaMemcpyDeviceToHost, s->stream));
        CUDA_TRY(cudaMemcpyAsync(T.data(), P.fT[s->cur], sizeof(W) * nf, cudaMemcpyDeviceToHost, s->stream));
        CUDA_TRY(cudaStreamSynchronize(s->stream));
        for (long long f = 0; f < nf; ++f) { out[2 * f] = double(u[f]); out[2 * f + 1] = double(T[f]); }
    }
    return POND_OK;
}

// ------------------------------------------------------------------ D3Q64 grids

template <typename R>
pond::Params3<R> &params3_of(pond_state *s) { return *reinterpret_cast<pond::Params3<R> *>(s->params3); }

template <typename R>
pond_status setup3(pond_state *s)
{
    using P_t = pond::Params3<R>;
    using W = typename P_t::W;
    P_t P{};
    const pond_grid3 &g = s->grid3;
    P.nx = g.nx;
    P.ny = g.ny;
    P.nz = g.nz;
    P.dx = (g.x1 - g.x0) / double(g.nx);
    P.dy = (g.y1 - g.y0) / double(g.ny);
    P.dz = (g.z1 - g.z0) / double(g.nz);
    for (int k = 0; k < 6; ++k) P.bc[k] = g.bc[k];
    P.gamma = s->gamma;
    P.Cv = 1.0 / (s->gamma - 1.0);
    P.tau = s->tau;
    P.limiter = s->opts.limiter;
    P.Cv_r = R(P.Cv);
    P.Cvh_r = R(P.Cv - 1.5);
    P.tol_r = R(s->opts.tol);
    P.max_iter = s->opts.max_iter;
    P.fixed_iters = s->opts.fixed_iters;
    const long long n = P.ncell();
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off = align_up(off + b, 256); return o; };
    const size_t o_sf = take(sizeof(R) * pond::kNFS3 * n), o_sg = take(sizeof(R) * pond::kNG3 * n);
    const size_t o_sfr = take(sizeof(W) * 4 * n);
    size_t o_ff[3], o_fg[3], o_ffr[3];
    long long nf_all = 0;
    for (int a = 0; a < 3; ++a) {
        const long long nf = P.nf(a);
        nf_all += nf;
        o_ff[a] = take(sizeof(R) * pond::kNF3 * nf);
        o_fg[a] = take(sizeof(R) * pond::kNG3 * nf);
        o_ffr[a] = take(sizeof(W) * 4 * nf);
    }
    const size_t o_clock = take(sizeof(pond::Clock)), o_diag = take(sizeof(pond::Diag));
    size_t stage = std::max<size_t>(5 * size_t(n), size_t(pond::kNF3 + pond::kNG3 + 4) * size_t(n));
    stage = std::max<size_t>(stage, 4 * size_t(nf_all));
    stage += 2 * (size_t(kReduceBlocks) * 8 + 8);
    const size_t o_stage = take(8 * stage);
    s->bytes = off;
    s->base = static_cast<char *>(dev_alloc(s, off));
    if (!s->base) return fail(POND_ERR_OOM, "device allocation of %zu bytes failed", off);
    P.sf = reinterpret_cast<R *>(s->base + o_sf);
    P.sg = reinterpret_cast<R *>(s->base + o_sg);
    P.sfr = reinterpret_cast<W *>(s->base + o_sfr);
    for (int a = 0; a < 3; ++a) {
        P.ff[a] = reinterpret_cast<R *>(s->base + o_ff[a]);
        P.fg[a] = reinterpret_cast<R *>(s->base + o_fg[a]);
        P.ffr[a] = reinterpret_cast<W *>(s->base + o_ffr[a]);
    }
    P.clock = reinterpret_cast<pond::Clock *>(s->base + o_clock);
    P.diag = reinterpret_cast<pond::Diag *>(s->base + o_diag);
    s->clock = P.clock;
    s->diag = P.diag;
    s->stage = reinterpret_cast<double *>(s->base + o_stage);
    s->stage_doubles = stage;
    CUDA_TRY(cudaMemsetAsync(s->base, 0, off, s->stream));
    CUDA_TRY(pond::prepare3<R>());
    new (s->params3) P_t(P);
    return POND_OK;
}

template <typename R>
pond_status set_primitive3_impl(pond_state *s, const double *rho, const double *ux, const double *uy, const double *uz,
                                const double *p, int on_device)
{
    auto &P = params3_of<R>(s);
    const long long n = P.ncell();
    const double *src[5] = {rho, ux, uy, uz, p};
    const double *d[5];
    for (int k = 0; k < 5; ++k) {
        if (on_device) {
            d[k] = src[k];
        } else {
            CUDA_TRY(cudaMemcpyAsync(s->stage + k * n, src[k], 8 * n, cudaMemcpyHostToDevice, s->stream));
            d[k] = s->stage + k * n;
        }
    }
    pond_status r = reset_clock(s);
    if (r != POND_OK) return r;
    pond::launch_init3<R>(P, d[0], d[1], d[2], d[3], d[4], s->stream);
    s->launches += 2;
    CUDA_TRY(cudaGetLastError());
    if (!on_device) CUDA_TRY(cudaStreamSynchronize(s->stream));
    return POND_OK;
}

template <typename R>
void launch_step3(pond_state *s)
{
    auto &P = params3_of<R>(s);
    pond::launch_face3<R>(s->face_v, P, s->stream);
    pond::launch_cell3<R>(s->cell_v, P, s->stream);
}

template <typename R>
pond_status step3_impl(pond_state *s, int64_t n_steps)
{
    int64_t left = n_steps;
    if (left >= kGraphSteps) {
        if (!s->graph_exec) {
            CUDA_TRY(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
            for (int k = 0; k < kGraphSteps; ++k) launch_step3<R>(s);
            cudaGraph_t g = nullptr;
            CUDA_TRY(cudaStreamEndCapture(s->stream, &g));
            if (pond_status st = keep_graph(s, g)) return st;
        }
        while (left >= kGraphSteps) {
            CUDA_TRY(cudaGraphLaunch(s->graph_exec, s->stream));
            s->launches += 2 * kGraphSteps;
            left -= kGraphSteps;
        }
    }
    for (; left > 0; --left) {
        launch_step3<R>(s);
        s->launches += 2;
    }
    CUDA_TRY(cudaGetLastError());
    return POND_OK;
}

template <typename R>
pond_status step3_timed_impl(pond_state *s, int64_t n_steps, double *ms)
{
    auto &P = params3_of<R>(s);
    Events ev(size_t(2 * n_steps + 1));
    CUDA_TRY(ev.create());
    CUDA_TRY(cudaEventRecord(ev[0], s->stream));
    for (int64_t k = 0; k < n_steps; ++k) {
        pond::launch_face3<R>(s->face_v, P, s->stream);
        CUDA_TRY(cudaEventRecord(ev[2 * k + 1], s->stream));
        pond::launch_cell3<R>(s->cell_v, P, s->stream);
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
    return POND_OK;
}

template <typename R>
pond_status moments3_impl(pond_state *s, double *rho, double *mx, double *my, double *mz, double *E, double *totals,
                          int on_device)
{
    auto &P = params3_of<R>(s);
    const long long n = P.ncell();
    double *o[5] = {rho, mx, my, mz, E};
    double *d[5];
    for (int k = 0; k < 5; ++k) d[k] = (on_device && o[k]) ? o[k] : s->stage + k * n;
    pond::launch_conserved3<R>(P, d[0], d[1], d[2], d[3], d[4], s->stream);
    s->launches += 1;
    if (totals) {
        double *part = s->stage + 5 * n;
        double *part2 = part + kReduceBlocks * 8 + 8;
        const int nb = int(std::min<long long>(kReduceBlocks, (n + 255) / 256));
        const double vol = P.dx * P.dy * P.dz;
        pond::dd_partial_kernel<<<nb, 256, 0, s->stream>>>(d[0], d[1], d[2], d[3], n, part);
        pond::dd_final_kernel<<<1, 32, 0, s->stream>>>(part, nb, vol, part + kReduceBlocks * 8);
        pond::dd_partial_kernel<<<nb, 256, 0, s->stream>>>(d[4], nullptr, nullptr, nullptr, n, part2);
        pond::dd_final_kernel<<<1, 32, 0, s->stream>>>(part2, nb, vol, part2 + kReduceBlocks * 8);
        s->launches += 4;
        CUDA_TRY(cudaMemcpyAsync(totals, part + kReduceBlocks * 8, 4 * 8, cudaMemcpyDeviceToHost, s->stream));
        CUDA_TRY(cudaMemcpyAsync(totals + 4, part2 + kReduceBlocks * 8, 8, cudaMemcpyDeviceToHost, s->stream));
    }
    if (!on_device)
        for (int k = 0; k < 5; ++k)
            if (o[k]) CUDA_TRY(cudaMemcpyAsync(o[k], d[k], 8 * n, cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    return POND_OK;
}

template <typename R>
pond_status get_state3_impl(pond_state *s, double *cf, double *cg, double *fr)
{
    auto &P = params3_of<R>(s);
    const long long n = P.ncell();
    double *dcf = s->stage, *dcg = dcf + pond::kNF3 * n, *dfr = dcg + pond::kNG3 * n;
    pond::launch_export3<R>(P, dcf, dcg, dfr, s->stream);
    s->launches += 1;
    CUDA_TRY(cudaGetLastError());
    if (cf) CUDA_TRY(cudaMemcpyAsync(cf, dcf, 8 * pond::kNF3 * n, cudaMemcpyDeviceToHost, s->stream));
    if (cg) CUDA_TRY(cudaMemcpyAsync(cg, dcg, 8 * pond::kNG3 * n, cudaMemcpyDeviceToHost, s->stream));
    if (fr) CUDA_TRY(cudaMemcpyAsync(fr, dfr, 8 * 4 * n, cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    return POND_OK;
}

// face frames are stored plane-major [4][nf]; the ABI exchanges [nf][4]
template <typename R>
pond_status face_gauges3_impl(pond_state *s, double *const *out, const double *const *in)
{
    auto &P = params3_of<R>(s);
    using W = typename pond::Params3<R>::W;
    for (int a = 0; a < 3; ++a) {
        const long long nf = P.nf(a);
        std::vector<W> h(size_t(4) * nf);
        if (in) {
            if (!in[a]) continue;
            for (long long f = 0; f < nf; ++f)
                for (int q = 0; q < 4; ++q) pond::fr_store(h[size_t(q) * nf + f], in[a][f * 4 + q]);
            CUDA_TRY(cudaMemcpyAsync(P.ffr[a], h.data(), sizeof(W) * 4 * nf, cudaMemcpyHostToDevice, s->stream));
            CUDA_TRY(cudaStreamSynchronize(s->stream));
        } else {
            if (!out[a]) continue;
            CUDA_TRY(cudaMemcpyAsync(h.data(), P.ffr[a], sizeof(W) * 4 * nf, cudaMemcpyDeviceToHost, s->stream));
            CUDA_TRY(cudaStreamSynchronize(s->stream));
            for (long long f = 0; f < nf; ++f)
                for (int q = 0; q < 4; ++q) out[a][f * 4 + q] = pond::fr_value(h[size_t(q) * nf + f]);
        }
    }
    return POND_OK;
}

template <typename Fn>
pond_status dispatch_batch(pond_state *s, Fn &&fn)
{
    return s->prec == POND_FP32 ? fn(float{}) : fn(double{});
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
    if (velset == POND_D3Q64) return fail(POND_ERR_UNSUPPORTED, "D3Q64 grids are created by pond_init3");
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
    if (opts->scheme != POND_FV && opts->scheme != POND_SL) return fail(POND_ERR_INVALID_ARG, "bad scheme %d", opts->scheme);
    if (opts->scheme == POND_SL && !(opts->cfl < 1.0))
        return fail(POND_ERR_INVALID_ARG, "the semi-Lagrangian stencil needs cfl < 1");
    for (int k = 0; k < 4; ++k)
        if (grid->bc[k] < 0 || grid->bc[k] > 3) return fail(POND_ERR_INVALID_ARG, "bad boundary condition on side %d", k);
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
    s->scheme = opts->scheme;
    s->gamma = gamma;
    s->tau = tau;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e != cudaSuccess) { delete s; return fail(POND_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e)); }
    e = cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device);
    if (e != cudaSuccess) { delete s; return fail(POND_ERR_CUDA, "cudaDeviceGetAttribute: %s", cudaGetErrorString(e)); }
    if (opts->stream) {
        s->stream = static_cast<cudaStream_t>(opts->stream);
    } else {
        e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete s; return fail(POND_ERR_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(e)); }
        s->own_stream = true;
    }
    pond_status st = dispatch(s, [&](auto d, auto r) { return setup<decltype(d)::value, decltype(r)>(s); });
    if (st == POND_OK && D == 2 && s->scheme == POND_SL) {
        // the 2D semi-Lagrangian kernel's scratch can exceed the default dynamic shared memory
        const cudaError_t ea = s->prec == POND_FP32
            ? cudaFuncSetAttribute(pond::sl2_kernel<float, Sl2Tile<float>::TX, Sl2Tile<float>::TY>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, int(Sl2Tile<float>::scratch))
            : cudaFuncSetAttribute(pond::sl2_kernel<double, Sl2Tile<double>::TX, Sl2Tile<double>::TY>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, int(Sl2Tile<double>::scratch));
        if (ea != cudaSuccess) st = fail(POND_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(ea));
    }
    if (st == POND_OK && D == 2) {
        st = mlp_setup(s);
        if (st == POND_OK) {
            auto wire = [&](auto &P) {
                P.mlp = s->mlp; P.mlp_err = s->mlp_err; P.pair_count = s->pair_count; P.pair_every = 1;
                P.gauge_gate = 0.01f;
                P.gauge_trust = 0.5f;
            };
            if (s->prec == POND_FP32) wire(params_of<2, float>(s));
            else wire(params_of<2, double>(s));
        }
    }
    if (st == POND_OK) st = reset_clock(s);
    if (st != POND_OK) { pond_destroy(s); return st; }
    s->learned = D == 2 && opts->learned != 0;
    if (s->learned) {
        if (s->prec == POND_FP32) params_of<2, float>(s).use_learned = 1;
        else params_of<2, double>(s).use_learned = 1;
    }
    *out = s;
    return POND_OK;
}

pond_status pond_init3(const pond_grid3 *grid, double gamma, double tau, const pond_options *opts, pond_state **out)
{
    if (!grid || !opts || !out) return fail(POND_ERR_INVALID_ARG, "grid, opts and out must not be NULL");
    *out = nullptr;
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return fail(POND_ERR_INVALID_ARG, "grid must have at least one cell");
    if (!(grid->x1 > grid->x0) || !(grid->y1 > grid->y0) || !(grid->z1 > grid->z0)) return fail(POND_ERR_INVALID_ARG, "empty domain");
    if (!(gamma > 1.0)) return fail(POND_ERR_INVALID_ARG, "gamma must exceed 1");
    if (1.0 / (gamma - 1.0) < 1.5) return fail(POND_ERR_UNSUPPORTED, "gamma > 5/3 makes Cv - 3/2 negative");
    if (!(tau > 0.0)) return fail(POND_ERR_INVALID_ARG, "tau must be positive");
    if (opts->precision != POND_FP32 && opts->precision != POND_FP64) return fail(POND_ERR_INVALID_ARG, "bad precision");
    if (opts->limiter != POND_VANLEER && opts->limiter != POND_MINMOD) return fail(POND_ERR_INVALID_ARG, "bad limiter");
    if (!(opts->cfl > 0.0) || opts->max_iter < 1 || opts->fixed_iters < 0) return fail(POND_ERR_INVALID_ARG, "bad cfl/max_iter/fixed_iters");
    if (opts->scheme != POND_FV) return fail(POND_ERR_UNSUPPORTED, "D3Q64 grids run the finite-volume scheme");
    if (opts->learned) return fail(POND_ERR_UNSUPPORTED, "the learned predictor is a D2Q16 feature");
    for (int k = 0; k < 6; ++k)
        if (grid->bc[k] != POND_BC_TRANSMISSIVE && grid->bc[k] != POND_BC_PERIODIC && grid->bc[k] != POND_BC_REFLECTIVE)
            return fail(POND_ERR_INVALID_ARG, "side %d: D3Q64 sides are transmissive, periodic or reflective", k);
    for (int a = 0; a < 3; ++a)
        if ((grid->bc[2 * a] == POND_BC_PERIODIC) != (grid->bc[2 * a + 1] == POND_BC_PERIODIC))
            return fail(POND_ERR_INVALID_ARG, "periodic sides must come in pairs");
    pond_state *s = new (std::nothrow) pond_state();
    if (!s) return fail(POND_ERR_OOM, "host allocation failed");
    s->D = 3;
    s->prec = opts->precision;
    s->grid3 = *grid;
    s->grid.dim = 3;
    s->grid.nx = grid->nx;
    s->grid.ny = grid->ny;
    s->opts = *opts;
    s->scheme = POND_FV;
    s->gamma = gamma;
    s->tau = tau;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e != cudaSuccess) { delete s; return fail(POND_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e)); }
    e = cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device);
    if (e != cudaSuccess) { delete s; return fail(POND_ERR_CUDA, "cudaDeviceGetAttribute: %s", cudaGetErrorString(e)); }
    if (opts->stream) {
        s->stream = static_cast<cudaStream_t>(opts->stream);
    } else {
        e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete s; return fail(POND_ERR_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(e)); }
        s->own_stream = true;
    }
    pond_status st = s->prec == POND_FP32 ? setup3<float>(s) : setup3<double>(s);
    if (st == POND_OK) st = reset_clock(s);
    if (st != POND_OK) { pond_destroy(s); return st; }
    *out = s;
    return POND_OK;
}

pond_status pond_set_primitive3(pond_state *s, const double *rho, const double *ux, const double *uy, const double *uz,
                                const double *p, int on_device)
{
    if (pond_status st = check_state(s)) return st;
    if (s->D != 3) return fail(POND_ERR_INVALID_ARG, "pond_set_primitive3 needs a D3Q64 state");
    if (!rho || !ux || !uy || !uz || !p) return fail(POND_ERR_INVALID_ARG, "rho, ux, uy, uz, p must not be NULL");
    return s->prec == POND_FP32 ? set_primitive3_impl<float>(s, rho, ux, uy, uz, p, on_device)
                                : set_primitive3_impl<double>(s, rho, ux, uy, uz, p, on_device);
}

pond_status pond_moments3(pond_state *s, double *rho, double *mx, double *my, double *mz, double *E, double totals[5],
                          int on_device)
{
    if (pond_status st = check_state(s)) return st;
    if (s->D != 3) return fail(POND_ERR_INVALID_ARG, "pond_moments3 needs a D3Q64 state");
    return s->prec == POND_FP32 ? moments3_impl<float>(s, rho, mx, my, mz, E, totals, on_device)
                                : moments3_impl<double>(s, rho, mx, my, mz, E, totals, on_device);
}

pond_status pond_get_face_gauges3(pond_state *s, double *xg, double *yg, double *zg)
{
    if (pond_status st = check_state(s)) return st;
    if (s->D != 3) return fail(POND_ERR_INVALID_ARG, "pond_get_face_gauges3 needs a D3Q64 state");
    double *out[3] = {xg, yg, zg};
    return s->prec == POND_FP32 ? face_gauges3_impl<float>(s, out, nullptr) : face_gauges3_impl<double>(s, out, nullptr);
}

pond_status pond_set_face_gauges3(pond_state *s, const double *xg, const double *yg, const double *zg)
{
    if (pond_status st = check_state(s)) return st;
    if (s->D != 3) return fail(POND_ERR_INVALID_ARG, "pond_set_face_gauges3 needs a D3Q64 state");
    const double *in[3] = {xg, yg, zg};
    return s->prec == POND_FP32 ? face_gauges3_impl<float>(s, nullptr, in) : face_gauges3_impl<double>(s, nullptr, in);
}

pond_status pond_set_primitive(pond_state *s, const double *rho, const double *ux, const double *uy, const double *p, int on_device)
{
    if (pond_status st = check_state(s)) return st;
    if (s->D == 3) return fail(POND_ERR_INVALID_ARG, "D3Q64 states take pond_set_primitive3");
    if (!rho || !ux || !p || (s->D == 2 && !uy)) return fail(POND_ERR_INVALID_ARG, "rho, ux, p (and uy in 2D) must not be NULL");
    if (s->batch) return dispatch_batch(s, [&](auto r) { return batch_set_primitive<decltype(r)>(s, rho, ux, p, on_device); });
    return dispatch(s, [&](auto d, auto r) { return set_primitive_impl<decltype(d)::value, decltype(r)>(s, rho, ux, uy, p, on_device); });
}

pond_status pond_step(pond_state *s, int64_t n_steps)
{
    if (pond_status st = check_state(s)) return st;
    if (n_steps < 0) return fail(POND_ERR_INVALID_ARG, "n_steps must be >= 0");
    if (s->batch) return dispatch_batch(s, [&](auto r) { return batch_step<decltype(r)>(s, n_steps, nullptr); });
    if (s->D == 3) return s->prec == POND_FP32 ? step3_impl<float>(s, n_steps) : step3_impl<double>(s, n_steps);
    return dispatch(s, [&](auto d, auto r) { return step_impl<decltype(d)::value, decltype(r)>(s, n_steps); });
}

pond_status pond_step_timed(pond_state *s, int64_t n_steps, double ms[2])
{
    if (pond_status st = check_state(s)) return st;
    if (n_steps < 0 || !ms) return fail(POND_ERR_INVALID_ARG, "n_steps must be >= 0 and ms not NULL");
    if (s->batch) return dispatch_batch(s, [&](auto r) { return batch_step<decltype(r)>(s, n_steps, ms); });
    if (s->D == 3) return s->prec == POND_FP32 ? step3_timed_impl<float>(s, n_steps, ms) : step3_timed_impl<double>(s, n_steps, ms);
    return dispatch(s, [&](auto d, auto r) { return step_timed_impl<decltype(d)::value, decltype(r)>(s, n_steps, ms); });
}

pond_status pond_moments(pond_state *s, double *rho, double *mx, double *my, double *E, double totals[4], int on_device)
{
    if (pond_status st = check_state(s)) return st;
    if (s->batch) return dispatch_batch(s, [&](auto r) { return batch_moments<decltype(r)>(s, rho, mx, my, E, totals, on_device); });
    if (s->D == 3) return fail(POND_ERR_INVALID_ARG, "D3Q64 states take pond_moments3");
    return dispatch(s, [&](auto d, auto r) { return moments_impl<decltype(d)::value, decltype(r)>(s, rho, mx, my, E, totals, on_device); });
}

pond_status pond_get_state(pond_state *s, double *coef_f, double *coef_g, double *frame)
{
    if (pond_status st = check_state(s)) return st;
    if (s->batch) return dispatch_batch(s, [&](auto r) { return batch_get_state<decltype(r)>(s, coef_f, coef_g, frame); });
    if (s->D == 3) return s->prec == POND_FP32 ? get_state3_impl<float>(s, coef_f, coef_g, frame)
                                               : get_state3_impl<double>(s, coef_f, coef_g, frame);
    return dispatch(s, [&](auto d, auto r) { return get_state_impl<decltype(d)::value, decltype(r)>(s, coef_f, coef_g, frame); });
}

pond_status pond_get_face_gauges(pond_state *s, double *xg, double *yg)
{
    if (pond_status st = check_state(s)) return st;
    if (!xg && !yg) return POND_OK;
    if (s->D == 3) return fail(POND_ERR_INVALID_ARG, "D3Q64 states take pond_get_face_gauges3");
    if (s->scheme == POND_SL) return fail(POND_ERR_UNSUPPORTED, "the semi-Lagrangian scheme has no face frames");
    if (s->batch) return xg ? dispatch_batch(s, [&](auto r) { return batch_face_gauges<decltype(r)>(s, xg, nullptr); }) : POND_OK;
    return dispatch(s, [&](auto d, auto r) { return face_gauges_impl<decltype(d)::value, decltype(r)>(s, xg, yg, nullptr, nullptr); });
}

pond_status pond_set_face_gauges(pond_state *s, const double *xg, const double *yg)
{
    if (pond_status st = check_state(s)) return st;
    if (!xg && !yg) return POND_OK;
    if (s->D == 3) return fail(POND_ERR_INVALID_ARG, "D3Q64 states take pond_set_face_gauges3");
    if (s->scheme == POND_SL) return fail(POND_ERR_UNSUPPORTED, "the semi-Lagrangian scheme has no face frames");
    if (s->batch) return xg ? dispatch_batch(s, [&](auto r) { return batch_face_gauges<decltype(r)>(s, nullptr, xg); }) : POND_OK;
    return dispatch(s, [&](auto d, auto r) { return face_gauges_impl<decltype(d)::value, decltype(r)>(s, nullptr, nullptr, xg, yg); });
}

pond_status pond_sync(pond_state *s, pond_diag *diag)
{
    if (pond_status st = check_state(s)) return st;
    pond::Clock c{};
    pond::Diag d{};
    CUDA_TRY(cudaMemcpyAsync(&c, s->clock, sizeof(c), cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaMemcpyAsync(&d, s->diag, sizeof(d), cudaMemcpyDeviceToHost, s->stream));
    unsigned int mlp_e = 0;   // set by a tensor-core wait of the learned predictor that expired
    if (s->mlp_err) CUDA_TRY(cudaMemcpyAsync(&mlp_e, s->mlp_err, sizeof(mlp_e), cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    CUDA_TRY(cudaGetLastError());
    if (mlp_e) d.flags |= pond::FLAG_TIMEOUT;
    if (s->batch) {
        c.t = 0.0;
        c.dt = 0.0;
        c.steps = s->steps_taken;
    }
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
        diag->staged_tma = (int64_t)d.tma_tiles;
    }
    if (d.flags & pond::FLAG_NONPHYSICAL) return fail(POND_ERR_NONPHYSICAL, "non-physical state: %llu cells/faces, first cell %lld",
                                                      (unsigned long long)d.nonphys, (long long)d.first_bad);
    if (d.flags & pond::FLAG_TIMEOUT)
        return fail(POND_ERR_TIMEOUT, "a bounded device-side wait expired: a tensor-core wait of the learned predictor "
                                      "(its faces started from the previous half step's frame) or a face tile's TMA "
                                      "staging (the tile was staged per thread)");
    if (s->opts.strict_convergence && (d.flags & pond::FLAG_NOT_CONVERGED))
        return fail(POND_ERR_NOT_CONVERGED, "%llu faces stopped at max_iter", (unsigned long long)d.nonconv);
    return POND_OK;
}

pond_status pond_init_batch(int64_t n_tubes, const int64_t *lengths, const double *gammas, const double *dx, double tau,
                            const pond_options *opts, pond_state **out)
{
    if (!lengths || !gammas || !opts || !out || n_tubes <= 0) return fail(POND_ERR_INVALID_ARG, "bad batch arguments");
    *out = nullptr;
    if (n_tubes > (int64_t(1) << 31) - 1) return fail(POND_ERR_INVALID_ARG, "too many tubes");
    for (int64_t k = 0; k < n_tubes; ++k) {
        if (lengths[k] < 1 || lengths[k] > (int64_t(1) << 30)) return fail(POND_ERR_INVALID_ARG, "tube %lld: bad length", (long long)k);
        if (!(gammas[k] > 1.0)) return fail(POND_ERR_INVALID_ARG, "tube %lld: gamma must exceed 1", (long long)k);
        if (1.0 / (gammas[k] - 1.0) < 0.5) return fail(POND_ERR_UNSUPPORTED, "tube %lld: gamma > 3 makes Cv - 1/2 negative", (long long)k);
        if (dx && !(dx[k] > 0.0)) return fail(POND_ERR_INVALID_ARG, "tube %lld: dx must be positive", (long long)k);
    }
    if (!(tau > 0.0)) return fail(POND_ERR_INVALID_ARG, "tau must be positive");
    if (opts->precision != POND_FP32 && opts->precision != POND_FP64) return fail(POND_ERR_INVALID_ARG, "bad precision");
    if (opts->limiter != POND_VANLEER && opts->limiter != POND_MINMOD) return fail(POND_ERR_INVALID_ARG, "bad limiter");
    if (!(opts->cfl > 0.0) || opts->max_iter < 1 || opts->fixed_iters < 0) return fail(POND_ERR_INVALID_ARG, "bad cfl/max_iter/fixed_iters");
    if (opts->scheme != POND_FV) return fail(POND_ERR_UNSUPPORTED, "batches run the finite-volume scheme only");
    pond_state *s = new (std::nothrow) pond_state();
    if (!s) return fail(POND_ERR_OOM, "host allocation failed");
    s->batch = true;
    s->D = 1;
    s->prec = opts->precision;
    s->opts = *opts;
    s->tau = tau;
    s->n_tubes = n_tubes;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e != cudaSuccess) { delete s; return fail(POND_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e)); }
    e = cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device);
    if (e != cudaSuccess) { delete s; return fail(POND_ERR_CUDA, "cudaDeviceGetAttribute: %s", cudaGetErrorString(e)); }
    if (opts->stream) {
        s->stream = static_cast<cudaStream_t>(opts->stream);
    } else {
        e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete s; return fail(POND_ERR_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(e)); }
        s->own_stream = true;
    }
    pond_status st = dispatch_batch(s, [&](auto r) { return batch_setup<decltype(r)>(s, lengths, gammas, dx); });
    if (st != POND_OK) { pond_destroy(s); return st; }
    *out = s;
    return POND_OK;
}

pond_status pond_batch_status(pond_state *s, int32_t *status, int64_t *steps_done)
{
    if (pond_status st = check_state(s)) return st;
    if (!s->batch) return fail(POND_ERR_INVALID_ARG, "not a batch state");
    const int *sp = s->prec == POND_FP32 ? tparams_of<float>(s).status : tparams_of<double>(s).status;
    const long long *dp = s->prec == POND_FP32 ? tparams_of<float>(s).steps_done : tparams_of<double>(s).steps_done;
    if (status) CUDA_TRY(cudaMemcpyAsync(status, sp, 4 * s->n_tubes, cudaMemcpyDeviceToHost, s->stream));
    if (steps_done) CUDA_TRY(cudaMemcpyAsync(steps_done, dp, 8 * s->n_tubes, cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    return POND_OK;
}

pond_status pond_batch_times(pond_state *s, double *t, double *dt)
{
    if (pond_status st = check_state(s)) return st;
    if (!s->batch) return fail(POND_ERR_INVALID_ARG, "not a batch state");
    const double *dtp = s->prec == POND_FP32 ? tparams_of<float>(s).dt : tparams_of<double>(s).dt;
    const double *tp = s->prec == POND_FP32 ? tparams_of<float>(s).t : tparams_of<double>(s).t;
    if (t) CUDA_TRY(cudaMemcpyAsync(t, tp, 8 * s->n_tubes, cudaMemcpyDeviceToHost, s->stream));
    if (dt) CUDA_TRY(cudaMemcpyAsync(dt, dtp, 8 * s->n_tubes, cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    return POND_OK;
}

// ------------------------------------------------------------ learned predictor

}  // extern "C"

namespace {

pond_status check_gauge(pond_state *s)
{
    if (pond_status st = check_state(s)) return st;
    if (s->batch || s->D != 2 || !s->mlp) return fail(POND_ERR_UNSUPPORTED, "the learned predictor needs a D2Q16 grid state");
    return POND_OK;
}

template <typename R>
pond_status gauge_collect_impl(pond_state *s, int64_t n_steps, float *pairs, int64_t cap, int every, int64_t *n_out)
{
    auto &P = params_of<2, R>(s);
    CUDA_TRY(cudaMemsetAsync(s->pair_count, 0, sizeof(unsigned long long), s->stream));
    P.pairs = pairs;
    P.pair_cap = cap;
    P.pair_every = every;
    for (int64_t k = 0; k < n_steps; ++k) {
        launch_step<2, R>(s, true);
        s->launches += 2;
    }
    P.pairs = nullptr;
    CUDA_TRY(cudaGetLastError());
    unsigned long long cnt = 0;
    CUDA_TRY(cudaMemcpyAsync(&cnt, s->pair_count, sizeof(cnt), cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    if (n_out) *n_out = int64_t(std::min<unsigned long long>(cnt, (unsigned long long)cap));
    return POND_OK;
}

// scratch of a training minibatch of `rows` rows: the activations out, H1, H2, dOut, dZ1,
// dZ2, and the partial weight gradients of the split batch
constexpr size_t kWgradPartBytes = size_t(pond::mlp::kWgradMaxSplit) * pond::mlp::kParams * 4;
struct TrainScratch {
    float *out;
    __nv_bfloat16 *H1, *H2, *dOut, *dZ1, *dZ2;
    float *part;
    static constexpr size_t bytes(int64_t rows)
    {
        return size_t(rows) * (16 * 4 + 2 * (64 + 64 + 16 + 64 + 64)) + 1024 + kWgradPartBytes + 256;
    }
    static TrainScratch carve(char *base, int64_t rows)
    {
        TrainScratch t;
        size_t off = 0;
        auto take = [&](size_t b) { size_t o = off; off = align_up(off + b, 256); return base + o; };
        t.part = reinterpret_cast<float *>(take(kWgradPartBytes));
        t.out = reinterpret_cast<float *>(take(size_t(rows) * 64));
        t.H1 = reinterpret_cast<__nv_bfloat16 *>(take(size_t(rows) * 128));
        t.H2 = reinterpret_cast<__nv_bfloat16 *>(take(size_t(rows) * 128));
        t.dOut = reinterpret_cast<__nv_bfloat16 *>(take(size_t(rows) * 32));
        t.dZ1 = reinterpret_cast<__nv_bfloat16 *>(take(size_t(rows) * 128));
        t.dZ2 = reinterpret_cast<__nv_bfloat16 *>(take(size_t(rows) * 128));
        return t;
    }
};

// one gradient evaluation: forward, loss, backward through the activations, weight grads
pond_status mlp_grad_launch(const float *prm, const float *x, int ldx, const float *y, int ldy, int64_t n,
                            const TrainScratch &t, float *grad, float *loss, unsigned int *err, cudaStream_t st)
{
    namespace M = pond::mlp;
    const unsigned tiles = unsigned((n + M::kRows - 1) / M::kRows);
    M::tile_kernel<<<tiles, M::kThreads, M::kTileSmem, st>>>(prm, x, ldx, y, ldy, n, t.out, t.H1, t.H2, t.dOut, t.dZ1,
                                                               t.dZ2, loss, err);
    const int nsplit = M::wgrad_splits(n);
    M::wgrad_kernel<<<dim3(3, unsigned(nsplit)), M::kThreads, 0, st>>>(x, ldx, t.H1, t.H2, t.dOut, t.dZ1, t.dZ2, n, t.part,
                                                                          err);
    M::wgrad_reduce_kernel<<<(M::kParams + 255) / 256, 256, 0, st>>>(t.part, nsplit, grad, err);
    CUDA_TRY(cudaGetLastError());
    return POND_OK;
}

__device__ unsigned int g_standalone_err;
__device__ unsigned int g_wait_check_err;

// One CTA waits on an mbarrier that nothing arrives on, through the same bounded poll as the
// tensor-core kernels, and records that the bound expired.
__global__ void wait_timeout_check_kernel(long long polls, unsigned int *err)
{
    __shared__ __align__(8) uint64_t mbar;
    if (threadIdx.x == 0) pond::tc::mbar_init(&mbar, 1);
    __syncthreads();
    const bool ok = pond::tc::mbar_wait(&mbar, 0u, polls);
    if (!ok && threadIdx.x == 0) atomicOr(err, 1u);
}

}  // namespace

extern "C" {

pond_status pond_gauge_collect(pond_state *s, int64_t n_steps, float *pairs, int64_t cap, int every, int64_t *n_out)
{
    if (pond_status st = check_gauge(s)) return st;
    if (!pairs || cap <= 0 || every < 1 || n_steps < 0) return fail(POND_ERR_INVALID_ARG, "bad collect arguments");
    return s->prec == POND_FP32 ? gauge_collect_impl<float>(s, n_steps, pairs, cap, every, n_out)
                                : gauge_collect_impl<double>(s, n_steps, pairs, cap, every, n_out);
}

pond_status pond_gauge_train(pond_state *s, const float *pairs, int64_t n, int epochs, int batch, float lr, float *loss_out)
{
    namespace M = pond::mlp;
    if (pond_status st = check_gauge(s)) return st;
    if (!pairs || n <= 0 || epochs < 1 || batch < 1 || !(lr > 0.f)) return fail(POND_ERR_INVALID_ARG, "bad train arguments");
    if (s->train_rows < batch) {
        dev_free(s, s->train_scratch);
        s->train_scratch = static_cast<char *>(dev_alloc(s, TrainScratch::bytes(batch)));
        if (!s->train_scratch) return fail(POND_ERR_OOM, "training scratch allocation failed");
        s->train_rows = batch;
    }
    CUDA_TRY(cudaFuncSetAttribute(M::tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, M::kTileSmem));
    const TrainScratch t = TrainScratch::carve(s->train_scratch, batch);
    CUDA_TRY(cudaMemsetAsync(s->mlp_err, 0, sizeof(unsigned int), s->stream));
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int ep = 0; ep < epochs; ++ep) {
        CUDA_TRY(cudaMemsetAsync(s->mlp_loss, 0, sizeof(float), s->stream));
        int64_t nb = 0;
        for (int64_t b0 = 0; b0 < n; b0 += batch, ++nb) {
            const int64_t rows = std::min<int64_t>(batch, n - b0);
            const float *xb = pairs + b0 * M::kPairStride;
            pond_status st = mlp_grad_launch(s->mlp, xb, M::kPairStride, xb, M::kPairStride, rows, t, s->mlp_grad,
                                             s->mlp_loss, s->mlp_err, s->stream);
            if (st != POND_OK) return st;
            ++s->adam_t;
            const float bc1 = 1.f - std::pow(b1, float(s->adam_t)), bc2 = 1.f - std::pow(b2, float(s->adam_t));
            M::adam_kernel<<<(M::kParams + 255) / 256, 256, 0, s->stream>>>(s->mlp, s->mlp_grad, s->mlp_m, s->mlp_v, lr, b1,
                                                                             b2, eps, bc1, bc2);
            s->launches += 4;   // tile, weight-gradient, reduction and Adam kernels
        }
        CUDA_TRY(cudaGetLastError());
        float l = 0.f;
        CUDA_TRY(cudaMemcpyAsync(&l, s->mlp_loss, sizeof(float), cudaMemcpyDeviceToHost, s->stream));
        CUDA_TRY(cudaStreamSynchronize(s->stream));
        if (loss_out) loss_out[ep] = l / float(nb);
    }
    unsigned int err = 0;
    CUDA_TRY(cudaMemcpy(&err, s->mlp_err, sizeof(err), cudaMemcpyDeviceToHost));
    if (err) return fail(POND_ERR_TIMEOUT, "a tensor-core wait timed out during training");
    return POND_OK;
}

pond_status pond_gauge_enable(pond_state *s, int on)
{
    if (pond_status st = check_gauge(s)) return st;
    if (on && s->equilibrate) return fail(POND_ERR_UNSUPPORTED, "the learned predictor runs with Grad's projection only");
    if (bool(on) != s->learned) {
        // the captured step graph depends on the set of kernels
        drop_graph(s);
    }
    s->learned = on != 0;
    if (s->prec == POND_FP32) params_of<2, float>(s).use_learned = s->learned;
    else params_of<2, double>(s).use_learned = s->learned;
    return POND_OK;
}

pond_status pond_set_equilibration(pond_state *s, int on)
{
    if (pond_status st = check_state(s)) return st;
    if (s->batch || s->D == 3 || s->scheme == POND_SL || s->learned)
        return fail(POND_ERR_UNSUPPORTED, "the equilibration alternative runs on finite-volume D1Q4 and D2Q16 grids "
                                          "without the learned predictor");
    if (bool(on) != s->equilibrate) drop_graph(s);   // the captured graph depends on the kernels
    s->equilibrate = on != 0;
    const int eq = s->equilibrate ? 1 : 0;
    if (s->D == 1) {
        if (s->prec == POND_FP32) params_of<1, float>(s).equilibrate = eq;
        else params_of<1, double>(s).equilibrate = eq;
    } else {
        if (s->prec == POND_FP32) params_of<2, float>(s).equilibrate = eq;
        else params_of<2, double>(s).equilibrate = eq;
    }
    return POND_OK;
}

pond_status pond_gauge_set_gate(pond_state *s, float gate)
{
    if (pond_status st = check_gauge(s)) return st;
    if (!(gate >= 0.f)) return fail(POND_ERR_INVALID_ARG, "gate must be >= 0");
    if (s->prec == POND_FP32) params_of<2, float>(s).gauge_gate = gate;
    else params_of<2, double>(s).gauge_gate = gate;
    drop_graph(s);
    return POND_OK;
}

pond_status pond_gauge_set_trust(pond_state *s, float trust)
{
    if (pond_status st = check_gauge(s)) return st;
    if (!(trust > 0.f)) return fail(POND_ERR_INVALID_ARG, "trust must be > 0");
    if (s->prec == POND_FP32) params_of<2, float>(s).gauge_trust = trust;
    else params_of<2, double>(s).gauge_trust = trust;
    drop_graph(s);
    return POND_OK;
}

pond_status pond_gauge_set_params(pond_state *s, const float *params)
{
    if (pond_status st = check_gauge(s)) return st;
    if (!params) return fail(POND_ERR_INVALID_ARG, "params is NULL");
    CUDA_TRY(cudaMemcpyAsync(s->mlp, params, 4 * pond::mlp::kParams, cudaMemcpyHostToDevice, s->stream));
    CUDA_TRY(cudaMemsetAsync(s->mlp_m, 0, 4 * pond::mlp::kParams, s->stream));
    CUDA_TRY(cudaMemsetAsync(s->mlp_v, 0, 4 * pond::mlp::kParams, s->stream));
    s->adam_t = 0;
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    return POND_OK;
}

pond_status pond_gauge_save(pond_state *s, void *buf, size_t *size)
{
    if (pond_status st = check_gauge(s)) return st;
    if (!size) return fail(POND_ERR_INVALID_ARG, "size is NULL");
    const size_t need = 16 + 4 * size_t(pond::mlp::kParams);
    const size_t have = *size;
    *size = need;
    if (!buf || have < need) return POND_OK;
    unsigned char *b = static_cast<unsigned char *>(buf);
    const uint32_t hdr[4] = {0x444E4F50u /* "POND" */, 1u, uint32_t(pond::mlp::kParams), 0u};
    std::memcpy(b, hdr, 16);
    CUDA_TRY(cudaMemcpyAsync(b + 16, s->mlp, 4 * pond::mlp::kParams, cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    return POND_OK;
}

pond_status pond_gauge_load(pond_state *s, const void *buf, size_t size)
{
    if (pond_status st = check_gauge(s)) return st;
    if (!buf || size < 16 + 4 * size_t(pond::mlp::kParams)) return fail(POND_ERR_INVALID_ARG, "blob too small");
    uint32_t hdr[4];
    std::memcpy(hdr, buf, 16);
    if (hdr[0] != 0x444E4F50u || hdr[1] != 1u || hdr[2] != uint32_t(pond::mlp::kParams))
        return fail(POND_ERR_INVALID_ARG, "not a predictor blob of this version");
    return pond_gauge_set_params(s, reinterpret_cast<const float *>(static_cast<const unsigned char *>(buf) + 16));
}

pond_status pond_gauge_get_params(pond_state *s, float *params)
{
    if (pond_status st = check_gauge(s)) return st;
    if (!params) return fail(POND_ERR_INVALID_ARG, "params is NULL");
    CUDA_TRY(cudaMemcpyAsync(params, s->mlp, 4 * pond::mlp::kParams, cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    return POND_OK;
}

pond_status pond_wait_timeout_check(int64_t polls, void *stream)
{
    if (polls < 1 || polls > (int64_t(1) << 24)) return fail(POND_ERR_INVALID_ARG, "polls must be in [1, 2^24]");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned int *err = nullptr;
    CUDA_TRY(cudaGetSymbolAddress(reinterpret_cast<void **>(&err), g_wait_check_err));
    CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(unsigned int), st));
    wait_timeout_check_kernel<<<1, 32, 0, st>>>(polls, err);
    CUDA_TRY(cudaGetLastError());
    unsigned int e = 0;
    CUDA_TRY(cudaMemcpyAsync(&e, err, sizeof(e), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (e) return fail(POND_ERR_TIMEOUT, "the bounded wait expired after %lld polls", (long long)polls);
    return POND_OK;
}

pond_status pond_mlp_forward(const float *params, const float *x, int ldx, int64_t n, float *out, void *stream)
{
    namespace M = pond::mlp;
    if (!params || !x || !out || n <= 0 || ldx < M::kIn) return fail(POND_ERR_INVALID_ARG, "bad forward arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CUDA_TRY(cudaFuncSetAttribute(M::tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, M::kTileSmem));
    unsigned int *err = nullptr;
    CUDA_TRY(cudaGetSymbolAddress(reinterpret_cast<void **>(&err), g_standalone_err));
    CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(unsigned int), st));
    M::tile_kernel<<<unsigned((n + M::kRows - 1) / M::kRows), M::kThreads, M::kTileSmem, st>>>(
        params, x, ldx, nullptr, 0, n, out, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, err);
    CUDA_TRY(cudaGetLastError());
    unsigned int e = 0;
    CUDA_TRY(cudaMemcpyAsync(&e, err, sizeof(e), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (e) return fail(POND_ERR_TIMEOUT, "a tensor-core wait timed out");
    return POND_OK;
}

pond_status pond_mlp_gradient(const float *params, const float *x, int ldx, const float *y, int ldy, int64_t n, float *grad,
                              float *loss, void *stream)
{
    namespace M = pond::mlp;
    if (!params || !x || !y || !grad || !loss || n <= 0 || ldx < M::kIn || ldy < M::kIn + M::kOut)
        return fail(POND_ERR_INVALID_ARG, "bad gradient arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CUDA_TRY(cudaFuncSetAttribute(M::tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, M::kTileSmem));
    char *scratch = nullptr;
    CUDA_TRY(cudaMalloc(&scratch, TrainScratch::bytes(n)));
    unsigned int *err = nullptr;
    pond_status r = POND_OK;
    cudaError_t ce = cudaGetSymbolAddress(reinterpret_cast<void **>(&err), g_standalone_err);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(err, 0, sizeof(unsigned int), st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(loss, 0, sizeof(float), st);
    if (ce != cudaSuccess) r = fail(POND_ERR_CUDA, "%s", cudaGetErrorString(ce));
    if (r == POND_OK) r = mlp_grad_launch(params, x, ldx, y, ldy, n, TrainScratch::carve(scratch, n), grad, loss, err, st);
    unsigned int e = 0;
    if (r == POND_OK) {
        ce = cudaMemcpyAsync(&e, err, sizeof(e), cudaMemcpyDeviceToHost, st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
        if (ce != cudaSuccess) r = fail(POND_ERR_CUDA, "%s", cudaGetErrorString(ce));
        else if (e) r = fail(POND_ERR_TIMEOUT, "a tensor-core wait timed out");
    }
    cudaStreamSynchronize(st);
    cudaFree(scratch);
    return r;
}

}  // extern "C"

// ---------------------------------------------------------- allocation-free gradient

namespace {

// Scratch of pond_mlp_gradient_noalloc: the activations of up to POND_MLP_NOALLOC_MAX_ROWS
// rows, followed by the error word.  In host code this name only stands for the symbol;
// its device address comes from cudaGetSymbolAddress for the current device.
constexpr size_t kNoallocScratch = align_up(TrainScratch::bytes(POND_MLP_NOALLOC_MAX_ROWS), 256) + 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratch];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
bool g_noalloc_ready[kMaxDevices] = {};

// With the caller's device current: the array's device address in the current context
// (looked up on every call, which allocates nothing, so a context created after a device
// reset gets its own address) and, once per device, the tile kernel's shared-memory limit.
pond_status noalloc_setup(unsigned char **out)
{
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(POND_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
    void *p = nullptr;
    CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ready[dev]) {
        CUDA_TRY(cudaFuncSetAttribute(pond::mlp::tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, pond::mlp::kTileSmem));
        g_noalloc_ready[dev] = true;
    }
    *out = static_cast<unsigned char *>(p);
    return POND_OK;
}

}  // namespace

extern "C" {

pond_status pond_mlp_gradient_noalloc(const float *params, const float *x, int ldx, const float *y, int ldy, int64_t n,
                                      float *grad, float *loss, void *stream)
{
    namespace M = pond::mlp;
    if (!params || !x || !y || !grad || !loss || n <= 0 || ldx < M::kIn || ldy < M::kIn + M::kOut)
        return fail(POND_ERR_INVALID_ARG, "bad gradient arguments");
    if (n > POND_MLP_NOALLOC_MAX_ROWS)
        return fail(POND_ERR_INVALID_ARG, "n = %lld rows exceeds the allocation-free limit of %d rows", (long long)n,
                    POND_MLP_NOALLOC_MAX_ROWS);
    unsigned char *base = nullptr;
    if (pond_status st = noalloc_setup(&base)) return st;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const TrainScratch t = TrainScratch::carve(reinterpret_cast<char *>(base), POND_MLP_NOALLOC_MAX_ROWS);
    unsigned int *err = reinterpret_cast<unsigned int *>(base + kNoallocScratch - 256);
    // the loss accumulates and the error word is or-ed into: both start at zero
    CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(unsigned int), st));
    CUDA_TRY(cudaMemsetAsync(loss, 0, sizeof(float), st));
    pond_status r = mlp_grad_launch(params, x, ldx, y, ldy, n, t, grad, loss, err, st);
    if (r != POND_OK) return r;
    unsigned int e = 0;
    CUDA_TRY(cudaMemcpyAsync(&e, err, sizeof(e), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (e) return fail(POND_ERR_TIMEOUT, "a tensor-core wait timed out");
    return POND_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ autotuner
//
// Each step kernel exists in several compiled variants (pond_launch.cuh).  The tuner times
// them on the state's own data: the device block is copied aside, every variant runs from
// that copy (so all see the same state and the same corrector work), and the copy is put
// back at the end, so tuning leaves the solution untouched.  The face variants are timed
// with the cell kernel fixed, then the cell variants with the chosen face kernel.  Choices
// can be kept in a cache file of lines "key<TAB>face cell tube", the key naming the device,
// the problem kind and its size.

namespace {

std::string tune_key(const pond_state *s)
{
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, s->device);
    char buf[512];
    if (s->batch)
        std::snprintf(buf, sizeof(buf), "%s|sm%d|tubes|%s|%lld|%lld", prop.name, prop.multiProcessorCount,
                      s->prec == POND_FP32 ? "fp32" : "fp64", (long long)s->n_tubes, (long long)s->ncell);
    else if (s->D == 3)
        std::snprintf(buf, sizeof(buf), "%s|sm%d|D3|%s|%lldx%lldx%lld", prop.name, prop.multiProcessorCount,
                      s->prec == POND_FP32 ? "fp32" : "fp64", (long long)s->grid3.nx, (long long)s->grid3.ny,
                      (long long)s->grid3.nz);
    else
        std::snprintf(buf, sizeof(buf), "%s|sm%d|D%d|%s|%lldx%lld|learned%d", prop.name, prop.multiProcessorCount, s->D,
                      s->prec == POND_FP32 ? "fp32" : "fp64", (long long)s->grid.nx, (long long)s->grid.ny,
                      s->learned ? 1 : 0);
    for (char *c = buf; *c; ++c)
        if (*c == '\t' || *c == '\n') *c = ' ';
    return buf;
}

// the last entry for key in the cache file; false if there is none
bool cache_lookup(const char *path, const std::string &key, int v[3])
{
    FILE *f = path ? std::fopen(path, "r") : nullptr;
    if (!f) return false;
    bool found = false;
    char line[1024];
    while (std::fgets(line, sizeof(line), f)) {
        char *tab = std::strchr(line, '\t');
        if (!tab) continue;
        *tab = '\0';
        int a = 0, b = 0, c = 0;
        if (key == line && std::sscanf(tab + 1, "%d %d %d", &a, &b, &c) == 3) {
            v[0] = a; v[1] = b; v[2] = c;
            found = true;
        }
    }
    std::fclose(f);
    return found;
}

void cache_store(const char *path, const std::string &key, const int v[3])
{
    FILE *f = path ? std::fopen(path, "a") : nullptr;
    if (!f) return;
    std::fprintf(f, "%s\t%d %d %d\n", key.c_str(), v[0], v[1], v[2]);
    std::fclose(f);
}

int grid_face_variants(const pond_state *s)
{
    if (s->D == 2) return s->prec == POND_FP32 ? pond::face_variants<2, float>() : pond::face_variants<2, double>();
    return s->prec == POND_FP32 ? pond::face_variants<1, float>() : pond::face_variants<1, double>();
}

// the whole-step choices of a grid: the separate face and cell kernels, then each fused variant
int grid_step_variants(const pond_state *s)
{
    if (s->D == 2) return 1 + (s->prec == POND_FP32 ? pond::step_variants<2, float>() : pond::step_variants<2, double>());
    return 1 + (s->prec == POND_FP32 ? pond::step_variants<1, float>() : pond::step_variants<1, double>());
}

int variant_total(const pond_state *s)
{
    if (s->D == 3) return pond::face3_variant_count + pond::cell3_variant_count;
    if (s->scheme == POND_SL) return 0;
    if (s->batch) return s->prec == POND_FP32 ? pond::tube_variants<float>() : pond::tube_variants<double>();
    return grid_face_variants(s) + pond::kCellVariants + grid_step_variants(s);
}

// mean ms per launch of the face (which = 0) or cell (which = 1) kernel over `steps` steps
// after one untimed step, starting from the saved block
template <int D, typename R>
pond_status time_grid_variant(pond_state *s, const char *saved, int steps, int which, double *ms)
{
    auto &P = params_of<D, R>(s);
    CUDA_TRY(cudaMemcpyAsync(s->base, saved, s->bytes, cudaMemcpyDeviceToDevice, s->stream));
    launch_step<D, R>(s);
    Events ev(size_t(2 * steps));
    CUDA_TRY(ev.create());
    for (int k = 0; k < steps; ++k) {
        if constexpr (D == 2) {
            if (s->learned)
                pond::gauge_predict_kernel<R><<<predict_blocks(s), pond::mlp::kThreads, pond::mlp::kInferSmem, s->stream>>>(P);
        }
        if (which == 0) CUDA_TRY(cudaEventRecord(ev[2 * k], s->stream));
        pond::launch_face<D, R>(s->face_v, false, P, s->stream);
        if (which == 0) CUDA_TRY(cudaEventRecord(ev[2 * k + 1], s->stream));
        if (which == 1) CUDA_TRY(cudaEventRecord(ev[2 * k], s->stream));
        pond::launch_cell_any<D, R>(s->cell_v, P, s->stream);
        if (which == 1) CUDA_TRY(cudaEventRecord(ev[2 * k + 1], s->stream));
    }
    s->launches += int64_t(steps + 1) * (2 + ((D == 2 && s->learned) ? 1 : 0));
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaEventSynchronize(ev.back()));
    double sum = 0.0;
    for (int k = 0; k < steps; ++k) {
        float a = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&a, ev[2 * k], ev[2 * k + 1]));
        sum += a;
    }
    *ms = sum / steps;
    return POND_OK;
}

// mean ms per whole step (face and cell kernels, or one fused kernel) over `steps` steps after
// one untimed step, starting from the saved block and the saved buffer assignment
template <int D, typename R>
pond_status time_grid_step(pond_state *s, const char *saved, const pond::Params<D, R> &P0, int parity0, int steps,
                           double *ms)
{
    auto &P = params_of<D, R>(s);
    CUDA_TRY(cudaMemcpyAsync(s->base, saved, s->bytes, cudaMemcpyDeviceToDevice, s->stream));
    P = P0;
    s->sl_parity = parity0;
    launch_step<D, R>(s);
    Events ev(2);
    CUDA_TRY(ev.create());
    CUDA_TRY(cudaEventRecord(ev[0], s->stream));
    for (int k = 0; k < steps; ++k) launch_step<D, R>(s);
    CUDA_TRY(cudaEventRecord(ev[1], s->stream));
    s->launches += int64_t(steps + 1) * (fused_step<D, R>(s, false) ? 1 : 2);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaEventSynchronize(ev[1]));
    float a = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&a, ev[0], ev[1]));
    *ms = double(a) / steps;
    P = P0;
    s->sl_parity = parity0;
    return POND_OK;
}

template <int D, typename R>
pond_status tune_grid(pond_state *s, const char *saved, int steps, pond_tune_result *res)
{
    const pond::Params<D, R> P0 = params_of<D, R>(s);
    const int parity0 = s->sl_parity;
    s->tube_v = 0;   // face and cell variants are timed as separate kernels
    const int nf = pond::face_variants<D, R>();
    double best = 0.0;
    int bf = 0;
    for (int v = 0; v < nf; ++v) {
        s->face_v = v;
        double ms = 0.0;
        if (pond_status st = time_grid_variant<D, R>(s, saved, steps, 0, &ms)) return st;
        if (res && res->n < POND_TUNE_MAX) res->ms[res->n++] = ms;
        if (v == 0 || ms < best) { best = ms; bf = v; }
    }
    s->face_v = bf;
    int bc = 0;
    for (int v = 0; v < pond::kCellVariants; ++v) {
        s->cell_v = v;
        double ms = 0.0;
        if (pond_status st = time_grid_variant<D, R>(s, saved, steps, 1, &ms)) return st;
        if (res && res->n < POND_TUNE_MAX) res->ms[res->n++] = ms;
        if (v == 0 || ms < best) { best = ms; bc = v; }
    }
    s->cell_v = bc;
    // whole steps: the chosen face and cell kernels against every fused variant
    int bs = 0;
    if (s->scheme == POND_FV && !s->learned && !s->equilibrate) {
        double best_step = 0.0;
        for (int v = 0; v <= pond::step_variants<D, R>(); ++v) {
            s->tube_v = v;
            double ms = 0.0;
            if (pond_status st = time_grid_step<D, R>(s, saved, P0, parity0, steps, &ms)) return st;
            if (res && res->n < POND_TUNE_MAX) res->ms[res->n++] = ms;
            if (v == 0 || ms < best_step) { best_step = ms; bs = v; }
        }
    }
    s->tube_v = bs;
    params_of<D, R>(s) = P0;
    s->sl_parity = parity0;
    return POND_OK;
}

template <typename R>
pond_status tune_batch(pond_state *s, const char *saved, int steps, pond_tune_result *res)
{
    auto &P = tparams_of<R>(s);
    const int nv = pond::tube_variants<R>();
    double best = 0.0;
    int bv = 0;
    Events ev(2);
    CUDA_TRY(ev.create());
    cudaEvent_t e0 = ev[0], e1 = ev[1];
    for (int v = 0; v < nv; ++v) {
        CUDA_TRY(cudaMemcpyAsync(s->base, saved, s->bytes, cudaMemcpyDeviceToDevice, s->stream));
        CUDA_TRY(cudaEventRecord(e0, s->stream));
        pond::launch_tube<R>(v, unsigned(s->n_tubes), P, steps, s->cur, s->stream);
        CUDA_TRY(cudaEventRecord(e1, s->stream));
        s->launches += 1;
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaEventSynchronize(e1));
        float a = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&a, e0, e1));
        if (res && res->n < POND_TUNE_MAX) res->ms[res->n++] = a / steps;
        if (v == 0 || a < best) { best = a; bv = v; }
    }
    s->tube_v = bv;
    return POND_OK;
}

// D3Q64 grids: every face tile variant with the current cell kernel, then every cell block
// variant with the chosen face kernel, each timed from the saved block
template <typename R>
pond_status time_3d_variant(pond_state *s, const char *saved, int steps, int which, double *ms)
{
    auto &P = params3_of<R>(s);
    CUDA_TRY(cudaMemcpyAsync(s->base, saved, s->bytes, cudaMemcpyDeviceToDevice, s->stream));
    launch_step3<R>(s);
    Events ev(size_t(2 * steps));
    CUDA_TRY(ev.create());
    for (int k = 0; k < steps; ++k) {
        if (which == 0) CUDA_TRY(cudaEventRecord(ev[2 * k], s->stream));
        pond::launch_face3<R>(s->face_v, P, s->stream);
        if (which == 0) CUDA_TRY(cudaEventRecord(ev[2 * k + 1], s->stream));
        if (which == 1) CUDA_TRY(cudaEventRecord(ev[2 * k], s->stream));
        pond::launch_cell3<R>(s->cell_v, P, s->stream);
        if (which == 1) CUDA_TRY(cudaEventRecord(ev[2 * k + 1], s->stream));
    }
    s->launches += int64_t(steps + 1) * 2;
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaEventSynchronize(ev.back()));
    double sum = 0.0;
    for (int k = 0; k < steps; ++k) {
        float a = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&a, ev[2 * k], ev[2 * k + 1]));
        sum += a;
    }
    *ms = sum / steps;
    return POND_OK;
}

template <typename R>
pond_status tune_3d(pond_state *s, const char *saved, int steps, pond_tune_result *res)
{
    double best = 0.0;
    int bf = 0, bc = 0;
    for (int v = 0; v < pond::face3_variant_count; ++v) {
        s->face_v = v;
        double ms = 0.0;
        if (pond_status st = time_3d_variant<R>(s, saved, steps, 0, &ms)) return st;
        if (res && res->n < POND_TUNE_MAX) res->ms[res->n++] = ms;
        if (v == 0 || ms < best) { best = ms; bf = v; }
    }
    s->face_v = bf;
    for (int v = 0; v < pond::cell3_variant_count; ++v) {
        s->cell_v = v;
        double ms = 0.0;
        if (pond_status st = time_3d_variant<R>(s, saved, steps, 1, &ms)) return st;
        if (res && res->n < POND_TUNE_MAX) res->ms[res->n++] = ms;
        if (v == 0 || ms < best) { best = ms; bc = v; }
    }
    s->cell_v = bc;
    s->tube_v = 0;
    return POND_OK;
}

}  // namespace

extern "C" {

pond_status pond_autotune(pond_state *s, int steps, const char *cache_path, pond_tune_result *out)
{
    if (pond_status st = check_state(s)) return st;
    if (steps < 1) return fail(POND_ERR_INVALID_ARG, "steps must be at least 1");
    pond_tune_result res{};
    if (s->D != 3 && (s->scheme == POND_SL || s->equilibrate)) {  // one compiled variant: nothing to choose
        if (out) *out = res;
        return POND_OK;
    }
    const std::string key = tune_key(s);
    int v[3] = {0, 0, 0};
    if (cache_lookup(cache_path, key, v) && pond_set_variants(s, v[0], v[1], v[2]) == POND_OK) {
        res.from_cache = 1;
    } else {
        CUDA_TRY(cudaStreamSynchronize(s->stream));
        char *saved = static_cast<char *>(dev_alloc(s, s->bytes));
        if (!saved) return fail(POND_ERR_OOM, "device allocation of %zu bytes for the tuning copy failed", s->bytes);
        pond_status st = POND_OK;
        if (cudaMemcpyAsync(saved, s->base, s->bytes, cudaMemcpyDeviceToDevice, s->stream) != cudaSuccess)
            st = fail(POND_ERR_CUDA, "saving the state for tuning failed");
        if (st == POND_OK) {
            if (s->batch) st = dispatch_batch(s, [&](auto r) { return tune_batch<decltype(r)>(s, saved, steps, &res); });
            else if (s->D == 3)
                st = s->prec == POND_FP32 ? tune_3d<float>(s, saved, steps, &res) : tune_3d<double>(s, saved, steps, &res);
            else st = dispatch(s, [&](auto d, auto r) { return tune_grid<decltype(d)::value, decltype(r)>(s, saved, steps, &res); });
        }
        // put the state back whatever happened, then release the copy
        const cudaError_t e1 = cudaMemcpyAsync(s->base, saved, s->bytes, cudaMemcpyDeviceToDevice, s->stream);
        const cudaError_t e2 = cudaStreamSynchronize(s->stream);
        dev_free(s, saved);
        if (st != POND_OK) return st;
        if (e1 != cudaSuccess || e2 != cudaSuccess) return fail(POND_ERR_CUDA, "restoring the state after tuning failed");
        v[0] = s->face_v; v[1] = s->cell_v; v[2] = s->tube_v;
        cache_store(cache_path, key, v);
    }
    drop_graph(s);
    res.face = s->face_v;
    res.cell = s->cell_v;
    res.tube = s->tube_v;
    if (out) *out = res;
    return POND_OK;
}

int pond_variant_count(const pond_state *s) { return s ? variant_total(s) : 0; }

const char *pond_variant_name(const pond_state *s, int i)
{
    thread_local char buf[128];
    buf[0] = '\0';
    if (!s || i < 0 || i >= variant_total(s)) return buf;
    const bool f32 = s->prec == POND_FP32;
    if (s->batch) {
        if (f32) pond::tube_name<float>(i, buf, sizeof(buf));
        else pond::tube_name<double>(i, buf, sizeof(buf));
        return buf;
    }
    if (s->D == 3) {
        if (i >= pond::face3_variant_count) pond::cell3_name(i - pond::face3_variant_count, buf, sizeof(buf));
        else if (f32) pond::face3_name<float>(i, buf, sizeof(buf));
        else pond::face3_name<double>(i, buf, sizeof(buf));
        return buf;
    }
    const int nf = grid_face_variants(s);
    if (i >= nf + pond::kCellVariants) {
        const int k = i - nf - pond::kCellVariants;
        if (k == 0) std::snprintf(buf, sizeof(buf), "step face and cell kernels");
        else if (s->D == 2 && f32) pond::StepNames<2, float, pond::StepList<2, float>::type>::name(k - 1, buf, sizeof(buf));
        else if (s->D == 2) pond::StepNames<2, double, pond::StepList<2, double>::type>::name(k - 1, buf, sizeof(buf));
        else if (f32) pond::StepNames<1, float, pond::StepList<1, float>::type>::name(k - 1, buf, sizeof(buf));
        else pond::StepNames<1, double, pond::StepList<1, double>::type>::name(k - 1, buf, sizeof(buf));
    } else if (i >= nf) {
        pond::cell_name(i - nf, buf, sizeof(buf));
    } else if (s->D == 2) {
        if (f32) pond::FaceNames<2, float, pond::FaceList<2, float>::type>::name(i, buf, sizeof(buf));
        else pond::FaceNames<2, double, pond::FaceList<2, double>::type>::name(i, buf, sizeof(buf));
    } else {
        if (f32) pond::FaceNames<1, float, pond::FaceList<1, float>::type>::name(i, buf, sizeof(buf));
        else pond::FaceNames<1, double, pond::FaceList<1, double>::type>::name(i, buf, sizeof(buf));
    }
    return buf;
}

pond_status pond_set_variants(pond_state *s, int face, int cell, int tube)
{
    if (pond_status st = check_state(s)) return st;
    if (s->batch) {
        const int nv = s->prec == POND_FP32 ? pond::tube_variants<float>() : pond::tube_variants<double>();
        if (tube < 0 || tube >= nv) return fail(POND_ERR_INVALID_ARG, "tube variant %d out of range", tube);
        s->tube_v = tube;
    } else if (s->D == 3) {
        if (face < 0 || face >= pond::face3_variant_count || cell < 0 || cell >= pond::cell3_variant_count || tube != 0)
            return fail(POND_ERR_INVALID_ARG, "D3Q64 face/cell variant (%d, %d, %d) out of range", face, cell, tube);
        s->face_v = face;
        s->cell_v = cell;
        s->tube_v = 0;
    } else {
        const int nf = grid_face_variants(s);
        if (face < 0 || face >= nf || cell < 0 || cell >= pond::kCellVariants)
            return fail(POND_ERR_INVALID_ARG, "face/cell variant (%d, %d) out of range", face, cell);
        if (tube < 0 || tube >= grid_step_variants(s) || (tube > 0 && s->scheme != POND_FV))
            return fail(POND_ERR_INVALID_ARG, "step variant %d out of range", tube);
        s->face_v = face;
        s->cell_v = cell;
        s->tube_v = tube;
    }
    drop_graph(s);
    return POND_OK;
}

int64_t pond_launch_count(const pond_state *s) { return s ? s->launches : 0; }

void pond_destroy(pond_state *s)
{
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    drop_graph(s);
    dev_free(s, s->base);
    dev_free(s, s->mlp_block);
    dev_free(s, s->train_scratch);
    if (s->own_stream) cudaStreamDestroy(s->stream);
    delete s;
}

const char *pond_last_error(void) { return g_err; }

}  // extern "C"
