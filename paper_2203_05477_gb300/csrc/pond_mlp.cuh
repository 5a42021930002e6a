// pond_mlp.cuh -- learned face-gauge predictor: a small MLP on the 5th-generation tensor cores.
//
// The corrector of Sec. III.B.3 starts each face from the previous half step's frame.
// This network predicts the converged frame from the face stencil, so the corrector starts
// nearer its fixed point; the corrector and its convergence test are unchanged and remain
// the judge of the result.
//
// Network: 48 (34 used) features -> 64 -> 64 -> 16 (3 used), ReLU, BF16 operands on the
// tensor cores (tcgen05.mma kind::f16) with FP32 accumulation in tensor memory; biases and
// activations on the CUDA cores in FP32.  Parameters (FP32 master copy, 8336 floats):
//   W1 [64][48] | b1 [64] | W2 [64][64] | b2 [64] | W3 [16][64] | b3 [16]
// Features of a face (normal n, tangent t, predictor frame (u_p, T_p)), for the eight
// stencil slots LL, L, R, RR, L-t, L+t, R-t, R+t:
//   log(rho_s / rho_LR), (u_s,n - u_p,n)/sqrt(T_p), (u_s,t - u_p,t)/sqrt(T_p), log(T_s/T_p)
// with rho_LR the mean density of L and R, then h sqrt(T_p)/dx_n and 1; all clipped to
// [-20, 20].  Targets: (u_b,n - u_p,n)/sqrt(T_p), (u_b,t - u_p,t)/sqrt(T_p), log(T_b/T_p)
// of the converged face frame.
#pragma once

#include "pond_tc.cuh"

namespace pond {
namespace mlp {

constexpr int kIn = 48, kUsed = 34, kHid = 64, kOutP = 16, kOut = 3;
constexpr int oW1 = 0, ob1 = oW1 + kHid * kIn, oW2 = ob1 + kHid, ob2 = oW2 + kHid * kHid, oW3 = ob2 + kHid,
              ob3 = oW3 + kOutP * kHid, kParams = ob3 + kOutP;
constexpr int kRows = 128;         // rows (faces, samples) per CTA: the MMA M
constexpr int kThreads = 128;      // one thread per row
constexpr long long kPolls = 1ll << 22;   // bound on every mbarrier wait
constexpr int kPairStride = 52;    // features (48), targets (3), corrector passes of the face

// shared-memory plan of the tile kernel (byte offsets, 128-aligned)
constexpr int sB1 = 0;                          // W1   [64][48]
constexpr int sB2 = sB1 + kHid * kIn * 2;       // W2   [64][64]
constexpr int sB3 = sB2 + kHid * kHid * 2;      // W3   [16][64]
constexpr int sB4 = sB3 + kOutP * kHid * 2;     // W3^T [64][16]
constexpr int sB5 = sB4 + kHid * kOutP * 2;     // W2^T [64][64]
constexpr int sA1 = sB5 + kHid * kHid * 2;      // X    [128][48]
constexpr int sA2 = sA1 + kRows * kIn * 2;      // H1   [128][64]
constexpr int sA3 = sA2 + kRows * kHid * 2;     // H2   [128][64]
constexpr int sA4 = sA3 + kRows * kHid * 2;     // dOut [128][16]
constexpr int sA5 = sA4 + kRows * kOutP * 2;    // dZ2  [128][64]
constexpr int kTileSmem = sA5 + kRows * kHid * 2;

// shared-memory plan of the inference kernel: weights, one input tile, one hidden tile
// (H1, then H2 over it once the second GEMM has read H1) and the biases in FP32
constexpr int iW1 = 0;                          // W1 [64][48]
constexpr int iW2 = iW1 + kHid * kIn * 2;       // W2 [64][64]
constexpr int iW3 = iW2 + kHid * kHid * 2;      // W3 [16][64]
constexpr int iX = iW3 + kOutP * kHid * 2;      // X  [128][48]
constexpr int iH = iX + kRows * kIn * 2;        // H  [128][64]
constexpr int iBias = iH + kRows * kHid * 2;    // b1 [64], b2 [64], b3 [16]
constexpr int kInferSmem = iBias + (2 * kHid + kOutP) * 4;
constexpr int kInferCtasPerSm = 4;              // 4 x 45.6 KB shared memory, 4 x 64 TMEM columns
constexpr uint32_t kInferTmemCols = 64;

__device__ __forceinline__ void put_bf16(unsigned char *base, uint32_t r, uint32_t k, uint32_t K, float v)
{
    *reinterpret_cast<__nv_bfloat16 *>(base + tc::kmajor_offset(r, k, K)) = __float2bfloat16_rn(v);
}
__device__ __forceinline__ float get_bf16(const unsigned char *base, uint32_t r, uint32_t k, uint32_t K)
{
    return __bfloat162float(*reinterpret_cast<const __nv_bfloat16 *>(base + tc::kmajor_offset(r, k, K)));
}

// 8 consecutive values k0 .. k0+7 (k0 a multiple of 8) of row r: one 16-byte store, since
// they form one row of a core matrix
__device__ __forceinline__ void put_bf16x8(unsigned char *base, uint32_t r, uint32_t k0, uint32_t K, const float *v)
{
    uint4 w;
    uint32_t *u = reinterpret_cast<uint32_t *>(&w);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const __nv_bfloat162 p = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);  // .x (k0 + 2i) at the lower address
        u[i] = *reinterpret_cast<const uint32_t *>(&p);
    }
    *reinterpret_cast<uint4 *>(base + tc::kmajor_offset(r, k0, K)) = w;
}

// weights and biases of the inference kernel
__device__ __forceinline__ void stage_infer(const float *prm, unsigned char *sm)
{
    for (int e = threadIdx.x; e < kHid * kIn; e += blockDim.x) put_bf16(sm + iW1, e / kIn, e % kIn, kIn, prm[oW1 + e]);
    for (int e = threadIdx.x; e < kHid * kHid; e += blockDim.x) put_bf16(sm + iW2, e / kHid, e % kHid, kHid, prm[oW2 + e]);
    for (int e = threadIdx.x; e < kOutP * kHid; e += blockDim.x) put_bf16(sm + iW3, e / kHid, e % kHid, kHid, prm[oW3 + e]);
    float *bias = reinterpret_cast<float *>(sm + iBias);
    for (int e = threadIdx.x; e < kHid; e += blockDim.x) {
        bias[e] = prm[ob1 + e];
        bias[kHid + e] = prm[ob2 + e];
        if (e < kOutP) bias[2 * kHid + e] = prm[ob3 + e];
    }
}

// stage the weights (B operands) of the forward pass and, for training, of the backward pass
__device__ __forceinline__ void stage_weights(const float *prm, unsigned char *sm, bool train)
{
    for (int e = threadIdx.x; e < kHid * kIn; e += blockDim.x) put_bf16(sm + sB1, e / kIn, e % kIn, kIn, prm[oW1 + e]);
    for (int e = threadIdx.x; e < kHid * kHid; e += blockDim.x) put_bf16(sm + sB2, e / kHid, e % kHid, kHid, prm[oW2 + e]);
    for (int e = threadIdx.x; e < kOutP * kHid; e += blockDim.x) put_bf16(sm + sB3, e / kHid, e % kHid, kHid, prm[oW3 + e]);
    if (train) {
        // W3^T: row i (hidden), column o (output); W2^T: row i (input), column o (output)
        for (int e = threadIdx.x; e < kOutP * kHid; e += blockDim.x) {
            const int o = e / kHid, i = e % kHid;
            put_bf16(sm + sB4, i, o, kOutP, prm[oW3 + e]);
        }
        for (int e = threadIdx.x; e < kHid * kHid; e += blockDim.x) {
            const int o = e / kHid, i = e % kHid;
            put_bf16(sm + sB5, i, o, kHid, prm[oW2 + e]);
        }
    }
}

// one GEMM on the tensor cores, waited for by every thread; returns false on time-out
__device__ __forceinline__ bool run_gemm(uint32_t d_tmem, const unsigned char *A, const unsigned char *B, uint32_t K,
                                         uint32_t N, uint64_t *mbar, uint32_t &phase, bool accumulate = false)
{
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (threadIdx.x == 0) {
        tc::gemm_issue(d_tmem, A, B, K, N, accumulate);
        tc::commit(mbar);
    }
    // block-uniform result: every thread takes the same path afterwards
    const bool ok = __syncthreads_and(tc::mbar_wait(mbar, phase, kPolls)) != 0;
    if (ok) phase ^= 1u;
    tc::fence_after_sync();
    return ok;
}

// after a time-out: wait once more (bounded) for the MMA still in flight before the
// tensor memory it writes is released
__device__ __forceinline__ void drain(uint64_t *mbar, uint32_t phase, bool ok)
{
    if (!ok) tc::mbar_wait(mbar, phase, kPolls);
}

// 16*nchunks accumulator columns of this thread's row
__device__ __forceinline__ void read_row(uint32_t tmem, uint32_t col, int nchunks, float *v)
{
    const uint32_t lane = (threadIdx.x & ~31u) << 16;
    for (int c = 0; c < nchunks; ++c) tc::tmem_ld16(tmem + lane + col + 16u * c, v + 16 * c);
}

// Forward pass of the 128 rows staged in iX, accumulators in 64 TMEM columns.  out: this
// thread's row of the output layer (16 values, 3 used).  Returns false on time-out.
__device__ __forceinline__ bool forward_infer(unsigned char *sm, uint32_t tmem, uint64_t *mbar, uint32_t &phase,
                                              float *out)
{
    const uint32_t r = threadIdx.x;
    const uint32_t lane = (threadIdx.x & ~31u) << 16;
    const float *bias = reinterpret_cast<const float *>(sm + iBias);
    float v[kHid];
    for (int layer = 0; layer < 2; ++layer) {
        if (!run_gemm(tmem, sm + (layer ? iH : iX), sm + (layer ? iW2 : iW1), layer ? kHid : kIn, kHid, mbar, phase))
            return false;
        tc::tmem_ld64(tmem + lane, v);
#pragma unroll
        for (int j = 0; j < kHid; ++j) v[j] = fmaxf(v[j] + bias[layer * kHid + j], 0.f);
#pragma unroll
        for (int k0 = 0; k0 < kHid; k0 += 8) put_bf16x8(sm + iH, r, k0, kHid, v + k0);
    }
    if (!run_gemm(tmem, sm + iH, sm + iW3, kHid, kOutP, mbar, phase)) return false;
    tc::tmem_ld16(tmem + lane, out);
#pragma unroll
    for (int j = 0; j < kOutP; ++j) out[j] += bias[2 * kHid + j];
    return true;
}

// Forward pass of the 128 rows staged in sA1 (weights in sB1..sB3).  out: this thread's
// row of the output layer (16 values, 3 used).  h1/h2 (post-ReLU) stay in sA2/sA3.
__device__ __forceinline__ bool forward_tile(const float *prm, unsigned char *sm, uint32_t tmem, uint64_t *mbar,
                                             uint32_t &phase, float *out)
{
    float v[kHid];
    const uint32_t r = threadIdx.x;
    bool ok = run_gemm(tmem, sm + sA1, sm + sB1, kIn, kHid, mbar, phase);
    if (!ok) return false;
    read_row(tmem, 0, 4, v);
#pragma unroll
    for (int j = 0; j < kHid; ++j) put_bf16(sm + sA2, r, j, kHid, fmaxf(v[j] + prm[ob1 + j], 0.f));
    ok = run_gemm(tmem + 64, sm + sA2, sm + sB2, kHid, kHid, mbar, phase);
    if (!ok) return false;
    read_row(tmem, 64, 4, v);
#pragma unroll
    for (int j = 0; j < kHid; ++j) put_bf16(sm + sA3, r, j, kHid, fmaxf(v[j] + prm[ob2 + j], 0.f));
    ok = run_gemm(tmem, sm + sA3, sm + sB3, kHid, kOutP, mbar, phase);
    if (!ok) return false;
    read_row(tmem, 0, 1, v);
#pragma unroll
    for (int j = 0; j < kOutP; ++j) out[j] = v[j] + prm[ob3 + j];
    return ok;
}

// Forward + loss + backward through the activations for 128 training rows.
//   x [n][48] features, y [n][kPairStride] (targets at 48..50), n rows in the batch
//   writes out [n][16], H1, H2 [n][64] (bf16), dOut [n][16] (bf16), dZ1, dZ2 [n][64] (bf16),
//   loss += mean squared error / n.  With y == nullptr only the forward pass runs.
__global__ void __launch_bounds__(kThreads)
tile_kernel(const float *prm, const float *x, int ldx, const float *y, int ldy, long long n, float *out,
            __nv_bfloat16 *H1, __nv_bfloat16 *H2, __nv_bfloat16 *dOut, __nv_bfloat16 *dZ1, __nv_bfloat16 *dZ2,
            float *loss, unsigned int *err)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const bool train = y != nullptr;
    const long long row = (long long)blockIdx.x * kRows + threadIdx.x;
    const bool valid = row < n;
    if (threadIdx.x < 32) tc::tmem_alloc(&tmem_base, 128);
    if (threadIdx.x == 0) tc::mbar_init(&mbar, 1);
    stage_weights(prm, sm, train);
    for (int k = 0; k < kIn; ++k) put_bf16(sm + sA1, threadIdx.x, k, kIn, valid ? x[row * ldx + k] : 0.f);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    uint32_t phase = 0;
    float o[kOutP];
    bool ok = forward_tile(prm, sm, tmem, &mbar, phase, o);
    const uint32_t r = threadIdx.x;
    if (valid && out)
        for (int j = 0; j < kOutP; ++j) out[row * kOutP + j] = o[j];
    if (train && ok) {
        // dL/dout for L = sum (out - y)^2 / (3 n)
        float d[kOutP], l = 0.f;
        for (int j = 0; j < kOutP; ++j) {
            const float e = (valid && j < kOut) ? o[j] - y[row * ldy + kIn + j] : 0.f;
            d[j] = 2.f * e / float(kOut * n);
            l += e * e;
        }
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) l += __shfl_down_sync(0xffffffffu, l, s);
        if ((threadIdx.x & 31) == 0) atomicAdd(loss, l / float(kOut * n));
        for (int j = 0; j < kOutP; ++j) {
            put_bf16(sm + sA4, r, j, kOutP, d[j]);
            if (valid) dOut[row * kOutP + j] = __float2bfloat16_rn(d[j]);
        }
        if (valid)
            for (int j = 0; j < kHid; ++j) {
                H1[row * kHid + j] = __float2bfloat16_rn(get_bf16(sm + sA2, r, j, kHid));
                H2[row * kHid + j] = __float2bfloat16_rn(get_bf16(sm + sA3, r, j, kHid));
            }
        float v[kHid];
        // dH2 = dOut W3, dZ2 = dH2 * [h2 > 0]
        ok = run_gemm(tmem + 64, sm + sA4, sm + sB4, kOutP, kHid, &mbar, phase);
        if (ok) {
            read_row(tmem, 64, 4, v);
            for (int j = 0; j < kHid; ++j) {
                const float dz = get_bf16(sm + sA3, r, j, kHid) > 0.f ? v[j] : 0.f;
                put_bf16(sm + sA5, r, j, kHid, dz);
                if (valid) dZ2[row * kHid + j] = __float2bfloat16_rn(dz);
            }
            // dH1 = dZ2 W2, dZ1 = dH1 * [h1 > 0]
            ok = run_gemm(tmem, sm + sA5, sm + sB5, kHid, kHid, &mbar, phase);
        }
        if (ok) {
            read_row(tmem, 0, 4, v);
            if (valid)
                for (int j = 0; j < kHid; ++j)
                    dZ1[row * kHid + j] = __float2bfloat16_rn(get_bf16(sm + sA2, r, j, kHid) > 0.f ? v[j] : 0.f);
        }
    }
    if (!ok && threadIdx.x == 0) atomicOr(err, 1u);
    drain(&mbar, phase, ok);
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) tc::tmem_free(tmem, 128);
}

// Weight gradients, one CTA per matrix: dW[o][i] = sum_b A[b][o] B[b][i] over the batch,
// with (A, B) = (dZ1, X), (dZ2, H1), (dOut, H2); bias gradients are the column sums of A.
// The batch is consumed in chunks of 64 rows as the K dimension of D[128 x N] += A^T B.
__global__ void __launch_bounds__(kThreads)
wgrad_kernel(const float *x, int ldx, const __nv_bfloat16 *H1, const __nv_bfloat16 *H2, const __nv_bfloat16 *dOut,
             const __nv_bfloat16 *dZ1, const __nv_bfloat16 *dZ2, long long n, float *grad, unsigned int *err)
{
    constexpr int KC = 64;
    __shared__ __align__(1024) unsigned char sA[kRows * KC * 2];
    __shared__ __align__(1024) unsigned char sB[kHid * KC * 2];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int which = blockIdx.x;  // 0: W1, 1: W2, 2: W3
    const int Mr = which == 2 ? kOutP : kHid;
    const int N = which == 0 ? kIn : kHid;
    const int lda = which == 2 ? kOutP : kHid;
    const __nv_bfloat16 *A = which == 0 ? dZ1 : which == 1 ? dZ2 : dOut;
    const __nv_bfloat16 *Bh = which == 1 ? H1 : H2;
    const int ow = which == 0 ? oW1 : which == 1 ? oW2 : oW3;
    const int ob = which == 0 ? ob1 : which == 1 ? ob2 : ob3;
    if (threadIdx.x < 32) tc::tmem_alloc(&tmem_base, 64);
    if (threadIdx.x == 0) tc::mbar_init(&mbar, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    uint32_t phase = 0;
    bool ok = true;
    float bsum = 0.f;
    for (long long b0 = 0; b0 < n && ok; b0 += KC) {
        // A^T chunk: row o (output unit, padded to 128), column k (sample b0 + k)
        for (int e = threadIdx.x; e < kRows * KC; e += blockDim.x) {
            const int o = e / KC, k = e % KC;
            const long long b = b0 + k;
            const float v = (o < Mr && b < n) ? __bfloat162float(A[b * lda + o]) : 0.f;
            put_bf16(sA, o, k, KC, v);
        }
        for (int e = threadIdx.x; e < N * KC; e += blockDim.x) {
            const int i = e / KC, k = e % KC;
            const long long b = b0 + k;
            float v = 0.f;
            if (b < n) v = which == 0 ? x[b * ldx + i] : __bfloat162float(Bh[b * kHid + i]);
            put_bf16(sB, i, k, KC, v);
        }
        if (threadIdx.x < Mr)
            for (int k = 0; k < KC && b0 + k < n; ++k) bsum += __bfloat162float(A[(b0 + k) * lda + threadIdx.x]);
        ok = run_gemm(tmem, sA, sB, KC, N, &mbar, phase, b0 > 0);
    }
    if (ok) {
        float v[kHid];
        read_row(tmem, 0, N / 16, v);
        if (threadIdx.x < Mr) {
            for (int i = 0; i < N; ++i) grad[ow + threadIdx.x * N + i] = v[i];
            grad[ob + threadIdx.x] = bsum;
        }
    } else if (threadIdx.x == 0) {
        atomicOr(err, 1u);
    }
    drain(&mbar, phase, ok);
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) tc::tmem_free(tmem, 64);
}

__global__ void adam_kernel(float *prm, const float *g, float *m, float *v, float lr, float b1, float b2, float eps,
                            float bc1, float bc2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kParams) return;
    const float gi = g[i];
    m[i] = b1 * m[i] + (1.f - b1) * gi;
    v[i] = b2 * v[i] + (1.f - b2) * gi * gi;
    prm[i] -= lr * (m[i] / bc1) / (sqrtf(v[i] / bc2) + eps);
}

// ------------------------------------------------------------------ features

// stencil slot data in face orientation: density, velocity differences from the
// predictor frame (normal, tangential), temperature
struct SlotPrim {
    float rho, dun, dut, T;
};

__device__ __forceinline__ float clip20(float v) { return fminf(fmaxf(v, -20.f), 20.f); }

__device__ __forceinline__ void features(const SlotPrim *s, float Tp, float h_dn, float *f)
{
    const float rsq = rsqrtf(Tp), rlr = 0.5f * (s[1].rho + s[2].rho);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        f[4 * q + 0] = clip20(__logf(s[q].rho / rlr));
        f[4 * q + 1] = clip20(s[q].dun * rsq);
        f[4 * q + 2] = clip20(s[q].dut * rsq);
        f[4 * q + 3] = clip20(__logf(s[q].T / Tp));
    }
    f[32] = clip20(h_dn * sqrtf(Tp));
    f[33] = 1.f;
#pragma unroll
    for (int q = kUsed; q < kIn; ++q) f[q] = 0.f;
}

}  // namespace mlp
}  // namespace pond
