// pond_mlp_train.cuh -- training kernels of the learned face-gauge predictor (forward, loss
// and backward through the activations; weight gradients; Adam), on the tcgen05 tensor cores.
#pragma once

#include "pond_mlp.cuh"

namespace pond {
namespace mlp {

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

// Weight gradients: dW[o][i] = sum_b A[b][o] B[b][i] over the batch, with (A, B) = (dZ1, X),
// (dZ2, H1), (dOut, H2), and bias gradients as the column sums of A.  CTA (which, split)
// takes one matrix and one of nsplit contiguous ranges of 64-row chunks, which it consumes as
// the K dimension of D[128 x N] += A^T B on the tensor cores, and writes its partial
// gradient to part[split][kParams]; wgrad_reduce_kernel then sums the partials in split
// order, so the result does not depend on scheduling.
constexpr int kWgradChunk = 64;
constexpr int kWgradMaxSplit = 48;

// how many row ranges a batch of n rows is split into: at least four 64-row chunks each
__host__ __device__ inline int wgrad_splits(long long n)
{
    const long long chunks = (n + kWgradChunk - 1) / kWgradChunk;
    long long s = chunks / 4;
    if (s < 1) s = 1;
    if (s > kWgradMaxSplit) s = kWgradMaxSplit;
    return int(s);
}

__global__ void __launch_bounds__(kThreads)
wgrad_kernel(const float *x, int ldx, const __nv_bfloat16 *H1, const __nv_bfloat16 *H2, const __nv_bfloat16 *dOut,
             const __nv_bfloat16 *dZ1, const __nv_bfloat16 *dZ2, long long n, float *part, unsigned int *err)
{
    constexpr int KC = kWgradChunk;
    __shared__ __align__(1024) unsigned char sA[kRows * KC * 2];
    __shared__ __align__(1024) unsigned char sB[kHid * KC * 2];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_base;
    // the tile kernel's activations are incomplete when one of its waits expired: leave grad
    // untouched (the call reports POND_ERR_TIMEOUT)
    if (*(volatile unsigned int *)err) return;
    const int which = blockIdx.x;  // 0: W1, 1: W2, 2: W3
    const int split = blockIdx.y, nsplit = gridDim.y;
    const long long nchunks = (n + KC - 1) / KC;
    const long long c_begin = nchunks * split / nsplit, c_end = nchunks * (split + 1) / nsplit;
    const int Mr = which == 2 ? kOutP : kHid;
    const int N = which == 0 ? kIn : kHid;
    const int lda = which == 2 ? kOutP : kHid;
    const __nv_bfloat16 *A = which == 0 ? dZ1 : which == 1 ? dZ2 : dOut;
    const __nv_bfloat16 *Bh = which == 1 ? H1 : H2;
    const int ow = which == 0 ? oW1 : which == 1 ? oW2 : oW3;
    const int ob = which == 0 ? ob1 : which == 1 ? ob2 : ob3;
    float *grad = part + size_t(split) * kParams;
    if (c_begin >= c_end) {   // an empty range contributes zero
        if (threadIdx.x < Mr) {
            for (int i = 0; i < N; ++i) grad[ow + threadIdx.x * N + i] = 0.f;
            grad[ob + threadIdx.x] = 0.f;
        }
        return;
    }
    if (threadIdx.x < 32) tc::tmem_alloc(&tmem_base, 64);
    if (threadIdx.x == 0) tc::mbar_init(&mbar, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    uint32_t phase = 0;
    bool ok = true;
    float bsum = 0.f;
    for (long long ci = c_begin; ci < c_end && ok; ++ci) {
        const long long b0 = ci * KC;
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
        ok = run_gemm(tmem, sA, sB, KC, N, &mbar, phase, ci > c_begin);
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

// grad[p] = sum over the splits of part[split][p], in split order (nothing on an error)
__global__ void wgrad_reduce_kernel(const float *part, int nsplit, float *grad, const unsigned int *err)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kParams || *(const volatile unsigned int *)err) return;
    float acc = 0.f;
    for (int sp = 0; sp < nsplit; ++sp) acc += part[size_t(sp) * kParams + p];
    grad[p] = acc;
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

}  // namespace mlp
}  // namespace pond
