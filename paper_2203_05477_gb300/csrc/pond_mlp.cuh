// pond_mlp.cuh -- learned face-gauge predictor: a small MLP on the 5th-generation tensor cores.
//
// The corrector of Sec. III.B.3 starts each face from the previous half step's frame.
// This network predicts the converged frame from the face stencil, so the corrector starts
// nearer its fixed point; the corrector and its convergence test are unchanged and alone
// decide the result.
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
