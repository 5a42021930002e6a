// pond_reduce.cuh -- compensated (double-double) global sums of the conserved fields.
#pragma once

namespace pond {

// Compensated (double-double) sums of four fields scaled by vol: per-block partials
// (hi, lo) into part[block][8]; a single block then folds the partials into out[4].
__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e)
{
    s = a + b;
    const double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void dd_add(double &hi, double &lo, double bh, double bl)
{
    double s, e;
    two_sum(hi, bh, s, e);
    e += lo + bl;
    hi = s + e;
    lo = e - (hi - s);
}

__global__ void dd_partial_kernel(const double *a0, const double *a1, const double *a2, const double *a3, long long n,
                                  double *part)
{
    __shared__ double sh[4][2][256];
    double hi[4] = {0, 0, 0, 0}, lo[4] = {0, 0, 0, 0};
    const double *src[4] = {a0, a1, a2, a3};
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (src[k]) dd_add(hi[k], lo[k], src[k][c], 0.0);
#pragma unroll
    for (int k = 0; k < 4; ++k) { sh[k][0][threadIdx.x] = hi[k]; sh[k][1][threadIdx.x] = lo[k]; }
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                double h = sh[k][0][threadIdx.x], l = sh[k][1][threadIdx.x];
                dd_add(h, l, sh[k][0][threadIdx.x + s], sh[k][1][threadIdx.x + s]);
                sh[k][0][threadIdx.x] = h;
                sh[k][1][threadIdx.x] = l;
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 4; ++k) { part[blockIdx.x * 8 + 2 * k] = sh[k][0][0]; part[blockIdx.x * 8 + 2 * k + 1] = sh[k][1][0]; }
}

__global__ void dd_final_kernel(const double *part, int nparts, double vol, double *out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int k = 0; k < 4; ++k) {
        double hi = 0.0, lo = 0.0;
        for (int b = 0; b < nparts; ++b) dd_add(hi, lo, part[b * 8 + 2 * k], part[b * 8 + 2 * k + 1]);
        out[k] = (hi + lo) * vol;
    }
}

}  // namespace pond
