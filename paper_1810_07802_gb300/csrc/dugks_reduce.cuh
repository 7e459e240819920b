// dugks_reduce.cuh -- deterministic FP64 reductions of the cell macros
// (phi mass, Eq. 44 residuals, max |u|).  Fixed grid and fixed tree order, so
// the result does not depend on scheduling.  Included by dugks_capi.cu only.
#pragma once

#include <cuda_runtime.h>

namespace dugks {

// ---- deterministic FP64 reductions (fixed grid, fixed tree order) ----
constexpr int RED_BLOCKS = 304;   // 2 x 152 SMs
constexpr int RED_THREADS = 256;
constexpr int RED_VALS = 6;       // sum phi, sum phi^2, sum dphi^2, sum |u|^2, sum |du|^2, max |u|

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Block b reduces cells b, b + RED_BLOCKS*RED_THREADS, ... of n consecutive
// cells of the [ny][nx] macro planes into partial[b][RED_VALS]; the snapshot
// holds phi, ux, uy at snap, snap + sstride, snap + 2 sstride (sstride = n
// for a whole grid).  have_snap = 0 skips the residual sums.
__global__ void __launch_bounds__(RED_THREADS)
reduce_partial_kernel(const double *__restrict__ phi, const double *__restrict__ ux, const double *__restrict__ uy,
                      const double *__restrict__ snap, long long n, long long sstride, int have_snap,
                      double *__restrict__ partial) {
    __shared__ double red[RED_VALS][RED_THREADS / 32];
    double v[RED_VALS] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (long long c = (long long)blockIdx.x * RED_THREADS + threadIdx.x; c < n; c += (long long)RED_BLOCKS * RED_THREADS) {
        const double p = phi[c], a = ux[c], b = uy[c];
        const double u2 = a * a + b * b;
        v[0] += p;
        v[1] += p * p;
        v[3] += u2;
        v[5] = fmax(v[5], sqrt(u2));
        if (have_snap) {
            const double dp = p - snap[c], da = a - snap[sstride + c], db = b - snap[2 * sstride + c];
            v[2] += dp * dp;
            v[4] += da * da + db * db;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < RED_VALS - 1; i++) {
        const double r = warp_sum(v[i]);
        if (lane == 0) red[i][warp] = r;
    }
    {
        const double r = warp_max(v[RED_VALS - 1]);
        if (lane == 0) red[RED_VALS - 1][warp] = r;
    }
    __syncthreads();
    if (threadIdx.x < RED_VALS) {
        const int i = threadIdx.x;
        double r = red[i][0];
        for (int w = 1; w < RED_THREADS / 32; w++) r = (i == 5) ? fmax(r, red[i][w]) : r + red[i][w];
        partial[blockIdx.x * RED_VALS + i] = r;
    }
}

// One warp sums the RED_BLOCKS partials in a fixed order.
__global__ void reduce_final_kernel(const double *__restrict__ partial, double *__restrict__ out) {
    const int lane = threadIdx.x;
    for (int i = 0; i < RED_VALS; i++) {
        double r = (i == 5) ? 0.0 : 0.0;
        for (int b = lane; b < RED_BLOCKS; b += 32) {
            const double p = partial[b * RED_VALS + i];
            r = (i == 5) ? fmax(r, p) : r + p;
        }
        r = (i == 5) ? warp_max(r) : warp_sum(r);
        if (lane == 0) out[i] = r;
    }
}

}  // namespace dugks
