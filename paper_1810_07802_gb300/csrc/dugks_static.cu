// dugks_static.cu -- dugks_reduce_fields_static: an FP64 field reduction that
// allocates no device memory.
//
// Who needs it: callers that must not call cudaMalloc/cudaFree at the point
// where they want a convergence check -- for example a code path being
// recorded into a CUDA graph (allocation calls are not allowed while a
// stream is captured), a serving loop that plans all device memory up front
// and forbids allocation afterwards, or a host that links this library
// without owning any allocator.  They hand in the macro fields (e.g. from
// dugks_macros with dst_is_device = 1) and a small device output buffer;
// the per-block partial sums go to a fixed array that lives in this
// library's device image instead of a workspace.
//
// The scratch array is sized for at most DUGKS_STATIC_REDUCE_MAX_CELLS cells
// (one record of partial sums per block of 4096 cells); larger requests are
// rejected.  It exists once per GPU that loads the library and stays
// resident until the process exits.  Every call overwrites the records it
// reads, so nothing has to be cleared between calls; two calls that overlap
// on the GPU (different streams, or different host threads) share the array
// and race.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "dugks.h"

namespace {

constexpr int kThreads = 256;
constexpr int kCellsPerThread = 16;
constexpr int kCellsPerBlock = kThreads * kCellsPerThread;          // 4096
constexpr int kMaxBlocks = DUGKS_STATIC_REDUCE_MAX_CELLS / kCellsPerBlock;
constexpr int kVals = 6;   // sum phi, sum phi^2, sum dphi^2, sum |u|^2, sum |du|^2, max |u|
constexpr int kMaxDevices = 64;

static_assert(DUGKS_STATIC_REDUCE_MAX_CELLS % kCellsPerBlock == 0, "whole blocks");

// One record of kVals partial sums per block: 4096 x 6 doubles = 192 KiB.
static __device__ __align__(256) double g_partials[kMaxBlocks * kVals];

// Set-up state per device: the context the address was looked up in and the
// address itself (null until a lookup has succeeded).
std::mutex g_scratch_mu;
CUcontext g_scratch_ctx[kMaxDevices];
double *g_scratch_addr[kMaxDevices];

// The calling thread's current context, through the runtime's driver entry
// point (no libcuda link); null if it cannot be had.
CUcontext current_context() {
    static PFN_cuCtxGetCurrent_v4000 fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return (PFN_cuCtxGetCurrent_v4000) nullptr;
        return reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
    }();
    CUcontext c = nullptr;
    if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
    return c;
}

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

// Block b sums cells [b * 4096, (b + 1) * 4096) into scratch[b * kVals + v].
__global__ void __launch_bounds__(kThreads)
static_partial_kernel(const double *__restrict__ phi, const double *__restrict__ ux, const double *__restrict__ uy,
                      const double *__restrict__ snap, long long n, double *__restrict__ scratch) {
    __shared__ double red[kVals][kThreads / 32];
    double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0, v4 = 0.0, v5 = 0.0;
    const long long base = (long long)blockIdx.x * kCellsPerBlock;
#pragma unroll 4
    for (int i = 0; i < kCellsPerThread; i++) {
        const long long c = base + (long long)i * kThreads + threadIdx.x;
        if (c < n) {
            const double p = phi[c], a = ux[c], b = uy[c];
            const double u2 = a * a + b * b;
            v0 += p;
            v1 += p * p;
            v3 += u2;
            v5 = fmax(v5, sqrt(u2));
            if (snap) {
                const double dp = p - snap[c], da = a - snap[n + c], db = b - snap[2 * n + c];
                v2 += dp * dp;
                v4 += da * da + db * db;
            }
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v0 = warp_sum(v0);
    v1 = warp_sum(v1);
    v2 = warp_sum(v2);
    v3 = warp_sum(v3);
    v4 = warp_sum(v4);
    v5 = warp_max(v5);
    if (lane == 0) {
        red[0][warp] = v0;
        red[1][warp] = v1;
        red[2][warp] = v2;
        red[3][warp] = v3;
        red[4][warp] = v4;
        red[5][warp] = v5;
    }
    __syncthreads();
    if (threadIdx.x < kVals) {
        const int i = threadIdx.x;
        double r = red[i][0];
        for (int w = 1; w < kThreads / 32; w++) r = (i == kVals - 1) ? fmax(r, red[i][w]) : r + red[i][w];
        scratch[blockIdx.x * kVals + i] = r;
    }
}

// One warp folds the nblocks records in a fixed order and writes
// out = {phi mass, residual of phi, residual of u, max |u|}.
__global__ void static_final_kernel(const double *__restrict__ scratch, int nblocks, int have_snap,
                                    double *__restrict__ out) {
    double s[kVals];
    for (int i = 0; i < kVals; i++) {
        double r = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += 32) {
            const double p = scratch[b * kVals + i];
            r = (i == kVals - 1) ? fmax(r, p) : r + p;
        }
        s[i] = (i == kVals - 1) ? warp_max(r) : warp_sum(r);
    }
    if (threadIdx.x == 0) {
        out[0] = s[0];
        out[1] = have_snap ? (s[1] > 0.0 ? s[2] / s[1] : 0.0) : 1.0;
        out[2] = have_snap ? (s[3] > 0.0 ? s[4] / s[3] : 0.0) : 1.0;
        out[3] = s[5];
    }
}

}  // namespace

extern "C" dugks_status dugks_reduce_fields_static(const double *phi, const double *ux, const double *uy,
                                                   const double *snap, int64_t n, double *out, void *cuda_stream) {
    if (!phi || !ux || !uy || !out || n < 1) return DUGKS_ERR_ARG;
    if (n > (int64_t)DUGKS_STATIC_REDUCE_MAX_CELLS) return DUGKS_ERR_ARG;   // beyond the scratch array
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return DUGKS_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return DUGKS_ERR_UNSUPPORTED;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // Set-up, once per device (and per context on it) with the device
    // current: the host name g_partials is only a stand-in, so fetch the
    // array's device address.  A failed lookup is not remembered (the next
    // call tries again); a context created after cudaDeviceReset is a new
    // context and gets its own lookup.
    double *scratch = nullptr;
    {
        const CUcontext ctx = current_context();
        if (!ctx) return DUGKS_ERR_CUDA;
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        if (g_scratch_ctx[dev] != ctx || !g_scratch_addr[dev]) {
            double *p = nullptr;
            if (cudaGetSymbolAddress(reinterpret_cast<void **>(&p), g_partials) != cudaSuccess || !p)
                return DUGKS_ERR_CUDA;
            g_scratch_ctx[dev] = ctx;
            g_scratch_addr[dev] = p;
        }
        scratch = g_scratch_addr[dev];
    }
    const int nblocks = (int)((n + kCellsPerBlock - 1) / kCellsPerBlock);
    static_partial_kernel<<<nblocks, kThreads, 0, st>>>(phi, ux, uy, snap, (long long)n, scratch);
    static_final_kernel<<<1, 32, 0, st>>>(scratch, nblocks, snap != nullptr, out);
    e = cudaGetLastError();
    return e == cudaSuccess ? DUGKS_OK : DUGKS_ERR_CUDA;
}
