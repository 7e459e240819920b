// dugks_launch.cuh -- host-side launchers of the device kernels, templated on
// the arithmetic/storage type.  Each precision is instantiated in its own
// translation unit (dugks_fp64.cu, dugks_fp32.cu) so the two compile in
// parallel.
#pragma once

#include "dugks_aux.cuh"
#include "dugks_internal.h"

#include <mutex>
#include <type_traits>

namespace dugks {

// Tile shapes compiled into the library, per precision.  Shape 0 is the
// default, chosen by sweeps on GB300 for large boxes (FP32 32 x 8: full
// 128-byte rows per warp; FP64 16 x 8: least halo recompute for an ALU-bound
// step); the narrower ones suit narrow domains (e.g. Nx = 4 channels) and are
// candidates for the autotuner.
template <typename Real> struct TileSet;
#ifndef DUGKS_TILE_F32_Y0
#define DUGKS_TILE_F32_Y0 8
#endif
template <> struct TileSet<float> {
    static constexpr int N = 4;
    static constexpr int TX[N] = {32, 16, 8, 4}, TY[N] = {DUGKS_TILE_F32_Y0, 16, 32, 64};
};
template <> struct TileSet<double> {
    static constexpr int N = 3;
    static constexpr int TX[N] = {16, 8, 4}, TY[N] = {8, 16, 32};
};

// Calls f(std::integral_constant<int, V>) for the compiled shape V == v.
template <typename Real, int V = 0, typename F>
cudaError_t with_tile(int v, F &&f) {
    if constexpr (V < TileSet<Real>::N) {
        if (v == V) return f(std::integral_constant<int, V>{});
        return with_tile<Real, V + 1>(v, f);
    } else {
        return cudaErrorInvalidValue;
    }
}

// Calls f(integral_constant<int, tile>, bool_constant<COUPLED>,
// bool_constant<WALLY>, bool_constant<UPW>) for the compiled kernel variant.
// The upwind reconstruction is compiled for the default tile shape only.
template <typename Real, typename F>
cudaError_t with_kernel(int tile, bool coupled, bool wally, bool upw, F &&f) {
    using T = std::true_type;
    using U = std::false_type;
    if (upw) {
        if (tile != 0) return cudaErrorInvalidValue;
        const std::integral_constant<int, 0> v0{};
        if (coupled) return wally ? f(v0, T{}, T{}, T{}) : f(v0, T{}, U{}, T{});
        return wally ? f(v0, U{}, T{}, T{}) : f(v0, U{}, U{}, T{});
    }
    return with_tile<Real>(tile, [&](auto v) {
        if (coupled) return wally ? f(v, T{}, T{}, U{}) : f(v, T{}, U{}, U{});
        return wally ? f(v, U{}, T{}, U{}) : f(v, U{}, U{}, U{});
    });
}

// CTAs of the persistent batched kernel that fit on the device at once
// (resident per SM x SMs), per device; set with the kernel attributes below.
template <typename Real, int TX, int TY, bool COUPLED, bool WALLY, bool UPW>
static int &persistent_capacity(int dev) {
    static int cap[64];
    return cap[dev];
}

// Raises the step kernels' dynamic shared-memory limit, once per device (the
// attribute belongs to the device's context), and sizes the persistent grid.
template <typename Real, int TX, int TY, bool COUPLED, bool WALLY, bool UPW>
static cudaError_t step_attr_t() {
    using S = TileShape<Real, TX, TY, COUPLED, UPW>;
    constexpr int kDevices = 64;
    static std::once_flag once[kDevices];
    static cudaError_t result[kDevices];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kDevices) return cudaErrorInvalidDevice;
    std::call_once(once[dev], [&] {
        cudaError_t a = cudaFuncSetAttribute(step_kernel<Real, TX, TY, COUPLED, WALLY, UPW>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::smem_bytes);
        cudaError_t b = cudaFuncSetAttribute(solo_step_kernel<Real, TX, TY, COUPLED, WALLY, UPW>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::smem_bytes);
        cudaError_t c = cudaFuncSetAttribute(persistent_step_kernel<Real, TX, TY, COUPLED, WALLY, UPW>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::smem_bytes);
        int per_sm = 0, sms = 0;
        if (c == cudaSuccess)
            c = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent_step_kernel<Real, TX, TY, COUPLED, WALLY, UPW>,
                                                              S::NT, S::smem_bytes);
        if (c == cudaSuccess) c = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        persistent_capacity<Real, TX, TY, COUPLED, WALLY, UPW>(dev) = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
        result[dev] = a != cudaSuccess ? a : (b != cudaSuccess ? b : c);
    });
    return result[dev];
}

#define DUGKS_KERNEL_PARAMS(v, c, w, u)                                                                          \
    constexpr int TX = TileSet<Real>::TX[decltype(v)::value], TY = TileSet<Real>::TY[decltype(v)::value];         \
    constexpr bool C = decltype(c)::value, W = decltype(w)::value, UP = decltype(u)::value;                       \
    using S = TileShape<Real, TX, TY, C, UP>;

// Must run outside stream capture (sets the kernels' shared-memory limit).
template <typename Real>
cudaError_t step_prepare(int tile, bool coupled, bool wally, bool upw) {
    return with_kernel<Real>(tile, coupled, wally, upw, [&](auto v, auto c, auto w, auto u) {
        DUGKS_KERNEL_PARAMS(v, c, w, u)
        (void)sizeof(S);
        return step_attr_t<Real, TX, TY, C, W, UP>();
    });
}

// Rows of the step kernel's input box (the tensor maps' box height).
template <typename Real>
int step_box_rows(int tile, bool upw) {
    const int ty = (tile >= 0 && tile < TileSet<Real>::N) ? TileSet<Real>::TY[tile] : 0;
    return ty + (upw ? 6 : 4);
}

// One step of one problem: maps, arguments and constants by value.
template <typename Real>
cudaError_t launch_step(int tile, bool upw, const CUtensorMap &tm_state, const CUtensorMap &tm_hist,
                        const StepArgs<Real> &a, const Phys<Real> &ph, bool coupled, bool wally, cudaStream_t st) {
    cudaError_t e = step_prepare<Real>(tile, coupled, wally, upw);
    if (e != cudaSuccess) return e;
    return with_kernel<Real>(tile, coupled, wally, upw, [&](auto v, auto c, auto w, auto u) {
        DUGKS_KERNEL_PARAMS(v, c, w, u)
        const int tiles_x = (a.nx + TX - 1) / TX;
        const int ntiles = tiles_x * ((a.ny + TY - 1) / TY);
        solo_step_kernel<Real, TX, TY, C, W, UP><<<ntiles, S::NT, S::smem_bytes, st>>>(tm_state, tm_hist, a, ph,
                                                                                        tiles_x);
        return cudaGetLastError();
    });
}

template <typename Real>
int tile_count() { return TileSet<Real>::N; }

template <typename Real>
int tile_dim(int tile, int axis) {
    if (tile < 0 || tile >= TileSet<Real>::N) return 0;
    return axis == 0 ? TileSet<Real>::TX[tile] : TileSet<Real>::TY[tile];
}

// ---- batched step ----
template <typename Real>
cudaError_t batch_prepare(int tile, bool coupled, bool wally, bool upw) {
    return step_prepare<Real>(tile, coupled, wally, upw);
}

// ksteps batched steps of one group.  With ctr (1 + ninst counters): one
// persistent launch over all ksteps (counters cleared first), then one
// advance of the descriptors.  Without: ksteps grid launches of one step,
// each followed by an advance.
template <typename Real>
cudaError_t launch_batch_step(int tile, bool upw, InstDesc<Real> *descs, const int2 *work, int nwork, int ninst,
                              bool coupled, bool wally, int ksteps, unsigned *ctr, cudaStream_t st) {
    if (nwork <= 0 || ksteps <= 0) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (ctr) {
        e = cudaMemsetAsync(ctr, 0, (size_t)(1 + ninst) * sizeof(unsigned), st);
        if (e != cudaSuccess) return e;
        e = with_kernel<Real>(tile, coupled, wally, upw, [&](auto v, auto c, auto w, auto u) {
            DUGKS_KERNEL_PARAMS(v, c, w, u)
            // at most one step's items: more CTAs would only wait for the next step
            const int resident = persistent_capacity<Real, TX, TY, C, W, UP>(dev);
            const int cap = nwork < resident ? nwork : resident;
            const int grid = cap > 0 ? cap : 1;
            persistent_step_kernel<Real, TX, TY, C, W, UP><<<grid, S::NT, S::smem_bytes, st>>>(descs, work, nwork,
                                                                                              ksteps, ctr);
            return cudaGetLastError();
        });
        if (e != cudaSuccess) return e;
        advance_kernel<Real><<<(ninst + 127) / 128, 128, 0, st>>>(descs, ninst, ksteps);
        return cudaGetLastError();
    }
    for (int k = 0; k < ksteps; k++) {
        e = with_kernel<Real>(tile, coupled, wally, upw, [&](auto v, auto c, auto w, auto u) {
            DUGKS_KERNEL_PARAMS(v, c, w, u)
            step_kernel<Real, TX, TY, C, W, UP><<<nwork, S::NT, S::smem_bytes, st>>>(descs, work);
            return cudaGetLastError();
        });
        if (e != cudaSuccess) return e;
        advance_kernel<Real><<<(ninst + 127) / 128, 128, 0, st>>>(descs, ninst, 1);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static inline dim3 cell_grid(int nx, int ny, int bx) { return dim3((nx + bx - 1) / bx, ny); }

template <typename Real>
cudaError_t launch_init(const double *in, Real *state, Real *hist, int nx, int ny, int pitch, long long plane,
                        const Phys<double> &ph, bool coupled, bool wally, cudaStream_t st) {
    const int bx = 128;
    dim3 grid = cell_grid(nx, ny, bx);
    if (coupled) {
        if (wally) init_kernel<Real, true, true><<<grid, bx, 0, st>>>(in, state, hist, nx, ny, pitch, plane, ph);
        else init_kernel<Real, true, false><<<grid, bx, 0, st>>>(in, state, hist, nx, ny, pitch, plane, ph);
    } else {
        if (wally) init_kernel<Real, false, true><<<grid, bx, 0, st>>>(in, state, hist, nx, ny, pitch, plane, ph);
        else init_kernel<Real, false, false><<<grid, bx, 0, st>>>(in, state, hist, nx, ny, pitch, plane, ph);
    }
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_macros(const FieldArgs<Real> &a, double *phid, const Phys<double> &ph, bool coupled, bool wally,
                          double *ophi, double *op, double *oux, double *ouy, cudaStream_t st) {
    const int bx = 128;
    dim3 grid = cell_grid(a.nx, a.ny, bx);
    phi_kernel<Real><<<grid, bx, 0, st>>>(a, phid);
    if (coupled) {
        if (wally) macro_kernel<Real, true, true><<<grid, bx, 0, st>>>(a, phid, ph, ophi, op, oux, ouy);
        else macro_kernel<Real, true, false><<<grid, bx, 0, st>>>(a, phid, ph, ophi, op, oux, ouy);
    } else {
        if (wally) macro_kernel<Real, false, true><<<grid, bx, 0, st>>>(a, phid, ph, ophi, op, oux, ouy);
        else macro_kernel<Real, false, false><<<grid, bx, 0, st>>>(a, phid, ph, ophi, op, oux, ouy);
    }
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_export(const FieldArgs<Real> &a, int nq, double phi_ref, double p_ref, double *dist,
                          double *hist_out, cudaStream_t st) {
    const int bx = 128;
    export_kernel<Real><<<cell_grid(a.nx, a.ny, bx), bx, 0, st>>>(a, nq, phi_ref, p_ref, dist, hist_out);
    return cudaGetLastError();
}

#define DUGKS_INSTANTIATE(Real)                                                                                     \
    template cudaError_t launch_step<Real>(int, bool, const CUtensorMap &, const CUtensorMap &,                    \
                                           const StepArgs<Real> &, const Phys<Real> &, bool, bool, cudaStream_t);  \
    template int tile_count<Real>();                                                                                \
    template int tile_dim<Real>(int, int);                                                                          \
    template int step_box_rows<Real>(int, bool);                                                                    \
    template cudaError_t launch_init<Real>(const double *, Real *, Real *, int, int, int, long long,                \
                                           const Phys<double> &, bool, bool, cudaStream_t);                         \
    template cudaError_t launch_macros<Real>(const FieldArgs<Real> &, double *, const Phys<double> &, bool, bool,  \
                                             double *, double *, double *, double *, cudaStream_t);                 \
    template cudaError_t launch_export<Real>(const FieldArgs<Real> &, int, double, double, double *, double *,     \
                                             cudaStream_t);                                                        \
    template cudaError_t batch_prepare<Real>(int, bool, bool, bool);                                               \
    template cudaError_t launch_batch_step<Real>(int, bool, InstDesc<Real> *, const int2 *, int, int, bool, bool,  \
                                                 int, unsigned *, cudaStream_t);

}  // namespace dugks
