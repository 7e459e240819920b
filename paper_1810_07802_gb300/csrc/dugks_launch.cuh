// dugks_launch.cuh -- host-side launchers of the device kernels, templated on
// the arithmetic/storage type.  Each precision is instantiated in its own
// translation unit (dugks_fp64.cu, dugks_fp32.cu) so the two compile in
// parallel.
#pragma once

#include "dugks_aux.cuh"
#include "dugks_internal.h"

namespace dugks {

// Tile shapes (build-time; measured on GB300, see profiles/): FP64 favours
// square tiles (least halo recompute for an ALU-bound step), FP32 wide tiles
// (full 128-byte rows per warp).
#ifndef DUGKS_TILE_F64_X
#define DUGKS_TILE_F64_X 16
#endif
#ifndef DUGKS_TILE_F64_Y
#define DUGKS_TILE_F64_Y 8
#endif
#ifndef DUGKS_TILE_F32_X
#define DUGKS_TILE_F32_X 32
#endif
#ifndef DUGKS_TILE_F32_Y
#define DUGKS_TILE_F32_Y 8
#endif
template <typename Real> struct Tile;
template <> struct Tile<double> { static constexpr int TX = DUGKS_TILE_F64_X, TY = DUGKS_TILE_F64_Y; };
template <> struct Tile<float> { static constexpr int TX = DUGKS_TILE_F32_X, TY = DUGKS_TILE_F32_Y; };

template <typename Real, bool COUPLED, bool WALLY>
static cudaError_t step_attr_t() {
    constexpr int TX = Tile<Real>::TX, TY = Tile<Real>::TY;
    using S = TileShape<Real, TX, TY, COUPLED>;
    static const cudaError_t attr = cudaFuncSetAttribute(step_kernel<Real, TX, TY, COUPLED, WALLY>,
                                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                         (int)S::smem_bytes);
    static const cudaError_t attr_solo = cudaFuncSetAttribute(solo_step_kernel<Real, TX, TY, COUPLED, WALLY>,
                                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                              (int)S::smem_bytes);
    return attr != cudaSuccess ? attr : attr_solo;
}

// Must run outside stream capture (sets the kernel's shared-memory limit).
template <typename Real>
cudaError_t step_prepare(bool coupled, bool wally) {
    if (coupled) return wally ? step_attr_t<Real, true, true>() : step_attr_t<Real, true, false>();
    return wally ? step_attr_t<Real, false, true>() : step_attr_t<Real, false, false>();
}

template <typename Real, bool COUPLED, bool WALLY>
static void batch_launch_t(const InstDesc<Real> *descs, const int2 *work, int nitems, cudaStream_t st) {
    constexpr int TX = Tile<Real>::TX, TY = Tile<Real>::TY;
    using S = TileShape<Real, TX, TY, COUPLED>;
    step_kernel<Real, TX, TY, COUPLED, WALLY><<<nitems, S::NT, S::smem_bytes, st>>>(descs, work);
}

// One step of one problem: maps, arguments and constants by value.
template <typename Real>
cudaError_t launch_step(const CUtensorMap &tm_state, const CUtensorMap &tm_hist, const StepArgs<Real> &a,
                        const Phys<Real> &ph, bool coupled, bool wally, cudaStream_t st) {
    cudaError_t e = step_prepare<Real>(coupled, wally);
    if (e != cudaSuccess) return e;
    constexpr int TX = Tile<Real>::TX, TY = Tile<Real>::TY;
    const int tiles_x = (a.nx + TX - 1) / TX;
    const int ntiles = tiles_x * ((a.ny + TY - 1) / TY);
    if (coupled) {
        using S = TileShape<Real, TX, TY, true>;
        if (wally) solo_step_kernel<Real, TX, TY, true, true><<<ntiles, S::NT, S::smem_bytes, st>>>(tm_state, tm_hist, a, ph, tiles_x);
        else solo_step_kernel<Real, TX, TY, true, false><<<ntiles, S::NT, S::smem_bytes, st>>>(tm_state, tm_hist, a, ph, tiles_x);
    } else {
        using S = TileShape<Real, TX, TY, false>;
        if (wally) solo_step_kernel<Real, TX, TY, false, true><<<ntiles, S::NT, S::smem_bytes, st>>>(tm_state, tm_hist, a, ph, tiles_x);
        else solo_step_kernel<Real, TX, TY, false, false><<<ntiles, S::NT, S::smem_bytes, st>>>(tm_state, tm_hist, a, ph, tiles_x);
    }
    return cudaGetLastError();
}

template <typename Real>
size_t step_smem_bytes(bool coupled) {
    constexpr int TX = Tile<Real>::TX, TY = Tile<Real>::TY;
    return coupled ? TileShape<Real, TX, TY, true>::smem_bytes : TileShape<Real, TX, TY, false>::smem_bytes;
}

template <typename Real>
int step_tile(int axis) { return axis == 0 ? Tile<Real>::TX : Tile<Real>::TY; }

// ---- batched step ----
template <typename Real>
cudaError_t batch_prepare(bool coupled, bool wally) {
    return step_prepare<Real>(coupled, wally);
}

template <typename Real>
cudaError_t launch_batch_step(InstDesc<Real> *descs, const int2 *work, int nwork, int ninst, bool coupled, bool wally,
                              cudaStream_t st) {
    if (nwork <= 0) return cudaSuccess;
    if (coupled) {
        if (wally) batch_launch_t<Real, true, true>(descs, work, nwork, st);
        else batch_launch_t<Real, true, false>(descs, work, nwork, st);
    } else {
        if (wally) batch_launch_t<Real, false, true>(descs, work, nwork, st);
        else batch_launch_t<Real, false, false>(descs, work, nwork, st);
    }
    advance_kernel<Real><<<(ninst + 127) / 128, 128, 0, st>>>(descs, ninst);
    return cudaGetLastError();
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
    template cudaError_t launch_step<Real>(const CUtensorMap &, const CUtensorMap &, const StepArgs<Real> &,       \
                                           const Phys<Real> &, bool, bool, cudaStream_t);                          \
    template size_t step_smem_bytes<Real>(bool);                                                                    \
    template int step_tile<Real>(int);                                                                              \
    template cudaError_t launch_init<Real>(const double *, Real *, Real *, int, int, int, long long,                \
                                           const Phys<double> &, bool, bool, cudaStream_t);                         \
    template cudaError_t launch_macros<Real>(const FieldArgs<Real> &, double *, const Phys<double> &, bool, bool,  \
                                             double *, double *, double *, double *, cudaStream_t);                 \
    template cudaError_t launch_export<Real>(const FieldArgs<Real> &, int, double, double, double *, double *,     \
                                             cudaStream_t);                                                        \
    template cudaError_t batch_prepare<Real>(bool, bool);                                                          \
    template cudaError_t launch_batch_step<Real>(InstDesc<Real> *, const int2 *, int, int, bool, bool, cudaStream_t);

}  // namespace dugks
