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
static cudaError_t launch_step_t(const StepArgs<Real> &a, const Phys<Real> &ph, const CUtensorMap *tm_state,
                                 const CUtensorMap *tm_hist, cudaStream_t st) {
    constexpr int TX = Tile<Real>::TX, TY = Tile<Real>::TY;
    using S = TileShape<Real, TX, TY, COUPLED>;
    auto kern = step_kernel<Real, TX, TY, COUPLED, WALLY>;
    static const cudaError_t attr =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::smem_bytes);
    if (attr != cudaSuccess) return attr;
    dim3 grid((a.nx + TX - 1) / TX, (a.ny + TY - 1) / TY);
    StepArgs<Real> b = a;
    b.small = (a.nx < TX + 4 || a.ny < TY + 4) ? 1 : 0;   // halo indices may wrap more than once
    kern<<<grid, S::NT, S::smem_bytes, st>>>(*tm_state, *tm_hist, b, ph);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_step(const StepArgs<Real> &a, const Phys<Real> &ph, bool coupled, bool wally,
                        const CUtensorMap *tm_state, const CUtensorMap *tm_hist, cudaStream_t st) {
    if (coupled)
        return wally ? launch_step_t<Real, true, true>(a, ph, tm_state, tm_hist, st)
                     : launch_step_t<Real, true, false>(a, ph, tm_state, tm_hist, st);
    return wally ? launch_step_t<Real, false, true>(a, ph, tm_state, tm_hist, st)
                 : launch_step_t<Real, false, false>(a, ph, tm_state, tm_hist, st);
}

template <typename Real>
size_t step_smem_bytes(bool coupled) {
    constexpr int TX = Tile<Real>::TX, TY = Tile<Real>::TY;
    return coupled ? TileShape<Real, TX, TY, true>::smem_bytes : TileShape<Real, TX, TY, false>::smem_bytes;
}

template <typename Real>
int step_tile(int axis) { return axis == 0 ? Tile<Real>::TX : Tile<Real>::TY; }

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
    template cudaError_t launch_step<Real>(const StepArgs<Real> &, const Phys<Real> &, bool, bool,                 \
                                           const CUtensorMap *, const CUtensorMap *, cudaStream_t);                 \
    template size_t step_smem_bytes<Real>(bool);                                                                    \
    template int step_tile<Real>(int);                                                                              \
    template cudaError_t launch_init<Real>(const double *, Real *, Real *, int, int, int, long long,                \
                                           const Phys<double> &, bool, bool, cudaStream_t);                         \
    template cudaError_t launch_macros<Real>(const FieldArgs<Real> &, double *, const Phys<double> &, bool, bool,  \
                                             double *, double *, double *, double *, cudaStream_t);                 \
    template cudaError_t launch_export<Real>(const FieldArgs<Real> &, int, double, double, double *, double *,     \
                                             cudaStream_t);

}  // namespace dugks
