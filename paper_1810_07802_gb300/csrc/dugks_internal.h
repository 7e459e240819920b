// dugks_internal.h -- declarations shared by the host C-ABI and the
// per-precision kernel translation units.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "dugks_device.cuh"

namespace dugks {

template <typename Real> struct FieldArgs;

template <typename Real>
cudaError_t launch_step(const StepArgs<Real> &a, const Phys<Real> &ph, bool coupled, bool wally,
                        const CUtensorMap *tm_state, const CUtensorMap *tm_hist, cudaStream_t st);
template <typename Real>
size_t step_smem_bytes(bool coupled);
template <typename Real>
int step_tile(int axis);
template <typename Real>
cudaError_t launch_init(const double *in, Real *state, Real *hist, int nx, int ny, int pitch, long long plane,
                        const Phys<double> &ph, bool coupled, bool wally, cudaStream_t st);
template <typename Real>
cudaError_t launch_macros(const FieldArgs<Real> &a, double *phid, const Phys<double> &ph, bool coupled, bool wally,
                          double *ophi, double *op, double *oux, double *ouy, cudaStream_t st);
template <typename Real>
cudaError_t launch_export(const FieldArgs<Real> &a, int nq, double phi_ref, double p_ref, double *dist,
                          double *hist_out, cudaStream_t st);
cudaError_t launch_reduce(const double *phi, const double *ux, const double *uy, const double *snap, long long n,
                          int have_snap, double *partial, double *out, cudaStream_t st);

}  // namespace dugks
