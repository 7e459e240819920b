// dugks_internal.h -- declarations shared by the host C-ABI and the
// per-precision kernel translation units.  Not part of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <string.h>

#include <cstring>

#include "dugks.h"
#include "dugks_device.cuh"

namespace dugks {

template <typename Real> struct FieldArgs;
template <typename Real> struct InstDesc;

template <typename Real>
cudaError_t launch_step(int tile, bool upw, const CUtensorMap &tm_state, const CUtensorMap &tm_hist,
                        const StepArgs<Real> &a, const Phys<Real> &ph, bool coupled, bool wally, cudaStream_t st);
template <typename Real>
int step_box_rows(int tile, bool upw);
template <typename Real>
int tile_count();
template <typename Real>
int tile_dim(int tile, int axis);   // 0 for a shape that is not compiled
template <typename Real>
cudaError_t launch_init(const double *in, Real *state, Real *hist, int nx, int ny, int pitch, long long plane,
                        const Phys<double> &ph, bool coupled, bool wally, cudaStream_t st);
template <typename Real>
cudaError_t launch_macros(const FieldArgs<Real> &a, double *phid, const Phys<double> &ph, bool coupled, bool wally,
                          double *ophi, double *op, double *oux, double *ouy, cudaStream_t st);
template <typename Real>
cudaError_t launch_export(const FieldArgs<Real> &a, int nq, double phi_ref, double p_ref, double *dist,
                          double *hist_out, cudaStream_t st);
template <typename Real>
cudaError_t batch_prepare(int tile, bool coupled, bool wally, bool upw);
template <typename Real>
cudaError_t launch_batch_step(int tile, bool upw, InstDesc<Real> *descs, const int2 *work, int nwork, int ninst,
                              bool coupled, bool wally, int ksteps, unsigned *ctr, cudaStream_t st);
cudaError_t launch_reduce(const double *phi, const double *ux, const double *uy, const double *snap, long long n,
                          long long sstride, int have_snap, double *partial, double *out, cudaStream_t st);


// Workspace layout of one solver (offsets in bytes, 256-byte aligned regions).
struct Layout {
    int nq, pitch;
    size_t elt, plane, n;
    size_t off_state[2], off_hist[2], off_vel, off_stage, off_phid, off_snap, off_partial, off_redout, off_status;
    size_t vel_bytes;   // sampled velocity field [4][ny][pitch] (0 unless used)
    size_t total;
};

}  // namespace dugks

// The handle behind dugks_handle.
struct dugks_ctx {
    dugks_params P;
    dugks::Layout L;
    bool fp32, coupled, wally;
    int tile;   // index of the compiled tile shape the step kernels use
    bool upw;   // upwind reconstruction (R14) instead of the central one
    int vel_faces;   // sampled velocity field: face planes set
    cudaStream_t st;
    unsigned char *ws;
    bool owns;
    int cur;
    int64_t steps;
    int have_snap;
    unsigned status_seen;
    dugks::Phys<double> phd;
    dugks::Phys<float> phf;
    bool tma_ok;
    CUtensorMap tm_state[2], tm_hist[2];

    void *state(int b) const { return ws + L.off_state[b]; }
    void *hist(int b) const { return ws + L.off_hist[b]; }
    void *vel() const { return L.vel_bytes ? ws + L.off_vel : nullptr; }
    double *stage() const { return reinterpret_cast<double *>(ws + L.off_stage); }
    double *phid() const { return reinterpret_cast<double *>(ws + L.off_phid); }
    double *snap() const { return reinterpret_cast<double *>(ws + L.off_snap); }
    double *partial() const { return reinterpret_cast<double *>(ws + L.off_partial); }
    double *redout() const { return reinterpret_cast<double *>(ws + L.off_redout); }
    unsigned *status() const { return reinterpret_cast<unsigned *>(ws + L.off_status); }

    // Arguments of the next step (psi~^n in buffer cur).
    template <typename Real>
    dugks::StepArgs<Real> step_args() const {
        const int tx = dugks::tile_dim<Real>(tile, 0), ty = dugks::tile_dim<Real>(tile, 1);
        dugks::StepArgs<Real> a;
        a.src = static_cast<const Real *>(state(cur));
        a.dst = static_cast<Real *>(state(cur ^ 1));
        a.hsrc = static_cast<const Real *>(hist(cur));
        a.hdst = static_cast<Real *>(hist(cur ^ 1));
        a.nx = P.nx;
        a.ny = P.ny;
        a.pitch = L.pitch;
        a.plane = (long long)L.plane;
        a.first_step = steps == 0;
        a.t_n = double(steps) * double(fp32 ? (double)phf.dt : phd.dt);
        a.small = (P.nx < tx + 4 || P.ny < ty + 4) ? 1 : 0;
        a.use_tma = tma_ok ? 1 : 0;
        a.vel = static_cast<const Real *>(vel());
        a.vel_faces = vel_faces;
        a.status = status();
        return a;
    }

    template <typename Real>
    dugks::FieldArgs<Real> fields() const {
        dugks::FieldArgs<Real> a;
        a.state = static_cast<const Real *>(state(cur));
        a.hist = static_cast<const Real *>(hist(cur));
        a.nx = P.nx;
        a.ny = P.ny;
        a.pitch = L.pitch;
        a.plane = (long long)L.plane;
        a.t = double(steps) * P.cfl;
        a.vel = static_cast<const Real *>(vel());
        return a;
    }
};

namespace dugks {
// Enqueues nsteps single-problem steps of c on stream st and advances its
// step count and ping-pong index (dugks_step on the handle's own stream; a
// batch's large members on the batch's stream).
cudaError_t step_on(dugks_ctx *c, long long nsteps, cudaStream_t st);

// Descriptor of one problem for the step kernel (device image built on the host).
template <typename Real>
inline void fill_desc(InstDesc<Real> *d, const dugks_ctx *c, const Phys<Real> &ph, int tx, int ty) {
    std::memset(static_cast<void *>(d), 0, sizeof *d);
    for (int b = 0; b < 2; b++) {
        d->tm_state[b] = c->tm_state[b];
        d->tm_hist[b] = c->tm_hist[b];
        d->state[b] = static_cast<Real *>(c->state(b));
        d->hist[b] = static_cast<Real *>(c->hist(b));
    }
    d->status = c->status();
    d->ph = ph;
    d->plane = (long long)c->L.plane;
    d->steps = c->steps;
    d->nx = c->P.nx;
    d->ny = c->P.ny;
    d->pitch = c->L.pitch;
    d->tiles_x = (c->P.nx + tx - 1) / tx;
    d->ntiles = d->tiles_x * ((c->P.ny + ty - 1) / ty);
    d->cur = c->cur;
    d->use_tma = c->tma_ok ? 1 : 0;
    d->vel = static_cast<const Real *>(c->vel());
    d->vel_faces = c->vel_faces;
}
}  // namespace dugks
