// dugks_capi.cu -- the C ABI of include/dugks.h: parameter validation,
// workspace layout, stream-ordered launches and host<->device transfers.
// All arithmetic of the scheme runs in the kernels (dugks_device.cuh,
// dugks_aux.cuh); this file only marshals.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "dugks.h"
#include "dugks_aux.cuh"
#include "dugks_internal.h"
#include "dugks_reduce.cuh"
#include "dugks_trace.h"

using dugks::FieldArgs;
using dugks::Layout;
using dugks::Phys;
using dugks::StepArgs;

namespace dugks {
// Self-check of the bounded mbarrier wait the step kernel relies on: one
// thread arms a barrier for 16 bytes of a copy that is never issued, waits
// with at most max_polls polls, and records the timeout in *status.  Nothing
// spins beyond the limit and no copy is left in flight.
__global__ void wait_probe_kernel(long max_polls, unsigned *status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_expect_tx(&bar, 16u);
        if (!mbar_wait(&bar, 0, max_polls)) atomicOr(status, STATUS_TIMEOUT);
    }
}

// Self-check of the persistent batched kernel's wait for a member's previous
// step: one thread waits, with the kernel's wait function, for one tile of a
// member whose counter (*ctr, cleared by the caller) nothing raises, giving up
// after budget_ns of sleeps, and records the timeout in *status.
__global__ void batch_wait_probe_kernel(unsigned long long budget_ns, const unsigned *ctr, unsigned *status) {
    if (threadIdx.x == 0 && !member_wait(ctr, 1u, 1u, budget_ns)) atomicOr(status, STATUS_TIMEOUT);
}

// Rows [row0, row0 + nrows) of the stored state (nq distribution planes, then
// the 2 history planes, elements of T) to or from a contiguous buffer
// [nq + 2][nrows][nx].  One thread per element; the grid covers the buffer.
template <typename T>
__global__ void rows_kernel(T *state, T *hist, int nq, int pitch, long long plane, int nx, int row0, int nrows,
                            T *buf, int to_buf) {
    const long long n = (long long)(nq + 2) * nrows * nx;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int x = (int)(i % nx);
    const long long zr = i / nx;
    const int r = (int)(zr % nrows), z = (int)(zr / nrows);
    T *p = z < nq ? state + z * plane : hist + (z - nq) * plane;
    p += (long long)(row0 + r) * pitch + x;
    if (to_buf) buf[i] = *p;
    else *p = buf[i];
}

cudaError_t launch_rows(void *state, void *hist, size_t elt, int nq, int pitch, long long plane, int nx, int row0,
                        int nrows, void *buf, int to_buf, cudaStream_t st) {
    const long long n = (long long)(nq + 2) * nrows * nx;
    const int bx = 256;
    const unsigned grid = (unsigned)((n + bx - 1) / bx);
    if (elt == 4)
        rows_kernel<float><<<grid, bx, 0, st>>>(static_cast<float *>(state), static_cast<float *>(hist), nq, pitch,
                                                plane, nx, row0, nrows, static_cast<float *>(buf), to_buf);
    else
        rows_kernel<double><<<grid, bx, 0, st>>>(static_cast<double *>(state), static_cast<double *>(hist), nq, pitch,
                                                 plane, nx, row0, nrows, static_cast<double *>(buf), to_buf);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const double *phi, const double *ux, const double *uy, const double *snap, long long n,
                          long long sstride, int have_snap, double *partial, double *out, cudaStream_t st) {
    reduce_partial_kernel<<<RED_BLOCKS, RED_THREADS, 0, st>>>(phi, ux, uy, snap, n, sstride, have_snap, partial);
    reduce_final_kernel<<<1, 32, 0, st>>>(partial, out);
    return cudaGetLastError();
}

cudaError_t step_on(dugks_ctx *c, long long nsteps, cudaStream_t st) {
    for (long long n = 0; n < nsteps; n++) {
        cudaError_t e;
        if (c->fp32)
            e = launch_step<float>(c->tile, c->upw, c->tm_state[c->cur], c->tm_hist[c->cur], c->step_args<float>(),
                                   c->phf, c->coupled, c->wally, st);
        else
            e = launch_step<double>(c->tile, c->upw, c->tm_state[c->cur], c->tm_hist[c->cur], c->step_args<double>(),
                                    c->phd, c->coupled, c->wally, st);
        if (e != cudaSuccess) return e;
        c->cur ^= 1;
        c->steps++;
    }
    return cudaSuccess;
}
}  // namespace dugks

namespace {

constexpr size_t kAlign = 256;
constexpr uint64_t kStateMagic = 0x31534b4755440a31ull;  // checkpoint tag
constexpr uint64_t kStateVersion = 1;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }



bool valid(const dugks_params *p) {
    if (!p) return false;
    if (p->nx < 3 || p->ny < 3 || p->lattice != 9) return false;
    if (p->model != DUGKS_COUPLED && p->model != DUGKS_AC_PRESCRIBED_U) return false;
    if (p->precision != DUGKS_FP64 && p->precision != DUGKS_FP32_SHIFTED) return false;
    const int ntiles = p->precision == DUGKS_FP32_SHIFTED ? dugks::tile_count<float>() : dugks::tile_count<double>();
    if (p->tile_shape < 0 || p->tile_shape > ntiles) return false;
    if (p->recon != DUGKS_RECON_CENTRAL && p->recon != DUGKS_RECON_UPWIND) return false;
    if (p->reserved3 != 0) return false;
    if (p->bc_x != DUGKS_BC_PERIODIC && p->bc_x != DUGKS_BC_WALL) return false;
    if (p->bc_y != DUGKS_BC_PERIODIC && p->bc_y != DUGKS_BC_WALL) return false;
    if (p->visc_interp != DUGKS_VISC_RECIPROCAL && p->visc_interp != DUGKS_VISC_LINEAR) return false;
    if (p->gravity_mode != 0 && p->gravity_mode != 1) return false;
    if (p->velocity_field < 0 || p->velocity_field > 4 || p->reserved2 != 0) return false;
    if (p->velocity_field == 4 && p->model != DUGKS_AC_PRESCRIBED_U) return false;
    auto pos = [](double v) { return std::isfinite(v) && v > 0.0; };
    auto fin = [](double v) { return std::isfinite(v); };
    if (!pos(p->cfl) || !pos(p->mobility) || !pos(p->width)) return false;
    if (!fin(p->phi_ref) || !fin(p->p_ref) || !fin(p->u0x) || !fin(p->u0y)) return false;
    if (p->model == DUGKS_AC_PRESCRIBED_U && p->velocity_field >= 1 && p->velocity_field <= 3 &&
        (!pos(p->vel_u0) || !pos(p->vel_length)))
        return false;
    if (p->model == DUGKS_COUPLED) {
        if (!pos(p->rho_h) || !pos(p->rho_l) || !pos(p->mu_h) || !pos(p->mu_l)) return false;
        if (!fin(p->sigma) || p->sigma < 0.0 || !fin(p->gx) || !fin(p->gy) || !fin(p->rho_ref)) return false;
    }
    // grid dimensions of the kernels and 64-bit sizes
    if ((long long)p->nx * p->ny > (1ll << 40)) return false;
    return true;
}

Layout layout(const dugks_params *p) {
    Layout L;
    L.nq = p->model == DUGKS_COUPLED ? 18 : 9;
    L.elt = p->precision == DUGKS_FP64 ? 8 : 4;
    L.pitch = (int)align_up((size_t)p->nx, 32);  // 128-byte (FP32) / 256-byte (FP64) rows
    L.plane = (size_t)L.pitch * (size_t)p->ny;
    L.n = (size_t)p->nx * (size_t)p->ny;
    size_t o = 0;
    for (int b = 0; b < 2; b++) {
        L.off_state[b] = o;
        o = align_up(o + (size_t)L.nq * L.plane * L.elt, kAlign);
    }
    for (int b = 0; b < 2; b++) {
        L.off_hist[b] = o;
        o = align_up(o + 2 * L.plane * L.elt, kAlign);
    }
    L.vel_bytes = (p->model == DUGKS_AC_PRESCRIBED_U && p->velocity_field == 4) ? 4 * L.plane * L.elt : 0;
    L.off_vel = o;
    o = align_up(o + L.vel_bytes, kAlign);
    L.off_stage = o;   o = align_up(o + 4 * L.n * sizeof(double), kAlign);
    L.off_phid = o;    o = align_up(o + L.n * sizeof(double), kAlign);
    L.off_snap = o;    o = align_up(o + 3 * L.n * sizeof(double), kAlign);
    L.off_partial = o; o = align_up(o + (size_t)dugks::RED_BLOCKS * dugks::RED_VALS * sizeof(double), kAlign);
    L.off_redout = o;  o = align_up(o + 8 * sizeof(double), kAlign);
    L.off_status = o;  o = align_up(o + sizeof(unsigned), kAlign);
    L.total = o;
    return L;
}

template <typename Real>
Phys<Real> make_phys(const dugks_params &p) {
    Phys<Real> ph;
    std::memset(&ph, 0, sizeof ph);
    const double dt = p.cfl, h = 0.5 * dt, tau = p.mobility * 3.0;  // tau_f = M / RT (Eq. 34)
    ph.dt = Real(dt);
    ph.h = Real(h);
    ph.half_dt = Real(0.5 * dt);
    ph.half_h = Real(0.5 * h);
    ph.inv_dt = Real(1.0 / dt);
    ph.pf_a = Real((2 * tau - h) / (2 * tau + dt));  // Eq. 29
    ph.pf_b = Real(3 * h / (2 * tau + dt));
    ph.pf_c = Real(3 * tau * h / (2 * tau + dt));
    ph.ff_a = Real(2 * tau / (2 * tau + h));         // Eq. 28
    ph.ff_b = Real(h / (2 * tau + h));
    ph.ff_c = Real(tau * h / (2 * tau + h));
    ph.beta4 = Real(4.0 * 12.0 * p.sigma / p.width); // Eq. 3
    ph.kappa = Real(1.5 * p.sigma * p.width);
    ph.theta_k = Real(4.0 / p.width);                // Eq. 6 with phi_H = 1, phi_L = 0
    if (p.model == DUGKS_COUPLED) {
        ph.drho = Real(p.rho_h - p.rho_l);
        ph.rho_l = Real(p.rho_l);
        if (p.visc_interp == DUGKS_VISC_LINEAR) {
            ph.visc_a = Real(p.mu_h - p.mu_l);
            ph.visc_b = Real(p.mu_l);
        } else {
            ph.visc_a = Real(1.0 / p.mu_h - 1.0 / p.mu_l);
            ph.visc_b = Real(1.0 / p.mu_l);
        }
        ph.gx = Real(p.gx);
        ph.gy = Real(p.gy);
        ph.rho_ref = Real(p.rho_ref);
    }
    ph.phi_ref = Real(p.phi_ref);
    ph.p_ref = Real(p.p_ref);
    ph.u0x = Real(p.u0x);
    ph.u0y = Real(p.u0y);
    ph.vel_kind = p.model == DUGKS_AC_PRESCRIBED_U ? p.velocity_field : 0;
    if (ph.vel_kind >= 1 && ph.vel_kind <= 3) {
        ph.vel_u = Real(p.vel_u0);
        ph.vel_il = Real(1.0 / p.vel_length);
        ph.vel_ul = Real(p.vel_u0 / p.vel_length);
        ph.vel_tr = p.vel_length / p.vel_u0;
    }
    ph.visc_linear = p.visc_interp == DUGKS_VISC_LINEAR;
    ph.grav_mode = p.gravity_mode;
    return ph;
}

dugks_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return DUGKS_OK;
    return e == cudaErrorMemoryAllocation ? DUGKS_ERR_OOM : DUGKS_ERR_CUDA;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

// 3-D map over [planes][ny][pitch] (extent nx in x) with a box of
// (box_x, box_y, planes) elements.  Returns false if unavailable.
bool make_box_map(CUtensorMap *m, void *base, bool f64, int nx, int ny, int pitch, int planes, int box_x, int box_y) {
    std::memset(m, 0, sizeof *m);
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || box_x > 256 || box_y > 256 || planes > 256) return false;
    const size_t elt = f64 ? 8 : 4;
    cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)planes};
    cuuint64_t strides[2] = {(cuuint64_t)pitch * elt, (cuuint64_t)pitch * elt * (cuuint64_t)ny};
    cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, (cuuint32_t)planes};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(m, f64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides,
                     box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace



namespace {

// Waits for the stream and folds the device status word into a status code.
dugks_status sync_status(dugks_ctx *c) {
    unsigned s = 0;
    cudaError_t e = cudaMemcpyAsync(&s, c->status(), sizeof s, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return from_cuda(e);
    c->status_seen |= s;
    if (c->status_seen & dugks::STATUS_BOUNDS) return DUGKS_ERR_BOUNDS;
    if (c->status_seen & dugks::STATUS_TIMEOUT) return DUGKS_ERR_TIMEOUT;
    if (c->status_seen & dugks::STATUS_NONFINITE) return DUGKS_ERR_NONFINITE;
    if (c->status_seen & dugks::STATUS_NONPHYSICAL) return DUGKS_ERR_NONPHYSICAL;
    return DUGKS_OK;
}

cudaError_t run_macros(dugks_ctx *c, double *ophi, double *op, double *oux, double *ouy) {
    if (c->fp32)
        return dugks::launch_macros<float>(c->fields<float>(), c->phid(), c->phd, c->coupled, c->wally, ophi, op, oux,
                                           ouy, c->st);
    return dugks::launch_macros<double>(c->fields<double>(), c->phid(), c->phd, c->coupled, c->wally, ophi, op, oux,
                                        ouy, c->st);
}

}  // namespace

namespace {
// Uploads the sampled velocity field (R15) as [4][ny][pitch] values of the
// storage type: cell ux, uy, then the optional face normals (zero if absent).
template <typename Real>
cudaError_t upload_velocity_t(dugks_ctx *c, const double *uxc, const double *uyc, const double *uxf,
                              const double *uyf) {
    const int nx = c->P.nx, ny = c->P.ny, pitch = c->L.pitch;
    const size_t plane = c->L.plane;
    std::vector<Real> h(4 * plane, Real(0));
    const double *src[4] = {uxc, uyc, uxf, uyf};
    for (int q = 0; q < 4; q++) {
        if (!src[q]) continue;
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) h[q * plane + (size_t)y * pitch + x] = Real(src[q][(size_t)y * nx + x]);
    }
    cudaError_t e = cudaMemcpyAsync(c->vel(), h.data(), h.size() * sizeof(Real), cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e == cudaSuccess) c->vel_faces = uxf ? 1 : 0;
    return e;
}

cudaError_t upload_velocity(dugks_ctx *c, const double *uxc, const double *uyc, const double *uxf,
                            const double *uyf) {
    return c->fp32 ? upload_velocity_t<float>(c, uxc, uyc, uxf, uyf) : upload_velocity_t<double>(c, uxc, uyc, uxf, uyf);
}

}  // namespace

extern "C" {

size_t dugks_workspace_bytes(const dugks_params *params) {
    if (!valid(params)) return 0;
    return layout(params).total;
}

dugks_status dugks_create(const dugks_params *params, const double *phi0, const double *ux0, const double *uy0,
                          const double *p0, void *device_workspace, size_t ws_bytes, void *cuda_stream,
                          dugks_handle *out) {
    dugks::TraceRange trace_("dugks_create");
    if (!out) return DUGKS_ERR_ARG;
    *out = nullptr;
    if (!valid(params) || !phi0) return DUGKS_ERR_ARG;
    if (params->bc_x != DUGKS_BC_PERIODIC) return DUGKS_ERR_UNSUPPORTED;
    if (params->recon == DUGKS_RECON_UPWIND && params->tile_shape > 1) return DUGKS_ERR_UNSUPPORTED;
    const Layout L = layout(params);
    if (device_workspace && (reinterpret_cast<uintptr_t>(device_workspace) % kAlign)) return DUGKS_ERR_ARG;
    if (device_workspace && ws_bytes < L.total) return DUGKS_ERR_OOM;

    dugks_ctx *c = new (std::nothrow) dugks_ctx();
    if (!c) return DUGKS_ERR_OOM;
    c->P = *params;
    c->L = L;
    c->fp32 = params->precision == DUGKS_FP32_SHIFTED;
    c->coupled = params->model == DUGKS_COUPLED;
    c->wally = params->bc_y == DUGKS_BC_WALL;
    c->tile = params->tile_shape > 0 ? params->tile_shape - 1 : 0;
    c->upw = params->recon == DUGKS_RECON_UPWIND;
    c->st = static_cast<cudaStream_t>(cuda_stream);
    c->cur = 0;
    c->steps = 0;
    c->have_snap = 0;
    c->status_seen = 0;
    c->phd = make_phys<double>(*params);
    c->phf = make_phys<float>(*params);
    if (device_workspace) {
        c->ws = static_cast<unsigned char *>(device_workspace);
        c->owns = false;
    } else {
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, L.total);
        if (e != cudaSuccess) {
            delete c;
            return from_cuda(e);
        }
        c->ws = static_cast<unsigned char *>(p);
        c->owns = true;
    }

    {
        const int tx = c->fp32 ? dugks::tile_dim<float>(c->tile, 0) : dugks::tile_dim<double>(c->tile, 0);
        const int box_rows = c->fp32 ? dugks::step_box_rows<float>(c->tile, c->upw)
                                     : dugks::step_box_rows<double>(c->tile, c->upw);
        c->tma_ok = true;
        for (int b = 0; b < 2; b++) {
            c->tma_ok = c->tma_ok && make_box_map(&c->tm_state[b], c->state(b), !c->fp32, params->nx, params->ny,
                                                  L.pitch, L.nq, tx + 8, box_rows);
            c->tma_ok = c->tma_ok && make_box_map(&c->tm_hist[b], c->hist(b), !c->fp32, params->nx, params->ny,
                                                  L.pitch, 2, tx + 8, box_rows);
        }
    }
    cudaError_t e = cudaMemsetAsync(c->ws, 0, L.off_stage, c->st);  // state, history (incl. row padding)
    const size_t fb = L.n * sizeof(double);
    double *in = c->stage();
    const double *src[4] = {phi0, ux0, uy0, p0};
    for (int i = 0; i < 4 && e == cudaSuccess; i++) {
        if (src[i] && (i == 0 || c->coupled || (c->L.vel_bytes && i < 3)))
            e = cudaMemcpyAsync(in + i * L.n, src[i], fb, cudaMemcpyHostToDevice, c->st);
        else
            e = cudaMemsetAsync(in + i * L.n, 0, fb, c->st);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(c->status(), 0, sizeof(unsigned), c->st);
    if (e == cudaSuccess) {
        if (c->fp32)
            e = dugks::launch_init<float>(in, static_cast<float *>(c->state(0)), static_cast<float *>(c->hist(0)),
                                          params->nx, params->ny, L.pitch, (long long)L.plane, c->phd, c->coupled,
                                          c->wally, c->st);
        else
            e = dugks::launch_init<double>(in, static_cast<double *>(c->state(0)), static_cast<double *>(c->hist(0)),
                                           params->nx, params->ny, L.pitch, (long long)L.plane, c->phd, c->coupled,
                                           c->wally, c->st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e == cudaSuccess && L.vel_bytes) {
        // the sampled field starts as the cell velocity given here (zero where none)
        std::vector<double> zero(ux0 && uy0 ? 0 : L.n, 0.0);
        e = upload_velocity(c, ux0 ? ux0 : zero.data(), uy0 ? uy0 : zero.data(), nullptr, nullptr);
    }
    if (e != cudaSuccess) {
        if (c->owns) cudaFree(c->ws);
        delete c;
        return from_cuda(e);
    }
    *out = c;
    return DUGKS_OK;
}

dugks_status dugks_step(dugks_handle c, int64_t nsteps) {
    dugks::TraceRange trace_("dugks_step");
    if (!c || nsteps < 0) return DUGKS_ERR_ARG;
    return from_cuda(dugks::step_on(c, nsteps, c->st));
}

dugks_status dugks_macros(dugks_handle c, double *phi, double *p, double *ux, double *uy, int32_t dst_is_device) {
    dugks::TraceRange trace_("dugks_macros");
    if (!c) return DUGKS_ERR_ARG;
    cudaError_t e;
    if (dst_is_device) {
        e = run_macros(c, phi, p, ux, uy);
        return from_cuda(e);
    }
    double *s = c->stage();
    const size_t n = c->L.n;
    e = run_macros(c, s, s + n, s + 2 * n, s + 3 * n);
    double *dst[4] = {phi, p, ux, uy};
    for (int i = 0; i < 4 && e == cudaSuccess; i++)
        if (dst[i]) e = cudaMemcpyAsync(dst[i], s + i * n, n * sizeof(double), cudaMemcpyDeviceToHost, c->st);
    if (e != cudaSuccess) return from_cuda(e);
    return sync_status(c);
}

namespace {
// The FP64 sums of the macros over rows [row0, row0 + nrows) against the
// snapshot the previous reduction left, into r[RED_VALS] (*filled = 1 once
// they are there, also when the status word reports a failed step); then the
// whole grid becomes the new snapshot.  Synchronises.
dugks_status reduce_sums(dugks_handle c, int32_t row0, int32_t nrows, double *r, int *had_snap, int *filled) {
    *filled = 0;
    double *s = c->stage();
    const size_t n = c->L.n, off = (size_t)row0 * c->P.nx, m = (size_t)nrows * c->P.nx;
    cudaError_t e = run_macros(c, s, s + n, s + 2 * n, s + 3 * n);
    if (e == cudaSuccess)
        e = dugks::launch_reduce(s + off, s + 2 * n + off, s + 3 * n + off, c->snap() + off, (long long)m,
                                 (long long)n, c->have_snap, c->partial(), c->redout(), c->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(r, c->redout(), dugks::RED_VALS * sizeof(double), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->snap(), s, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->snap() + n, s + 2 * n, 2 * n * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
    if (e != cudaSuccess) return from_cuda(e);
    dugks_status st = sync_status(c);
    if (st == DUGKS_ERR_CUDA) return st;
    *filled = 1;
    *had_snap = c->have_snap;
    c->have_snap = 1;
    return st;
}
}  // namespace

dugks_status dugks_reduce_rows(dugks_handle c, int32_t row0, int32_t nrows, double *sums, int32_t *had_snapshot) {
    dugks::TraceRange trace_("dugks_reduce_rows");
    if (!c || !sums || nrows < 1 || row0 < 0 || row0 + nrows > c->P.ny) return DUGKS_ERR_ARG;
    double r[dugks::RED_VALS];
    int had = 0, filled = 0;
    dugks_status st = reduce_sums(c, row0, nrows, r, &had, &filled);
    if (!filled) return st;
    // [0] sum phi, [1] sum phi^2, [2] sum dphi^2, [3] sum |u|^2, [4] sum |du|^2, [5] max |u|
    for (int i = 0; i < dugks::RED_VALS; i++) sums[i] = r[i];
    if (!had) sums[2] = sums[4] = 0.0;
    if (had_snapshot) *had_snapshot = had;
    return st;
}

dugks_status dugks_reduce(dugks_handle c, double *phi_mass, double *resid_phi, double *resid_u, double *umax) {
    dugks::TraceRange trace_("dugks_reduce");
    if (!c) return DUGKS_ERR_ARG;
    double r[dugks::RED_VALS];
    int had = 0, filled = 0;
    dugks_status st = reduce_sums(c, 0, c->P.ny, r, &had, &filled);
    if (!filled) return st;
    if (phi_mass) *phi_mass = r[0];
    if (resid_phi) *resid_phi = had ? (r[1] > 0 ? r[2] / r[1] : 0.0) : 1.0;
    if (resid_u) *resid_u = had ? (r[3] > 0 ? r[4] / r[3] : 0.0) : 1.0;
    if (umax) *umax = r[5];
    return st;
}

dugks_status dugks_get_distributions(dugks_handle c, double *f, double *g, double *phiu_prev) {
    if (!c) return DUGKS_ERR_ARG;
    const size_t n = c->L.n;
    const int nq = c->L.nq;
    double *tmp = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&tmp), (size_t)(nq + 2) * n * sizeof(double), c->st);
    if (e != cudaSuccess) return from_cuda(e);
    if (c->fp32)
        e = dugks::launch_export<float>(c->fields<float>(), nq, c->P.phi_ref, c->P.p_ref, tmp, tmp + nq * n, c->st);
    else
        e = dugks::launch_export<double>(c->fields<double>(), nq, c->P.phi_ref, c->P.p_ref, tmp, tmp + nq * n, c->st);
    if (e == cudaSuccess && f) e = cudaMemcpyAsync(f, tmp, 9 * n * sizeof(double), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess && g) {
        if (c->coupled)
            e = cudaMemcpyAsync(g, tmp + 9 * n, 9 * n * sizeof(double), cudaMemcpyDeviceToHost, c->st);
        else
            std::memset(g, 0, 9 * n * sizeof(double));
    }
    if (e == cudaSuccess && phiu_prev)
        e = cudaMemcpyAsync(phiu_prev, tmp + nq * n, 2 * n * sizeof(double), cudaMemcpyDeviceToHost, c->st);
    cudaError_t e2 = cudaFreeAsync(tmp, c->st);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return from_cuda(e);
    return sync_status(c);
}

namespace {
struct StateHeader {
    uint64_t magic, version, nx, ny, nq, elt, model, precision, bc_y, steps;
};
}  // namespace

size_t dugks_state_bytes(dugks_handle c) {
    if (!c) return 0;
    return sizeof(StateHeader) + (size_t)(c->L.nq + 2) * c->L.n * c->L.elt;
}

dugks_status dugks_get_state(dugks_handle c, void *host_buf, size_t bytes) {
    if (!c || !host_buf || bytes < dugks_state_bytes(c)) return DUGKS_ERR_ARG;
    StateHeader hd = {kStateMagic, kStateVersion, (uint64_t)c->P.nx, (uint64_t)c->P.ny, (uint64_t)c->L.nq,
                      (uint64_t)c->L.elt, (uint64_t)c->P.model, (uint64_t)c->P.precision, (uint64_t)c->P.bc_y,
                      (uint64_t)c->steps};
    std::memcpy(host_buf, &hd, sizeof hd);
    unsigned char *dst = static_cast<unsigned char *>(host_buf) + sizeof hd;
    const size_t row = (size_t)c->P.nx * c->L.elt, dp = (size_t)c->L.pitch * c->L.elt;
    cudaError_t e = cudaMemcpy2DAsync(dst, row, c->state(c->cur), dp, row, (size_t)c->L.nq * c->P.ny,
                                      cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(dst + (size_t)c->L.nq * c->L.n * c->L.elt, row, c->hist(c->cur), dp, row,
                              (size_t)2 * c->P.ny, cudaMemcpyDeviceToHost, c->st);
    if (e != cudaSuccess) return from_cuda(e);
    return sync_status(c);
}

dugks_status dugks_set_state(dugks_handle c, const void *host_buf, size_t bytes) {
    if (!c || !host_buf || bytes < dugks_state_bytes(c)) return DUGKS_ERR_ARG;
    StateHeader hd;
    std::memcpy(&hd, host_buf, sizeof hd);
    if (hd.magic != kStateMagic || hd.version != kStateVersion || hd.nx != (uint64_t)c->P.nx ||
        hd.ny != (uint64_t)c->P.ny || hd.nq != (uint64_t)c->L.nq || hd.elt != (uint64_t)c->L.elt ||
        hd.model != (uint64_t)c->P.model || hd.precision != (uint64_t)c->P.precision ||
        hd.bc_y != (uint64_t)c->P.bc_y)
        return DUGKS_ERR_ARG;
    const unsigned char *src = static_cast<const unsigned char *>(host_buf) + sizeof hd;
    const size_t row = (size_t)c->P.nx * c->L.elt, dp = (size_t)c->L.pitch * c->L.elt;
    cudaError_t e = cudaMemcpy2DAsync(c->state(c->cur), dp, src, row, row, (size_t)c->L.nq * c->P.ny,
                                      cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(c->hist(c->cur), dp, src + (size_t)c->L.nq * c->L.n * c->L.elt, row, row,
                              (size_t)2 * c->P.ny, cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return from_cuda(e);
    c->steps = (int64_t)hd.steps;
    c->have_snap = 0;
    return DUGKS_OK;
}

size_t dugks_state_element_bytes(dugks_handle c) { return c ? c->L.elt : 0; }

namespace {
// Rows of the current state to (to_buf) or from a caller buffer: a kernel for
// device buffers, one 2-D copy per plane for host buffers (then synchronised).
dugks_status rows_copy(dugks_handle c, int32_t row0, int32_t nrows, void *buf, int32_t buf_is_device, int to_buf) {
    if (!c || !buf || nrows < 1 || row0 < 0 || row0 + nrows > c->P.ny) return DUGKS_ERR_ARG;
    const int nq = c->L.nq, nx = c->P.nx;
    const size_t elt = c->L.elt, row = (size_t)nx * elt, dp = (size_t)c->L.pitch * elt;
    cudaError_t e = cudaSuccess;
    if (buf_is_device) {
        e = dugks::launch_rows(c->state(c->cur), c->hist(c->cur), elt, nq, c->L.pitch, (long long)c->L.plane, nx,
                               row0, nrows, buf, to_buf, c->st);
    } else {
        for (int z = 0; z < nq + 2 && e == cudaSuccess; z++) {
            unsigned char *plane = static_cast<unsigned char *>(z < nq ? c->state(c->cur) : c->hist(c->cur)) +
                                   ((size_t)(z < nq ? z : z - nq) * c->L.plane + (size_t)row0 * c->L.pitch) * elt;
            unsigned char *hb = static_cast<unsigned char *>(buf) + (size_t)z * nrows * row;
            e = to_buf ? cudaMemcpy2DAsync(hb, row, plane, dp, row, nrows, cudaMemcpyDeviceToHost, c->st)
                       : cudaMemcpy2DAsync(plane, dp, hb, row, row, nrows, cudaMemcpyHostToDevice, c->st);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    }
    return from_cuda(e);
}
}  // namespace

dugks_status dugks_get_rows(dugks_handle c, int32_t row0, int32_t nrows, void *buf, int32_t buf_is_device) {
    dugks::TraceRange trace_("dugks_get_rows");
    return rows_copy(c, row0, nrows, buf, buf_is_device, 1);
}

dugks_status dugks_set_rows(dugks_handle c, int32_t row0, int32_t nrows, const void *buf, int32_t buf_is_device) {
    dugks::TraceRange trace_("dugks_set_rows");
    return rows_copy(c, row0, nrows, const_cast<void *>(buf), buf_is_device, 0);
}

int64_t dugks_step_count(dugks_handle c) { return c ? c->steps : -1; }

dugks_status dugks_sync(dugks_handle c) {
    if (!c) return DUGKS_ERR_ARG;
    return sync_status(c);
}

dugks_status dugks_destroy(dugks_handle c) {
    if (!c) return DUGKS_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(c->st);
    if (c->owns) {
        cudaError_t e2 = cudaFree(c->ws);
        if (e == cudaSuccess) e = e2;
    }
    delete c;
    return from_cuda(e);
}

dugks_status dugks_set_velocity_field(dugks_handle c, const double *ux_cell, const double *uy_cell,
                                      const double *ux_xface, const double *uy_yface) {
    if (!c || !ux_cell || !uy_cell || (!ux_xface) != (!uy_yface)) return DUGKS_ERR_ARG;
    if (!c->L.vel_bytes) return DUGKS_ERR_UNSUPPORTED;
    return from_cuda(upload_velocity(c, ux_cell, uy_cell, ux_xface, uy_yface));
}

dugks_status dugks_check_bounded_wait(int64_t max_polls, void *cuda_stream) {
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const long polls = max_polls > 0 ? (long)max_polls : dugks::kPollLimit;
    unsigned *d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(unsigned));
    if (e != cudaSuccess) return from_cuda(e);
    unsigned h = 0;
    e = cudaMemsetAsync(d, 0, sizeof(unsigned), st);
    if (e == cudaSuccess) {
        dugks::wait_probe_kernel<<<1, 32, 0, st>>>(polls, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof h, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d);
    if (e != cudaSuccess) return from_cuda(e);
    return (h & dugks::STATUS_TIMEOUT) ? DUGKS_ERR_TIMEOUT : DUGKS_OK;
}

dugks_status dugks_check_batch_wait(int64_t budget_ns, void *cuda_stream) {
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const unsigned long long budget = budget_ns > 0 ? (unsigned long long)budget_ns : dugks::kItemWaitNs;
    unsigned *d = nullptr;   // [0]: the counter nothing raises, [1]: status
    cudaError_t e = cudaMalloc(&d, 2 * sizeof(unsigned));
    if (e != cudaSuccess) return from_cuda(e);
    unsigned h = 0;
    e = cudaMemsetAsync(d, 0, 2 * sizeof(unsigned), st);
    if (e == cudaSuccess) {
        dugks::batch_wait_probe_kernel<<<1, 32, 0, st>>>(budget, d, d + 1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d + 1, sizeof h, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d);
    if (e != cudaSuccess) return from_cuda(e);
    return (h & dugks::STATUS_TIMEOUT) ? DUGKS_ERR_TIMEOUT : DUGKS_OK;
}

int32_t dugks_tile_shapes(int32_t precision, int32_t *tx, int32_t *ty, int32_t cap) {
    if (precision != DUGKS_FP64 && precision != DUGKS_FP32_SHIFTED) return -1;
    const bool f32 = precision == DUGKS_FP32_SHIFTED;
    const int n = f32 ? dugks::tile_count<float>() : dugks::tile_count<double>();
    for (int k = 0; k < n && k < cap; k++) {
        if (tx) tx[k] = f32 ? dugks::tile_dim<float>(k, 0) : dugks::tile_dim<double>(k, 0);
        if (ty) ty[k] = f32 ? dugks::tile_dim<float>(k, 1) : dugks::tile_dim<double>(k, 1);
    }
    return n;
}

dugks_status dugks_autotune(const dugks_params *params, const double *phi0, const double *ux0, const double *uy0,
                            const double *p0, int32_t trial_steps, void *cuda_stream, int32_t *best,
                            double *ms_per_step) {
    if (!best || !valid(params) || !phi0 || trial_steps < 1) return DUGKS_ERR_ARG;
    *best = 0;
    const int32_t n = dugks_tile_shapes(params->precision, nullptr, nullptr, 0);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return DUGKS_ERR_CUDA;
    }
    dugks_status worst = DUGKS_OK;
    float best_ms = 0.0f;
    for (int32_t k = 0; k < n; k++) {
        if (ms_per_step) ms_per_step[k] = -1.0;
        dugks_params q = *params;
        q.tile_shape = k + 1;
        dugks_handle h = nullptr;
        dugks_status r = dugks_create(&q, phi0, ux0, uy0, p0, nullptr, 0, cuda_stream, &h);
        float ms = 0.0f;
        if (r == DUGKS_OK) r = dugks_step(h, 2);   // warm-up: shared-memory attributes, caches
        if (r == DUGKS_OK && cudaEventRecord(e0, st) != cudaSuccess) r = DUGKS_ERR_CUDA;
        if (r == DUGKS_OK) r = dugks_step(h, trial_steps);
        if (r == DUGKS_OK && cudaEventRecord(e1, st) != cudaSuccess) r = DUGKS_ERR_CUDA;
        if (r == DUGKS_OK) r = dugks_sync(h);
        if (r == DUGKS_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) r = DUGKS_ERR_CUDA;
        if (h) {
            const dugks_status rd = dugks_destroy(h);
            if (r == DUGKS_OK) r = rd;
        }
        if (r != DUGKS_OK) {
            if (worst == DUGKS_OK) worst = r;
            continue;
        }
        ms /= (float)trial_steps;
        if (ms_per_step) ms_per_step[k] = ms;
        if (*best == 0 || ms < best_ms) {
            *best = k + 1;
            best_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return *best > 0 ? DUGKS_OK : worst;
}

const char *dugks_status_string(dugks_status s) {
    switch (s) {
    case DUGKS_OK: return "ok";
    case DUGKS_ERR_ARG: return "invalid argument";
    case DUGKS_ERR_OOM: return "out of device memory or workspace too small";
    case DUGKS_ERR_CUDA: return "CUDA runtime error";
    case DUGKS_ERR_NONFINITE: return "non-finite value produced by a step";
    case DUGKS_ERR_NONPHYSICAL: return "non-physical density or viscosity (<= 0)";
    case DUGKS_ERR_TIMEOUT: return "device wait timed out";
    case DUGKS_ERR_UNSUPPORTED: return "unsupported configuration";
    case DUGKS_ERR_BOUNDS: return "index out of range (bounds-checked build)";
    }
    return "unknown status";
}

}  // extern "C"
