// dugks_aux.cuh -- initial state, cell macros and state export of the GB300
// phase-field DUGKS library.  All of these run in FP64 arithmetic whatever
// the storage precision.
#pragma once

#include "dugks_device.cuh"

namespace dugks {

template <typename Real>
struct FieldArgs {
    const Real *__restrict__ state;   // [nq][ny][pitch] deviations
    const Real *__restrict__ hist;    // [2][ny][pitch]
    int nx, ny, pitch;
    long long plane;
    double t;                         // time of the state (prescribed velocity fields)
    const Real *__restrict__ vel;     // sampled velocity field [4][ny][pitch] (velocity field 4), or null
};

// phi at cell (x, y) of a [ny][nx] double field, periodic in x, periodic or
// mirrored in y.
template <bool WALLY>
__device__ __forceinline__ double phi_at(const double *__restrict__ phi, int nx, int ny, int x, int y) {
    return phi[(long long)map_row<WALLY>(y, ny) * nx + wrap(x, nx)];
}

template <bool WALLY>
__device__ __forceinline__ void phi_stencils_global(const double *__restrict__ p, int nx, int ny, int x, int y,
                                                    double &gx, double &gy, double &lp) {
    const double C = phi_at<WALLY>(p, nx, ny, x, y);
    const double E = phi_at<WALLY>(p, nx, ny, x + 1, y), Wv = phi_at<WALLY>(p, nx, ny, x - 1, y);
    const double N = phi_at<WALLY>(p, nx, ny, x, y + 1), S = phi_at<WALLY>(p, nx, ny, x, y - 1);
    const double NE = phi_at<WALLY>(p, nx, ny, x + 1, y + 1), NW = phi_at<WALLY>(p, nx, ny, x - 1, y + 1);
    const double SE = phi_at<WALLY>(p, nx, ny, x + 1, y - 1), SW = phi_at<WALLY>(p, nx, ny, x - 1, y - 1);
    gx = (E - Wv) * (1.0 / 3.0) + ((NE + SE) - (NW + SW)) * (1.0 / 12.0);
    gy = (N - S) * (1.0 / 3.0) + ((NE + NW) - (SE + SW)) * (1.0 / 12.0);
    lp = (4.0 * ((E + Wv) + (N + S)) + ((NE + NW) + (SE + SW)) - 20.0 * C) * (1.0 / 6.0);
}

// Initial state psi~0 = psi_eq - dt/2 S with d_t(phi u) = 0 (Eq. 23a with
// psi = psi_eq), and (phi u)^{-1} = phi0 u0.  in: phi0, ux0, uy0, p0 as
// [4][ny][nx] doubles (ux0, uy0, p0 zero where the caller gave none).
template <typename Real, bool COUPLED, bool WALLY>
__global__ void init_kernel(const double *__restrict__ in, Real *__restrict__ state, Real *__restrict__ hist,
                            int nx, int ny, int pitch, long long plane, Phys<double> ph) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= nx || y >= ny) return;
    const long long N = (long long)nx * ny, c = (long long)y * nx + x;
    const long long g = (long long)y * pitch + x;
    Pt<double> s;
    phi_stencils_global<WALLY>(in, nx, ny, x, y, s.dpx, s.dpy, s.lap);
    s.phi = in[c];
    closures<double, COUPLED>(ph, s);
    if (COUPLED) {
        s.ux = in[N + c];
        s.uy = in[2 * N + c];
        s.pd = in[3 * N + c] - ph.p_ref;
    } else if (ph.vel_kind == 4) {   // sampled field: the cell velocity given at creation
        s.ux = in[N + c];
        s.uy = in[2 * N + c];
    } else {
        prescribed_velocity(ph, double(x) + 0.5, double(y) + 0.5, 0.0, s.ux, s.uy);
    }
    s.Dx = 0.0;
    s.Dy = 0.0;
    const FLin<double> lf = f_lin(ph, s, 1.0, -0.5 * ph.dt);   // f_eq - dt/2 S^f
#pragma unroll
    for (int k = 0; k < 9; k++) state[k * plane + g] = Real(f_lin_k(k, lf));
    if (COUPLED) {
        const GCoef<double> gc = g_coef(s);
#pragma unroll
        for (int k = 0; k < 9; k++) {
            double eq, src;
            g_eq_src(k, s, gc, eq, src);
            state[(9 + k) * plane + g] = Real(eq - 0.5 * ph.dt * src);
        }
    }
    hist[g] = Real(s.phi * s.ux);
    hist[plane + g] = Real(s.phi * s.uy);
}

// phi' = sum_i d^f_i per cell, in FP64 (Eq. 31 on deviations).
template <typename Real>
__global__ void phi_kernel(FieldArgs<Real> a, double *__restrict__ phid) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    const long long g = (long long)y * a.pitch + x;
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 9; k++) s += double(a.state[k * a.plane + g]);
    phid[(long long)y * a.nx + x] = s;
}

// Cell-centre macros (Eqs. 31-33) in FP64 from phi' and the g deviations.
// out: phi, p, ux, uy planes of [ny][nx] (a NULL plane is skipped).
template <typename Real, bool COUPLED, bool WALLY>
__global__ void macro_kernel(FieldArgs<Real> a, const double *__restrict__ phid, Phys<double> ph,
                             double *__restrict__ ophi, double *__restrict__ op, double *__restrict__ oux,
                             double *__restrict__ ouy) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    const long long c = (long long)y * a.nx + x, g = (long long)y * a.pitch + x;
    Pt<double> s;
    phi_stencils_global<WALLY>(phid, a.nx, a.ny, x, y, s.dpx, s.dpy, s.lap);
    s.phi = ph.phi_ref + phid[c];
    closures<double, COUPLED>(ph, s);
    if (COUPLED) {
        double mx = 0.0, my = 0.0, sn = 0.0;
#pragma unroll
        for (int k = 0; k < 9; k++) {
            const double d = double(a.state[(9 + k) * a.plane + g]);
            mx += double(cx(k)) * d;
            my += double(cy(k)) * d;
            if (k) sn += d;
        }
        velocity_pressure(mx, my, sn, ph.half_dt, s);
    } else if (ph.vel_kind == 4) {
        s.ux = double(a.vel[g]);
        s.uy = double(a.vel[a.plane + g]);
        s.pd = 0.0;
    } else {
        prescribed_velocity(ph, double(x) + 0.5, double(y) + 0.5, a.t, s.ux, s.uy);
        s.pd = 0.0;
    }
    if (ophi) ophi[c] = s.phi;
    if (op) op[c] = ph.p_ref + s.pd;
    if (oux) oux[c] = s.ux;
    if (ouy) ouy[c] = s.uy;
}

// Absolute FP64 distributions [nq][ny][nx] and history [2][ny][nx].
template <typename Real>
__global__ void export_kernel(FieldArgs<Real> a, int nq, double phi_ref, double p_ref, double *__restrict__ dist,
                              double *__restrict__ hist_out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    const long long N = (long long)a.nx * a.ny, c = (long long)y * a.nx + x, g = (long long)y * a.pitch + x;
    for (int k = 0; k < nq; k++) {
        const int kk = k % 9;
        const double w = wq<double>(kk);
        const double ref = (k < 9) ? w * phi_ref : 3.0 * p_ref * (kk == 0 ? w - 1.0 : w);
        dist[k * N + c] = ref + double(a.state[k * a.plane + g]);
    }
    hist_out[c] = double(a.hist[g]);
    hist_out[N + c] = double(a.hist[a.plane + g]);
}

}  // namespace dugks
