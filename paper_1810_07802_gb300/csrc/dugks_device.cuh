// dugks_device.cuh -- device code of the GB300 phase-field DUGKS step.
//
// One time step of the two coupled D2Q9 kinetic models of arXiv:1810.07802,
// Sec. II.B (Allen-Cahn model for phi: Eqs. 12, 15-16; hydrodynamic model for
// p, u: Eqs. 13, 17-19) advanced by the DUGKS finite-volume update
// (Eqs. 20-30) with the closures of Eqs. 3-10 and 31-37, in one fused kernel
// per step.  Scheme details the paper leaves open are read as follows:
//   * RT = 1/3: xi_i = e_i and dt = CFL (Eq. 37, delta_x = 1).
//   * Central face reconstruction of psi-bar-plus at x_f - xi h (Eq. 27):
//     mean of the two cells, their difference as the normal slope, the mean
//     of their central differences as the tangential slope.
//   * Face macros: phi_f from f_bar; u_f, p_f from g_bar by Eqs. 32-33 with h
//     for dt; grad phi, lap phi and d_t(phi u) at the face are two-cell means.
//   * Isotropic D2Q9 gradient (1/RT) sum_i w_i xi_i phi(x + xi_i) and the
//     nine-point Laplacian [4(E+W+N+S) + (NE+NW+SE+SW) - 20 C] / 6.
//   * d_t(phi u) = ((phi u)^n - (phi u)^{n-1}) / dt, zero on the first step.
//   * n = grad phi / sqrt(|grad phi|^2 + 1e-16): the unit normal wherever an
//     interface is resolved, continuous where grad phi vanishes.
//   * No-slip walls on y = 0 and y = ny: phi mirrored into ghost rows;
//     one-sided y-slope for x-faces of the first/last row; at a wall face,
//     directions leaving the fluid or running along the wall are extrapolated
//     from the adjacent cell, directions entering it bounce back; the wall
//     face has u = 0 and no normal component of grad phi or d_t(phi u).
//
// Storage: distributions psi~ as deviations d_i = psi~_i - psi_ref_i from the
// rest state (f: w_i phi_ref; g: (p_ref/RT)(w_i - delta_i0)), structure of
// arrays [q][ny][pitch], x fastest.  Every linear step of the scheme keeps the
// rest state fixed (its weights sum to one), so the whole step is carried out
// on deviations; phi = phi_ref + sum_i d^f_i and p = p_ref + p' are formed
// only where the closures need absolute values.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dugks {

// D2Q9 in the paper's order (Eq. 14).  Folded to constants after unrolling.
__host__ __device__ constexpr int cx(int k) {
    return (k == 0 || k == 3 || k == 7) ? 0 : ((k == 1 || k == 2 || k == 8) ? 1 : -1);
}
__host__ __device__ constexpr int cy(int k) {
    return (k == 0 || k == 1 || k == 5) ? 0 : ((k == 2 || k == 3 || k == 4) ? 1 : -1);
}
__host__ __device__ constexpr int opp(int k) { return k == 0 ? 0 : ((k + 3) % 8) + 1; }
template <typename Real>
__host__ __device__ constexpr Real wq(int k) {
    return k == 0 ? Real(4) / Real(9) : ((k & 1) ? Real(1) / Real(9) : Real(1) / Real(36));
}
// Flux slots of the directions that cross x-faces (xi_x != 0) and y-faces (xi_y != 0).
__host__ __device__ constexpr int xslot(int k) {
    return k == 1 ? 0 : k == 2 ? 1 : k == 4 ? 2 : k == 5 ? 3 : k == 6 ? 4 : k == 8 ? 5 : -1;
}
__host__ __device__ constexpr int yslot(int k) {
    return k == 2 ? 0 : k == 3 ? 1 : k == 4 ? 2 : k == 6 ? 3 : k == 7 ? 4 : k == 8 ? 5 : -1;
}

enum : unsigned { STATUS_NONFINITE = 1u, STATUS_NONPHYSICAL = 2u };

// Constants of one problem, computed once on the host (passed by value).
template <typename Real>
struct Phys {
    Real dt, h, half_dt, half_h;
    Real pf_a, pf_b, pf_c;      // Eq. 29 coefficients for f (tau_f constant)
    Real ff_a, ff_b, ff_c;      // Eq. 28 coefficients for f
    Real beta4, kappa, theta_k; // 4 beta, kappa (Eq. 3), 4 / W (Eq. 6)
    Real drho, rho_l;           // rho = rho_l + drho phi (Eq. 10)
    Real visc_a, visc_b;        // 1/mu (Eq. 35) or mu (Eq. 36) = visc_a phi + visc_b
    Real gx, gy, rho_ref;
    Real phi_ref, p_ref;
    Real u0x, u0y;
    int visc_linear, grav_mode;
};

template <typename Real>
struct StepArgs {
    const Real *__restrict__ src;  // psi~^n  : [nq][ny][pitch]
    Real *__restrict__ dst;        // psi~^{n+1}
    const Real *__restrict__ hsrc; // (phi u)^{n-1} : [2][ny][pitch]
    Real *__restrict__ hdst;       // (phi u)^n
    int nx, ny, pitch;
    long long plane;               // ny * pitch
    int first_step;
    unsigned *status;
};

// Quantities at one point (cell centre or face).
template <typename Real>
struct Pt {
    Real phi, dpx, dpy, lap;
    Real rho, drx, dry, taug;
    Real theta, nx, ny;
    Real Fx, Fy, ux, uy, pd;  // pd = p - p_ref
    Real Dx, Dy;
};

__device__ __forceinline__ float rsqrt_r(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_r(double x) { return rsqrt(x); }
__device__ __forceinline__ bool finite_r(float x) { return isfinite(x); }
__device__ __forceinline__ bool finite_r(double x) { return isfinite(x); }

// theta, n (Eq. 6) and, for the coupled model, rho, mu_phi, mu, tau_g and F
// (Eqs. 3-4, 9-10, 34-36) from phi, grad phi and lap phi.
template <typename Real, bool COUPLED>
__device__ __forceinline__ void closures(const Phys<Real> &ph, Pt<Real> &s) {
    const Real phi = s.phi;
    s.theta = ph.theta_k * phi * (Real(1) - phi);
    const Real inv = rsqrt_r(s.dpx * s.dpx + s.dpy * s.dpy + Real(1e-16));
    s.nx = s.dpx * inv;
    s.ny = s.dpy * inv;
    if (COUPLED) {
        s.rho = ph.rho_l + ph.drho * phi;
        s.drx = ph.drho * s.dpx;
        s.dry = ph.drho * s.dpy;
        const Real muphi = ph.beta4 * phi * (phi - Real(1)) * (phi - Real(0.5)) - ph.kappa * s.lap;
        const Real lin = ph.visc_a * phi + ph.visc_b;
        const Real mu = ph.visc_linear ? lin : Real(1) / lin;
        s.taug = Real(3) * mu / s.rho;
        Real Gx = ph.gx, Gy = ph.gy;
        if (ph.grav_mode) {
            Gx = (s.rho - ph.rho_ref) * ph.gx;
            Gy = (s.rho - ph.rho_ref) * ph.gy;
        }
        s.Fx = muphi * s.dpx + Gx;
        s.Fy = muphi * s.dpy + Gy;
    }
}

// u and p' from the g moments (Eqs. 32-33; half = dt/2 at a cell, h/2 at a face).
template <typename Real>
__device__ __forceinline__ void velocity_pressure(Real mx, Real my, Real sn, Real half, Pt<Real> &s) {
    const Real irho = Real(1) / s.rho;
    s.ux = (mx + half * s.Fx) * irho;
    s.uy = (my + half * s.Fy) * irho;
    // RT/(1 - w0) = 3/5; rho (Gamma_0(u) - Gamma_0(0)) = -(2/3) rho |u|^2
    s.pd = Real(0.6) * (sn + half * (s.ux * s.drx + s.uy * s.dry)
                        - Real(2) / Real(3) * s.rho * (s.ux * s.ux + s.uy * s.uy));
}

// Deviation of f_eq (Eq. 15) and S^f (Eq. 16) in direction k.
template <typename Real>
__device__ __forceinline__ void f_eq_src(int k, const Phys<Real> &ph, const Pt<Real> &s, Real &eq, Real &src) {
    const Real w = wq<Real>(k);
    const Real ex = Real(cx(k)), ey = Real(cy(k));
    const Real eu = ex * s.ux + ey * s.uy;
    eq = w * ((s.phi - ph.phi_ref) + Real(3) * s.phi * eu);
    src = w * (s.theta * (ex * s.nx + ey * s.ny) + Real(3) * (ex * s.Dx + ey * s.Dy));
}

// Deviation of g_eq (Eqs. 17-18) and S^g (Eq. 19) in direction k.
template <typename Real>
__device__ __forceinline__ void g_eq_src(int k, const Pt<Real> &s, Real &eq, Real &src) {
    const Real w = wq<Real>(k);
    const Real ex = Real(cx(k)), ey = Real(cy(k));
    const Real eu = ex * s.ux + ey * s.uy;
    const Real usq = s.ux * s.ux + s.uy * s.uy;
    const Real gam = w * (Real(3) * eu + Real(4.5) * eu * eu - Real(1.5) * usq);  // Gamma_k(u) - w_k
    eq = Real(3) * s.pd * (k == 0 ? w - Real(1) : w) + s.rho * gam;
    const Real G = w + gam;
    src = (ex - s.ux) * (gam * s.drx + Real(3) * s.Fx * G) + (ey - s.uy) * (gam * s.dry + Real(3) * s.Fy * G);
}

__device__ __forceinline__ int wrap(int x, int n) {
    x %= n;
    return x < 0 ? x + n : x;
}
// Row index for phi stencils: periodic, or mirrored at the walls (rows far
// outside are clamped; no valid cell's stencil reaches them).
template <bool WALLY>
__device__ __forceinline__ int map_row(int y, int ny) {
    if (!WALLY) return wrap(y, ny);
    if (y < 0) y = -1 - y;
    if (y >= ny) y = 2 * ny - 1 - y;
    return y < 0 ? 0 : (y >= ny ? ny - 1 : y);
}

template <typename Real, int TX, int TY, bool COUPLED>
struct TileShape {
    static constexpr int NT = TX * TY;
    static constexpr int HX2 = TX + 4, HY2 = TY + 4;  // phi region (halo 2)
    static constexpr int HX1 = TX + 2, HY1 = TY + 2;  // psi-bar-plus region (halo 1)
    static constexpr int N2 = HX2 * HY2, N1 = HX1 * HY1;
    static constexpr int NQ = COUPLED ? 18 : 9;
    static constexpr int NFX = (TX + 1) * TY, NFY = TX * (TY + 1);
    static constexpr int NFD = COUPLED ? 12 : 6;  // flux slots per face
    static constexpr size_t off_phi = 0;
    static constexpr size_t off_bp = off_phi + N2;
    static constexpr size_t off_aux = off_bp + size_t(NQ) * N1;
    static constexpr size_t off_fx = off_aux + size_t(5) * N1;
    static constexpr size_t off_fy = off_fx + size_t(NFD) * NFX;
    static constexpr size_t smem_elems = off_fy + size_t(NFD) * NFY;
    static constexpr size_t smem_bytes = smem_elems * sizeof(Real);
};

// Central reconstruction (Eq. 27) of the 9 directions of one model whose
// psi-bar-plus planes are b[k * N1 + cell], at the face between cells L and
// R = L + nstride.  The tangential slope uses rows L +- tstride: tmode 0
// central, +1 one-sided towards +t, -1 one-sided towards -t.
template <typename Real, bool XFACE>
__device__ __forceinline__ void recon9(const Real *__restrict__ b, int N1, int L, int R, int tstride,
                                       int tmode, Real h, Real out[9]) {
#pragma unroll
    for (int k = 0; k < 9; k++) {
        const Real *p = b + k * N1;
        const Real A = p[L], B = p[R];
        Real st;
        if (tmode == 0)
            st = Real(0.25) * ((p[L + tstride] - p[L - tstride]) + (p[R + tstride] - p[R - tstride]));
        else if (tmode > 0)
            st = Real(0.5) * ((p[L + tstride] - A) + (p[R + tstride] - B));
        else
            st = Real(0.5) * ((A - p[L - tstride]) + (B - p[R - tstride]));
        const Real sn = B - A;
        const Real cn = Real(XFACE ? cx(k) : cy(k)), ct = Real(XFACE ? cy(k) : cx(k));
        out[k] = Real(0.5) * (A + B) - h * (cn * sn + ct * st);
    }
}

// Wall face, bottom (TOP == false) or top: linear extrapolation from cell c0
// (next cell into the fluid at c0 + inward) for directions leaving the fluid
// or tangential, bounce-back for directions entering it.
template <typename Real, bool TOP>
__device__ __forceinline__ void recon_wall9(const Real *__restrict__ b, int N1, int c0, int inward, Real h,
                                            Real out[9]) {
    const Real dyw = TOP ? Real(0.5) : Real(-0.5);
#pragma unroll
    for (int k = 0; k < 9; k++) {
        const bool keep = TOP ? (cy(k) >= 0) : (cy(k) <= 0);
        if (keep) {
            const Real *p = b + k * N1;
            const Real b0 = p[c0];
            const Real sx = Real(0.5) * (p[c0 + 1] - p[c0 - 1]);
            const Real sy = TOP ? (b0 - p[c0 + inward]) : (p[c0 + inward] - b0);
            out[k] = b0 + (-h * Real(cx(k))) * sx + (dyw - h * Real(cy(k))) * sy;
        }
    }
#pragma unroll
    for (int k = 0; k < 9; k++) {
        const bool enters = TOP ? (cy(k) < 0) : (cy(k) > 0);
        if (enters) out[k] = out[opp(k)];
    }
}

// Face state from f_bar, g_bar and the face values of the aux fields, then
// the original distributions (Eq. 28) of the directions crossing the face,
// written to out[slot * stride] (f slots 0..5, g slots 6..11).
template <typename Real, bool COUPLED, bool XFACE>
__device__ __forceinline__ void face_flux(const Phys<Real> &ph, const Real fb[9], const Real gb[9], Real dpx,
                                          Real dpy, Real lap, Real Dx, Real Dy, bool wall, Real *__restrict__ out,
                                          int stride) {
    Pt<Real> s;
    Real sphi = Real(0);
#pragma unroll
    for (int k = 0; k < 9; k++) sphi += fb[k];
    s.phi = ph.phi_ref + sphi;
    s.dpx = dpx;
    s.dpy = dpy;
    s.lap = lap;
    s.Dx = Dx;
    s.Dy = Dy;
    closures<Real, COUPLED>(ph, s);
    if (COUPLED) {
        Real mx = Real(0), my = Real(0), sn = Real(0);
#pragma unroll
        for (int k = 0; k < 9; k++) {
            mx += Real(cx(k)) * gb[k];
            my += Real(cy(k)) * gb[k];
            if (k) sn += gb[k];
        }
        if (wall) {
            s.ux = Real(0);
            s.uy = Real(0);
            s.pd = Real(0.6) * sn;
        } else {
            velocity_pressure(mx, my, sn, ph.half_h, s);
        }
    } else {
        s.ux = wall ? Real(0) : ph.u0x;
        s.uy = wall ? Real(0) : ph.u0y;
    }
#pragma unroll
    for (int k = 0; k < 9; k++) {
        const int slot = XFACE ? xslot(k) : yslot(k);
        if (slot >= 0) {
            Real eq, src;
            f_eq_src(k, ph, s, eq, src);
            out[slot * stride] = ph.ff_a * fb[k] + ph.ff_b * eq + ph.ff_c * src;
        }
    }
    if (COUPLED) {
        const Real inv = Real(1) / (Real(2) * s.taug + ph.h);
        const Real a = Real(2) * s.taug * inv, bb = ph.h * inv, c = s.taug * ph.h * inv;
#pragma unroll
        for (int k = 0; k < 9; k++) {
            const int slot = XFACE ? xslot(k) : yslot(k);
            if (slot >= 0) {
                Real eq, src;
                g_eq_src(k, s, eq, src);
                out[(6 + slot) * stride] = a * gb[k] + bb * eq + c * src;
            }
        }
    }
}

// Gradient and Laplacian of phi at smem index c of a row-major region of width W.
template <typename Real>
__device__ __forceinline__ void phi_stencils(const Real *__restrict__ p, int c, int W, Real &gx, Real &gy, Real &lp) {
    const Real C = p[c], E = p[c + 1], Wv = p[c - 1], N = p[c + W], S = p[c - W];
    const Real NE = p[c + W + 1], NW = p[c + W - 1], SE = p[c - W + 1], SW = p[c - W - 1];
    // (1/RT) sum_i w_i xi_i phi(x + xi_i)
    gx = (E - Wv) * Real(1.0 / 3.0) + ((NE + SE) - (NW + SW)) * Real(1.0 / 12.0);
    gy = (N - S) * Real(1.0 / 3.0) + ((NE + NW) - (SE + SW)) * Real(1.0 / 12.0);
    lp = (Real(4) * ((E + Wv) + (N + S)) + ((NE + NW) + (SE + SW)) - Real(20) * C) * Real(1.0 / 6.0);
}

// ---------------------------------------------------------------------------
// The fused step: one CTA per TX x TY tile, one thread per tile cell.
//   1. phi' = sum_i d^f_i on the tile + 2-cell halo (global -> smem)
//   2. cell macros, equilibria, sources and psi-bar-plus (Eq. 29) on the tile
//      + 1-cell halo (smem); (phi u)^n of the tile to global
//   3. every face of the tile: reconstruction (Eq. 27), face macros, Eq. 28
//   4. psi~+ (Eq. 30) and the flux update (Eq. 24) of the tile to global
// ---------------------------------------------------------------------------
template <typename Real, int TX, int TY, bool COUPLED, bool WALLY>
__global__ void __launch_bounds__(TX * TY)
step_kernel(StepArgs<Real> a, Phys<Real> ph) {
    using S = TileShape<Real, TX, TY, COUPLED>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Real *sm = reinterpret_cast<Real *>(smem_raw);
    Real *sphi = sm + S::off_phi;
    Real *sbp = sm + S::off_bp;
    Real *saux = sm + S::off_aux;
    Real *sfx = sm + S::off_fx;
    Real *sfy = sm + S::off_fy;

    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int nx = a.nx, ny = a.ny, pitch = a.pitch;
    const long long plane = a.plane;

    // 1. phi' on the halo-2 region
    for (int t = tid; t < S::N2; t += S::NT) {
        const int lx = t % S::HX2, ly = t / S::HX2;
        const int gx = wrap(x0 + lx - 2, nx);
        const int gy = map_row<WALLY>(y0 + ly - 2, ny);
        const Real *p = a.src + (long long)gy * pitch + gx;
        Real s = Real(0);
#pragma unroll
        for (int k = 0; k < 9; k++) s += p[k * plane];
        sphi[t] = s;
    }
    __syncthreads();

    // 2. cell macros and psi-bar-plus on the halo-1 region; item t < NT is tile cell t
    for (int t = tid; t < S::N1; t += S::NT) {
        int hx, hy;
        if (t < S::NT) {
            hx = t % TX + 1;
            hy = t / TX + 1;
        } else {
            const int r = t - S::NT;
            if (r < S::HX1) { hx = r; hy = 0; }
            else if (r < 2 * S::HX1) { hx = r - S::HX1; hy = S::HY1 - 1; }
            else if (r < 2 * S::HX1 + TY) { hx = 0; hy = r - 2 * S::HX1 + 1; }
            else { hx = S::HX1 - 1; hy = r - 2 * S::HX1 - TY + 1; }
        }
        const int c1 = hy * S::HX1 + hx;
        const int yraw = y0 + hy - 1;
        if (WALLY && (yraw < 0 || yraw >= ny)) {
#pragma unroll
            for (int k = 0; k < S::NQ; k++) sbp[k * S::N1 + c1] = Real(0);
#pragma unroll
            for (int k = 0; k < 5; k++) saux[k * S::N1 + c1] = Real(0);
            continue;
        }
        const int gx = wrap(x0 + hx - 1, nx);
        const int gy = WALLY ? yraw : wrap(yraw, ny);
        const long long g = (long long)gy * pitch + gx;

        Pt<Real> s;
        const int c2 = (hy + 1) * S::HX2 + (hx + 1);
        phi_stencils(sphi, c2, S::HX2, s.dpx, s.dpy, s.lap);
        s.phi = ph.phi_ref + sphi[c2];
        closures<Real, COUPLED>(ph, s);
        Real dg[9];
        if (COUPLED) {
            Real mx = Real(0), my = Real(0), sn = Real(0);
#pragma unroll
            for (int k = 0; k < 9; k++) {
                dg[k] = a.src[(9 + k) * plane + g];
                mx += Real(cx(k)) * dg[k];
                my += Real(cy(k)) * dg[k];
                if (k) sn += dg[k];
            }
            velocity_pressure(mx, my, sn, ph.half_dt, s);
        } else {
            s.ux = ph.u0x;
            s.uy = ph.u0y;
        }
        const Real phux = s.phi * s.ux, phuy = s.phi * s.uy;
        if (a.first_step) {
            s.Dx = Real(0);
            s.Dy = Real(0);
        } else {
            const Real idt = Real(1) / ph.dt;
            s.Dx = (phux - a.hsrc[g]) * idt;
            s.Dy = (phuy - a.hsrc[plane + g]) * idt;
        }
        saux[0 * S::N1 + c1] = s.dpx;
        saux[1 * S::N1 + c1] = s.dpy;
        saux[2 * S::N1 + c1] = s.lap;
        saux[3 * S::N1 + c1] = s.Dx;
        saux[4 * S::N1 + c1] = s.Dy;
#pragma unroll
        for (int k = 0; k < 9; k++) {
            Real eq, src;
            f_eq_src(k, ph, s, eq, src);
            const Real d = a.src[k * plane + g];
            sbp[k * S::N1 + c1] = ph.pf_a * d + ph.pf_b * eq + ph.pf_c * src;
        }
        if (COUPLED) {
            const Real inv = Real(1) / (Real(2) * s.taug + ph.dt);
            const Real ca = (Real(2) * s.taug - ph.h) * inv, cb = Real(3) * ph.h * inv, cc = Real(3) * s.taug * ph.h * inv;
#pragma unroll
            for (int k = 0; k < 9; k++) {
                Real eq, src;
                g_eq_src(k, s, eq, src);
                sbp[(9 + k) * S::N1 + c1] = ca * dg[k] + cb * eq + cc * src;
            }
        }
        if (t < S::NT && x0 + hx - 1 < nx && yraw < ny) {
            a.hdst[g] = phux;
            a.hdst[plane + g] = phuy;
            bool bad = !finite_r(s.phi) || !finite_r(s.ux) || !finite_r(s.uy);
            bool nonphys = COUPLED && !(s.rho > Real(0) && s.taug > Real(0));
            if (bad || nonphys) atomicOr(a.status, (bad ? STATUS_NONFINITE : 0u) | (nonphys ? STATUS_NONPHYSICAL : 0u));
        }
    }
    __syncthreads();

    // 3. faces: x-faces (west face of local cell (fx, fy)), then y-faces (south face)
    for (int t = tid; t < S::NFX + S::NFY; t += S::NT) {
        Real fb[9], gb[9];
        if (t < S::NFX) {
            const int fx = t % (TX + 1), fy = t / (TX + 1);
            const int gyr = y0 + fy;
            if (gyr >= ny || x0 + fx - 1 >= nx) continue;
            const int L = (fy + 1) * S::HX1 + fx, R = L + 1;
            int tmode = 0;
            if (WALLY) tmode = (gyr == 0) ? 1 : ((gyr == ny - 1) ? -1 : 0);
            recon9<Real, true>(sbp, S::N1, L, R, S::HX1, tmode, ph.h, fb);
            if (COUPLED) recon9<Real, true>(sbp + 9 * S::N1, S::N1, L, R, S::HX1, tmode, ph.h, gb);
            const Real hf = Real(0.5);
            face_flux<Real, COUPLED, true>(
                ph, fb, gb, hf * (saux[L] + saux[R]), hf * (saux[S::N1 + L] + saux[S::N1 + R]),
                hf * (saux[2 * S::N1 + L] + saux[2 * S::N1 + R]), hf * (saux[3 * S::N1 + L] + saux[3 * S::N1 + R]),
                hf * (saux[4 * S::N1 + L] + saux[4 * S::N1 + R]), false, sfx + t, S::NFX);
        } else {
            const int u = t - S::NFX;
            const int fx = u % TX, fy = u / TX;
            const int gyf = y0 + fy;  // face below row gyf
            if (x0 + fx >= nx || gyf - 1 >= ny) continue;
            const int D = fy * S::HX1 + fx + 1, U = D + S::HX1;
            if (WALLY && (gyf == 0 || gyf == ny)) {
                const bool top = (gyf == ny);
                const int c0 = top ? D : U;
                if (top) {
                    recon_wall9<Real, true>(sbp, S::N1, c0, -S::HX1, ph.h, fb);
                    if (COUPLED) recon_wall9<Real, true>(sbp + 9 * S::N1, S::N1, c0, -S::HX1, ph.h, gb);
                } else {
                    recon_wall9<Real, false>(sbp, S::N1, c0, S::HX1, ph.h, fb);
                    if (COUPLED) recon_wall9<Real, false>(sbp + 9 * S::N1, S::N1, c0, S::HX1, ph.h, gb);
                }
                face_flux<Real, COUPLED, false>(ph, fb, gb, saux[c0], Real(0), saux[2 * S::N1 + c0],
                                                saux[3 * S::N1 + c0], Real(0), true, sfy + u, S::NFY);
            } else {
                recon9<Real, false>(sbp, S::N1, D, U, 1, 0, ph.h, fb);
                if (COUPLED) recon9<Real, false>(sbp + 9 * S::N1, S::N1, D, U, 1, 0, ph.h, gb);
                const Real hf = Real(0.5);
                face_flux<Real, COUPLED, false>(
                    ph, fb, gb, hf * (saux[D] + saux[U]), hf * (saux[S::N1 + D] + saux[S::N1 + U]),
                    hf * (saux[2 * S::N1 + D] + saux[2 * S::N1 + U]), hf * (saux[3 * S::N1 + D] + saux[3 * S::N1 + U]),
                    hf * (saux[4 * S::N1 + D] + saux[4 * S::N1 + U]), false, sfy + u, S::NFY);
            }
        }
    }
    __syncthreads();

    // 4. psi~+ = 4/3 psi-bar-plus - 1/3 psi~ and the flux update of the tile
    {
        const int lx = tid % TX, ly = tid / TX;
        const int gx = x0 + lx, gy = y0 + ly;
        if (gx < nx && gy < ny) {
            const long long g = (long long)gy * pitch + gx;
            const int c1 = (ly + 1) * S::HX1 + lx + 1;
            const int fw = ly * (TX + 1) + lx, fe = fw + 1;  // x-faces
            const int fs = ly * TX + lx, fn = fs + TX;       // y-faces
#pragma unroll
            for (int k = 0; k < S::NQ; k++) {
                const int kk = k % 9, base = (k < 9) ? 0 : 6;
                const Real d = a.src[k * plane + g];
                const Real tp = Real(4.0 / 3.0) * sbp[k * S::N1 + c1] - Real(1.0 / 3.0) * d;
                Real flux = Real(0);
                if (cx(kk) != 0) {
                    const Real *q = sfx + (base + xslot(kk)) * S::NFX;
                    flux += Real(cx(kk)) * (q[fe] - q[fw]);
                }
                if (cy(kk) != 0) {
                    const Real *q = sfy + (base + yslot(kk)) * S::NFY;
                    flux += Real(cy(kk)) * (q[fn] - q[fs]);
                }
                a.dst[k * plane + g] = tp - ph.dt * flux;
            }
        }
    }
}

}  // namespace dugks
