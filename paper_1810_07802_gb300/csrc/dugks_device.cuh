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
//   * Prescribed velocity of the Allen-Cahn-only model (Eqs. 40-43): at cell
//     centres at t_n, at face centres at t_n + h, face coordinates on
//     periodic axes taken in [0, n); or sampled arrays (cells, optional face
//     normals; otherwise faces take the mean of their two cells).
//   * Upwind reconstruction (optional): each cell of a face carries a linear
//     profile with van Leer-limited slopes; a direction takes the profile of
//     the cell it leaves, one along the face the mean of both.  With walls a
//     cell next to a wall takes its one-sided y-difference into the fluid,
//     and the wall face takes the adjacent cell's profile for directions
//     leaving the fluid or running along the wall, bounce-back for the rest.
//
// Storage: distributions psi~ as deviations d_i = psi~_i - psi_ref_i from the
// rest state (f: w_i phi_ref; g: (p_ref/RT)(w_i - delta_i0)), structure of
// arrays [q][ny][pitch], x fastest.  Every linear step of the scheme keeps the
// rest state fixed (its weights sum to one), so the whole step is carried out
// on deviations; phi = phi_ref + sum_i d^f_i and p = p_ref + p' are formed
// only where the closures need absolute values.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

// FP32 arithmetic on pairs of lanes (one packed FFMA2 / FADD2 / FMUL2
// instruction for two values) in the phi' sums, the face reconstruction and
// the cell pre-step; 0 keeps every FP32 operation scalar.  (Packing the face
// distributions of Eq. 28 as well measured slower on GB300: 0.298 vs 0.288 ms
// per 2048^2 step, more register moves and spills.)
#ifndef DUGKS_PACKED_F32
#define DUGKS_PACKED_F32 1
#endif

namespace dugks {

// D2Q9 in the paper's order (Eq. 14).  Folded to constants after unrolling.
__host__ __device__ constexpr int cx(int k) {
    return (k == 0 || k == 3 || k == 7) ? 0 : ((k == 1 || k == 2 || k == 8) ? 1 : -1);
}
__host__ __device__ constexpr int cy(int k) {
    return (k == 0 || k == 1 || k == 5) ? 0 : ((k == 2 || k == 3 || k == 4) ? 1 : -1);
}
__host__ __device__ constexpr int opp(int k) { return k == 0 ? 0 : ((k + 3) % 8) + 1; }
// D2Q9 weights (Eq. 14).  In FP32 the diagonal weight is 1/36 rounded down by
// one unit in the last place, so that the nine FP32 weights sum to exactly 1
// and no rounding bias enters the phi mass through the equilibria.
template <typename Real>
__host__ __device__ constexpr Real wq(int k) {
    return k == 0 ? Real(4) / Real(9) : ((k & 1) ? Real(1) / Real(9) : Real(1) / Real(36));
}
template <>
__host__ __device__ constexpr float wq<float>(int k) {
    return k == 0 ? 4.0f / 9.0f : ((k & 1) ? 1.0f / 9.0f : 0x1.c71c70p-6f);
}
// Flux slots of the directions that cross x-faces (xi_x != 0) and y-faces (xi_y != 0).
__host__ __device__ constexpr int xslot(int k) {
    return k == 1 ? 0 : k == 2 ? 1 : k == 4 ? 2 : k == 5 ? 3 : k == 6 ? 4 : k == 8 ? 5 : -1;
}
__host__ __device__ constexpr int yslot(int k) {
    return k == 2 ? 0 : k == 3 ? 1 : k == 4 ? 2 : k == 6 ? 3 : k == 7 ? 4 : k == 8 ? 5 : -1;
}

// a * x for a in {-1, 0, 1}.  IEEE rules forbid the compiler from folding
// 0 * x or 0 - x, so every product with a lattice-velocity component is
// written out case by case (k is a compile-time constant after unrolling).
template <typename Real>
__device__ __forceinline__ Real sgnmul(int a, Real x) { return a > 0 ? x : -x; }
// xi_k . (x, y) for k != 0.
template <typename Real>
__device__ __forceinline__ Real edot(int k, Real x, Real y) {
    const int a = cx(k), b = cy(k);
    if (a == 0) return sgnmul(b, y);
    if (b == 0) return sgnmul(a, x);
    return b > 0 ? sgnmul(a, x) + y : sgnmul(a, x) - y;
}
// xi_k,a - u for a component a in {-1, 0, 1}.
template <typename Real>
__device__ __forceinline__ Real eminus(int a, Real u) { return a == 0 ? -u : (a > 0 ? Real(1) - u : Real(-1) - u); }

enum : unsigned { STATUS_NONFINITE = 1u, STATUS_NONPHYSICAL = 2u, STATUS_TIMEOUT = 4u, STATUS_BOUNDS = 8u };

// Bounds-checked build (-DDUGKS_BOUNDS_CHECK=1, a stand-in for a memory
// sanitizer): every computed index of the step kernel is checked before its
// access; a violation sets STATUS_BOUNDS in the status word (no trap) and
// the access is skipped.  In the normal build the checks compile away.
#ifndef DUGKS_BOUNDS_CHECK
#define DUGKS_BOUNDS_CHECK 0
#endif
__device__ __forceinline__ bool in_bounds(bool ok, unsigned *status) {
#if DUGKS_BOUNDS_CHECK
    if (!ok) atomicOr(status, STATUS_BOUNDS);
    return ok;
#else
    (void)ok;
    (void)status;
    return true;
#endif
}

// Constants of one problem, computed once on the host (passed by value).
template <typename Real>
struct Phys {
    Real dt, h, half_dt, half_h, inv_dt;
    Real pf_a, pf_b, pf_c;      // Eq. 29 coefficients for f (tau_f constant)
    Real ff_a, ff_b, ff_c;      // Eq. 28 coefficients for f
    Real beta4, kappa, theta_k; // 4 beta, kappa (Eq. 3), 4 / W (Eq. 6)
    Real drho, rho_l;           // rho = rho_l + drho phi (Eq. 10)
    Real visc_a, visc_b;        // 1/mu (Eq. 35) or mu (Eq. 36) = visc_a phi + visc_b
    Real gx, gy, rho_ref;
    Real phi_ref, p_ref;
    Real u0x, u0y;
    int visc_linear, grav_mode;
    int vel_kind;                 // prescribed field of the A-C-only model (0 uniform, 1-3 analytic, 4 sampled)
    Real vel_u, vel_il, vel_ul;   // U0, 1/L0, U0/L0
    double vel_tr;                // reversal time L0/U0 of the shear field
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
    double t_n;                    // time at the start of the step
    int small;                     // grid smaller than a tile plus halo: wrap with %
    int use_tma;                   // tensor maps are valid: interior tiles load by TMA
    const Real *__restrict__ vel;  // sampled velocity field [4][ny][pitch]: cell ux, uy, x-face ux, y-face uy
    int vel_faces;                 // the face planes of vel are set (else faces take the mean of their cells)
    unsigned *status;
};

// Quantities at one point (cell centre or face).
template <typename Real>
struct Pt {
    Real phi, dpx, dpy, lap;
    Real rho, irho, drx, dry, taug;
    Real inv;                 // FP64: 1 / (2 tau_g + step), see closures
    Real theta, nx, ny;
    Real Fx, Fy, ux, uy, pd;  // pd = p - p_ref
    Real Dx, Dy;
};

__device__ __forceinline__ float rsqrt_r(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_r(double x) { return rsqrt(x); }
// Reciprocal: the FP32 path uses the fast hardware reciprocal (a few ulp),
// the FP64 path IEEE division.
__device__ __forceinline__ float rcp_r(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double rcp_r(double x) { return 1.0 / x; }
__device__ __forceinline__ float sinpi_r(float x) { return sinpif(x); }
__device__ __forceinline__ double sinpi_r(double x) { return sinpi(x); }
__device__ __forceinline__ float cospi_r(float x) { return cospif(x); }
__device__ __forceinline__ double cospi_r(double x) { return cospi(x); }
__device__ __forceinline__ bool finite_r(float x) { return isfinite(x); }
__device__ __forceinline__ bool finite_r(double x) { return isfinite(x); }

// Two FP32 lanes per instruction, each lane rounded as its scalar operation
// would be (round to nearest).  a - b is fma(-1, b, a), exact like FADD.
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(make_float2(-1.0f, -1.0f), b, a); }

// Prescribed velocity of the A-C-only model at (x, y), time t: uniform
// (Eq. 40), rotation about the box centre (Eq. 41), shear reversed at
// t = L0/U0 (Eq. 42), smoothed deformation with period L0/U0 (Eq. 43).
template <typename Real>
__device__ __forceinline__ void prescribed_velocity(const Phys<Real> &ph, Real x, Real y, double t, Real &ux,
                                                    Real &uy) {
    const Real pi = Real(3.14159265358979323846);
    switch (ph.vel_kind) {
    case 1:
        ux = -ph.vel_u * pi * ph.vel_il * (y - Real(0.5) / ph.vel_il);
        uy = ph.vel_u * pi * ph.vel_il * (x - Real(0.5) / ph.vel_il);
        break;
    case 2: {
        const Real a = (t < ph.vel_tr ? Real(1) : Real(-1)) * ph.vel_u * pi;
        ux = a * sinpi_r(x * ph.vel_il) * cospi_r(y * ph.vel_il);
        uy = -a * cospi_r(x * ph.vel_il) * sinpi_r(y * ph.vel_il);
        break;
    }
    case 3: {
        const Real c = -ph.vel_u * cospi_r(Real(t) * ph.vel_ul);
        ux = c * sinpi_r(Real(4) * x * ph.vel_il) * sinpi_r(Real(4) * y * ph.vel_il);
        uy = c * cospi_r(Real(4) * x * ph.vel_il) * cospi_r(Real(4) * y * ph.vel_il);
        break;
    }
    default:
        ux = ph.u0x;
        uy = ph.u0y;
    }
}

// theta, n (Eq. 6) and, for the coupled model, rho, mu_phi, mu, tau_g and F
// (Eqs. 3-4, 9-10, 34-36) from phi, grad phi and lap phi; in FP64 also
// 1 / (2 tau_g + step), the factor of the relaxation (Eqs. 28-29: step = h at
// a face, dt at a cell).
template <typename Real, bool COUPLED>
__device__ __forceinline__ void closures(const Phys<Real> &ph, Pt<Real> &s, Real step = Real(0)) {
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
        if constexpr (sizeof(Real) == 8) {
            // One FP64 division instead of three: with mu = num / den (linear rule
            // lin / 1, reciprocal rule 1 / lin) and e = 6 num + step rho den
            // (= (2 tau_g + step) rho den), R = 1 / (rho den e) gives 1 / rho =
            // den e R, tau_g = 3 mu / rho = 3 num e R and 1 / (2 tau_g + step) =
            // (rho den)^2 R.
            const Real num = ph.visc_linear ? lin : Real(1), den = ph.visc_linear ? Real(1) : lin;
            const Real rd = s.rho * den, e = Real(6) * num + step * rd;
            const Real R = Real(1) / (rd * e);
            const Real er = e * R;
            s.irho = den * er;
            s.taug = Real(3) * num * er;
            s.inv = rd * rd * R;
        } else {
            const Real mu = ph.visc_linear ? lin : rcp_r(lin);
            s.irho = rcp_r(s.rho);
            s.taug = Real(3) * mu * s.irho;
            s.inv = Real(0);   // FP32 takes its cheap reciprocal where the factor is used
        }
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
    s.ux = (mx + half * s.Fx) * s.irho;
    s.uy = (my + half * s.Fy) * s.irho;
    // RT/(1 - w0) = 3/5; rho (Gamma_0(u) - Gamma_0(0)) = -(2/3) rho |u|^2
    s.pd = Real(0.6) * (sn + half * (s.ux * s.drx + s.uy * s.dry)
                        - Real(2.0 / 3.0) * s.rho * (s.ux * s.ux + s.uy * s.uy));
}

// The f model's equilibrium (Eq. 15, as a deviation from w_k phi_ref) and
// source (Eq. 16) are linear in xi_k, so any combination c1 f_eq + c2 S^f is
//     w_k (P + xi_k . V),  P = c1 (phi - phi_ref),
//     V = 3 c1 phi u + c2 theta n + 3 c2 d_t(phi u)      (1 / RT = 3).
template <typename Real>
struct FLin {
    Real P, Vx, Vy;
};
template <typename Real>
__device__ __forceinline__ FLin<Real> f_lin(const Phys<Real> &ph, const Pt<Real> &s, Real c1, Real c2) {
    FLin<Real> r;
    r.P = c1 * (s.phi - ph.phi_ref);
    const Real a = Real(3) * c1 * s.phi, b = c2 * s.theta, c = Real(3) * c2;
    r.Vx = a * s.ux + b * s.nx + c * s.Dx;
    r.Vy = a * s.uy + b * s.ny + c * s.Dy;
    return r;
}
template <typename Real>
__device__ __forceinline__ Real f_lin_k(int k, const FLin<Real> &L) {
    const Real w = wq<Real>(k);
    if (k == 0) return w * L.P;
    return w * (L.P + edot(k, L.Vx, L.Vy));
}

// Per-point terms of the g equilibrium (Eqs. 17-18) and source (Eq. 19)
// shared by all directions.
template <typename Real>
struct GCoef {
    Real usq15, udr, udf3, pd3, f3x, f3y;
};
template <typename Real>
__device__ __forceinline__ GCoef<Real> g_coef(const Pt<Real> &s) {
    GCoef<Real> c;
    c.usq15 = Real(1.5) * (s.ux * s.ux + s.uy * s.uy);
    c.udr = s.ux * s.drx + s.uy * s.dry;
    c.f3x = Real(3) * s.Fx;
    c.f3y = Real(3) * s.Fy;
    c.udf3 = s.ux * c.f3x + s.uy * c.f3y;
    c.pd3 = Real(3) * s.pd;
    return c;
}
// Deviation of g_eq from 3 p_ref (w_k - delta_k0), and S^g, in direction k:
//   Gamma_k - w_k = w_k (3 e + 4.5 e^2 - 1.5 |u|^2),  e = xi_k . u
//   S^g_k = (Gamma_k - w_k)(xi_k - u).grad rho + 3 Gamma_k (xi_k - u).F
template <typename Real>
__device__ __forceinline__ void g_eq_src(int k, const Pt<Real> &s, const GCoef<Real> &c, Real &eq, Real &src) {
    const Real w = wq<Real>(k);
    if (k == 0) {
        const Real gam = w * (-c.usq15);
        eq = c.pd3 * (w - Real(1)) + s.rho * gam;
        src = -(gam * c.udr + (w + gam) * c.udf3);
        return;
    }
    const Real eu = edot(k, s.ux, s.uy);
    const Real gam = w * (eu * (Real(3) + Real(4.5) * eu) - c.usq15);
    eq = c.pd3 * w + s.rho * gam;
    src = gam * (edot(k, s.drx, s.dry) - c.udr) + (w + gam) * (edot(k, c.f3x, c.f3y) - c.udf3);
}

// A combination cb g_eq_k + cc S^g_k (deviation form) of every direction,
// with the per-point products hoisted:
//     cb g_eq_k + cc S^g_k = w_k (P + B_k) + (Gamma_k - w_k)(R + A_k + B_k) - delta_k0 P
//     P = 3 cb p',  R = cb rho,  A_k = cc (xi_k - u).grad rho,  B_k = 3 cc (xi_k - u).F
template <typename Real>
struct GLin {
    Real P, R, ax, ay, a0, bx, by, b0, usq15, ux, uy;
};
template <typename Real>
__device__ __forceinline__ GLin<Real> g_lin(const Pt<Real> &s, Real cb, Real cc) {
    GLin<Real> g;
    g.P = Real(3) * cb * s.pd;
    g.R = cb * s.rho;
    g.ax = cc * s.drx;
    g.ay = cc * s.dry;
    g.a0 = s.ux * g.ax + s.uy * g.ay;
    const Real c3 = Real(3) * cc;
    g.bx = c3 * s.Fx;
    g.by = c3 * s.Fy;
    g.b0 = s.ux * g.bx + s.uy * g.by;
    g.usq15 = Real(1.5) * (s.ux * s.ux + s.uy * s.uy);
    g.ux = s.ux;
    g.uy = s.uy;
    return g;
}
template <typename Real>
__device__ __forceinline__ Real g_lin_k(int k, const GLin<Real> &g) {
    const Real w = wq<Real>(k);
    if (k == 0) {
        const Real gam = -w * g.usq15;
        return w * (g.P - g.b0) - g.P + gam * (g.R - g.a0 - g.b0);
    }
    const Real eu = edot(k, g.ux, g.uy);
    const Real gam = w * (eu * (Real(3) + Real(4.5) * eu) - g.usq15);
    const Real B = edot(k, g.bx, g.by) - g.b0;
    const Real A = edot(k, g.ax, g.ay) - g.a0;
    return w * (g.P + B) + gam * ((g.R + A) + B);
}

// Packed FP32 forms for a direction k in 1..4 and its opposite opp(k) = k + 4
// (lane 0: k, lane 1: opp(k)); xi_opp = -xi_k, so every xi-odd term changes
// sign between the lanes and each lane repeats its scalar operations.
template <int K>
__device__ __forceinline__ float2 f_lin_pair(const FLin<float> &L) {
    const float e = edot(K, L.Vx, L.Vy);
    return mul2(f2(wq<float>(K)), add2(f2(L.P), f2(e, -e)));
}
template <int K>
__device__ __forceinline__ float2 g_lin_pair(const GLin<float> &g) {
    const float w = wq<float>(K);
    const float eu = edot(K, g.ux, g.uy), eb = edot(K, g.bx, g.by), ea = edot(K, g.ax, g.ay);
    const float2 eu2 = f2(eu, -eu);
    const float2 gam = mul2(f2(w), fma2(eu2, fma2(f2(4.5f), eu2, f2(3.0f)), f2(-g.usq15)));
    const float2 B = sub2(f2(eb, -eb), f2(g.b0));
    const float2 A = sub2(f2(ea, -ea), f2(g.a0));
    return fma2(gam, add2(add2(f2(g.R), A), B), mul2(f2(w), add2(f2(g.P), B)));
}

__device__ __forceinline__ int wrap(int x, int n) {
    x %= n;
    return x < 0 ? x + n : x;
}
// Periodic index for x in [-n, 2n) (one correction either way).
__device__ __forceinline__ int wrap1(int x, int n) {
    x += (x < 0) ? n : 0;
    return x - ((x >= n) ? n : 0);
}
// Row index for phi stencils: periodic, or mirrored at the walls (rows far
// outside are clamped; no valid cell's stencil reaches them).
template <bool WALLY>
__device__ __forceinline__ int map_row(int y, int ny, bool small = true) {
    if (!WALLY) return small ? wrap(y, ny) : wrap1(y, ny);
    if (y < 0) y = -1 - y;
    if (y >= ny) y = 2 * ny - 1 - y;
    return y < 0 ? 0 : (y >= ny ? ny - 1 : y);
}

// ---------------------------------------------------------------------------
// Shared-memory records.
//
// psi-bar-plus of one cell is a record of slots grouped by lattice direction,
// so that a face reads only the groups it needs, 16 bytes at a time:
//   coupled:  [f2 f4 f6 f8] [g2 g4 g6 g8] [f1 f5 g1 g5] [f3 f7 g3 g7] [f0 g0 - -]
//   A-C only: [f2 f4 f6 f8] [f1 f5 f3 f7] [f0 - - -]
// The diagonal groups need tangential neighbours at every face, the axis
// groups only at the faces they run along.  Record strides are chosen so that
// eight consecutive cells fall in distinct banks for 16-byte accesses.
template <bool COUPLED> struct Rec;
template <> struct Rec<true> {
    static constexpr int NG = 5;
    __host__ __device__ static constexpr int model(int s) {
        return s < 4 ? 0 : s < 8 ? 1 : s < 16 ? ((s & 2) ? 1 : 0) : (s == 16 ? 0 : 1);
    }
    __host__ __device__ static constexpr int dir(int s) {
        return s < 8 ? 2 + 2 * (s & 3) : s < 12 ? ((s & 1) ? 5 : 1) : s < 16 ? ((s & 1) ? 7 : 3) : 0;
    }
    __host__ __device__ static constexpr bool used(int s) { return s < 18; }
    __host__ __device__ static constexpr int slot(int m, int k) {
        return k == 0 ? 16 + m : (k & 1) == 0 ? 4 * m + (k - 2) / 2 : (k == 1 || k == 5) ? 8 + 2 * m + (k == 5) : 12 + 2 * m + (k == 7);
    }
};
template <> struct Rec<false> {
    static constexpr int NG = 3;
    __host__ __device__ static constexpr int model(int) { return 0; }
    __host__ __device__ static constexpr int dir(int s) {
        return s < 4 ? 2 + 2 * s : s == 4 ? 1 : s == 5 ? 5 : s == 6 ? 3 : s == 7 ? 7 : 0;
    }
    __host__ __device__ static constexpr bool used(int s) { return s < 9; }
    __host__ __device__ static constexpr int slot(int, int k) {
        return k == 0 ? 8 : (k & 1) == 0 ? (k - 2) / 2 : k == 1 ? 4 : k == 5 ? 5 : k == 3 ? 6 : 7;
    }
};

// Does group G hold a direction whose tangential slope is needed at an
// x-face (xi_y != 0) or a y-face (xi_x != 0)?
template <bool COUPLED, bool XFACE>
__host__ __device__ constexpr bool group_tangential(int G) {
    bool any = false;
    for (int j = 0; j < 4; j++) {
        const int s = 4 * G + j;
        if (Rec<COUPLED>::used(s)) {
            const int k = Rec<COUPLED>::dir(s);
            any = any || (XFACE ? cy(k) != 0 : cx(k) != 0);
        }
    }
    return any;
}

// 16-byte aligned groups of four values.
__device__ __forceinline__ void ld4(const float *p, float o[4]) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void ld4(const double *p, double o[4]) {
    const double2 a = *reinterpret_cast<const double2 *>(p), b = *reinterpret_cast<const double2 *>(p + 2);
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
__device__ __forceinline__ void st4(float *p, float a, float b, float c, float d) {
    *reinterpret_cast<float4 *>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ void st4(double *p, double a, double b, double c, double d) {
    *reinterpret_cast<double2 *>(p) = make_double2(a, b);
    *reinterpret_cast<double2 *>(p + 2) = make_double2(c, d);
}
// Pairs (8-byte aligned for float, 16-byte for double).
__device__ __forceinline__ void ld2(const float *p, float o[2]) {
    const float2 v = *reinterpret_cast<const float2 *>(p);
    o[0] = v.x; o[1] = v.y;
}
__device__ __forceinline__ void ld2(const double *p, double o[2]) {
    const double2 v = *reinterpret_cast<const double2 *>(p);
    o[0] = v.x; o[1] = v.y;
}
__device__ __forceinline__ void st2(float *p, float a, float b) { *reinterpret_cast<float2 *>(p) = make_float2(a, b); }
__device__ __forceinline__ void st2(double *p, double a, double b) { *reinterpret_cast<double2 *>(p) = make_double2(a, b); }

// Warps per CTA beyond one thread per tile cell.  They take halo-ring cells
// in phase 2 and their share of faces in phase 3, which shortens the phase
// tails (FP32 32 x 8: the 84 ring cells run beside the 256 tile cells, the
// 552 faces take 2 rounds of 320 threads instead of 3 of 256) at the cost of
// idling in the flux update.  Measured on GB300 (2048^2 spinodal, FP32):
// 0.353 / 0.343 / 0.333 / 0.350 / 0.345 ms per step for 0 / 1 / 2 / 3 / 4
// extra warps (3 CTAs per SM, registers capped to fit); FP64 16 x 8: 10.40 /
// 10.38 / 10.22 ms for 0 / 1 / 2.
#ifndef DUGKS_EXTRA_WARPS_F32
#define DUGKS_EXTRA_WARPS_F32 2
#endif
#ifndef DUGKS_EXTRA_WARPS_F64
#define DUGKS_EXTRA_WARPS_F64 2
#endif

// UPW: the upwind reconstruction (R14) reads psi-bar-plus two cells from a
// face, so its records cover the tile + 2 cells (H = 2) instead of + 1.
template <typename Real, int TX, int TY, bool COUPLED, bool UPW = false>
struct TileShape {
    static constexpr bool F64 = sizeof(Real) == 8;
    static constexpr int H = UPW ? 2 : 1;                                         // record halo
    static constexpr int NC = TX * TY;                                            // tile cells
    static constexpr int NT = NC + 32 * (F64 ? DUGKS_EXTRA_WARPS_F64 : DUGKS_EXTRA_WARPS_F32);  // threads
    static constexpr int HX2 = TX + 2 * H + 2, HY2 = TY + 2 * H + 2;  // phi' region (halo H + 1)
    static constexpr int HX1 = TX + 2 * H, HY1 = TY + 2 * H;          // psi-bar-plus records (halo H)
    static constexpr int N2 = HX2 * HY2, N1 = HX1 * HY1;
    static constexpr int NQ = COUPLED ? 18 : 9;
    // Input box: columns x0-4 .. x0+TX+3 (the left edge rounded down to a
    // 16-byte boundary for TMA; covers the phi' region for H <= 2), rows
    // y0-H-1 .. y0+TY+H, the NQ distribution planes followed by the 2
    // history planes.
    static constexpr int BX = TX + 8, BY = TY + 2 * H + 2, BXY = BX * BY;
    static constexpr int NFX = (TX + 1) * TY, NFY = TX * (TY + 1);
#ifndef DUGKS_FACE_PAD
#define DUGKS_FACE_PAD 1
#endif
    static constexpr int NFXP = DUGKS_FACE_PAD ? (NFX + 31) / 32 * 32 : NFX;   // x-face items, padded
    static constexpr int NFD = COUPLED ? 12 : 6;                               // flux values per face
    static constexpr int RS = Rec<COUPLED>::NG * 4 + (F64 ? 2 : 0);            // record stride
    static constexpr int AS = F64 ? 6 : 4;                                     // aux stride (FP32: d_t(phi u)_y apart)
    static constexpr int FS = COUPLED ? (F64 ? 14 : 12) : 6;                   // flux record stride
    static constexpr int AL = 128 / int(sizeof(Real));                         // 128-byte alignment
    static constexpr size_t up(size_t v) { return (v + AL - 1) / AL * AL; }
    static constexpr size_t off_box = 0;
    static constexpr size_t off_hbox = up(off_box + size_t(NQ) * BXY);   // history planes (TMA-aligned)
    static constexpr size_t off_phi = up(off_hbox + size_t(2) * BXY);
    static constexpr size_t off_rec = up(off_phi + N2);
    static constexpr size_t off_aux = up(off_rec + size_t(RS) * N1);
    static constexpr size_t off_dy = up(off_aux + size_t(AS) * N1);
    static constexpr size_t off_bar = up(off_dy + (F64 ? 0 : size_t(N1)));  // mbarrier, then a flag
    static constexpr size_t smem_elems = off_bar + 16 / sizeof(Real);
    static constexpr size_t smem_bytes = smem_elems * sizeof(Real) + 128;    // + room to align the base
    // The face fluxes reuse the input box once phase 2 has consumed it.
    static constexpr size_t off_fx = off_box;
    static constexpr size_t off_fy = off_fx + (size_t(FS) * NFX + 3) / 4 * 4;
    static_assert(off_fy + size_t(FS) * NFY <= off_phi, "face fluxes must fit in the input box");
    static_assert(off_hbox % AL == 0, "TMA destinations must be 128-byte aligned");
    static_assert((BX * sizeof(Real)) % 16 == 0, "TMA box rows must be multiples of 16 bytes");
    // CTAs per SM that the shared memory allows (228 KiB per SM, 1 KiB reserved per CTA);
    // passed to __launch_bounds__ so registers do not lower the occupancy further
    static constexpr int MINB = (smem_bytes + 1024) * 3 <= 233472 ? 3 : ((smem_bytes + 1024) * 2 <= 233472 ? 2 : 1);
};

// ---- TMA (cp.async.bulk.tensor) and mbarrier helpers ----
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
#ifdef __CUDA_ARCH__
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
#else
    return 0;
#endif
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
#ifdef __CUDA_ARCH__
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
#endif
}
// Invalidates an initialised barrier whose phases have all completed, so
// that its memory can be initialised again (a persistent CTA re-arms it for
// every tile).
__device__ __forceinline__ void mbar_inval(uint64_t *bar) {
#ifdef __CUDA_ARCH__
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
#endif
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
#ifdef __CUDA_ARCH__
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
#endif
}
// 3-D tiled TMA load of the box at (x, y, z) into shared memory.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar) {
#ifdef __CUDA_ARCH__
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
#endif
}
// Waits for phase `parity` of the barrier, at most max_polls polls.  Returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long max_polls) {
#ifdef __CUDA_ARCH__
    for (long i = 0; i < max_polls; i++) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
#else
    return true;
#endif
}

// Central reconstruction (Eq. 27) at the face between cells A and B (record
// indices) of every direction needed there.  The tangential slope uses the
// records at A +- tstride, B +- tstride: tmode 0 central, +1 one-sided
// towards +t, -1 one-sided towards -t.  The rest direction of g is not needed
// by any face quantity and is skipped.
// FP32 form of recon_face: the two lanes of each half of a record group in
// one packed instruction; per lane the same operations (T = (n + n') - (s + s'),
// v = c_a a + c_b b - h c_t T / 4 or / 2).
template <bool COUPLED, bool XFACE, int RS>
__device__ __forceinline__ void recon_face_f2(const float *__restrict__ rec, int A, int B, int tstride, int tmode,
                                              float h, float fb[9], float gb[9]) {
    const float cp = 0.5f + h, cm = 0.5f - h;
    const float ht = tmode == 0 ? 0.25f * h : 0.5f * h;
#pragma unroll
    for (int G = 0; G < Rec<COUPLED>::NG; G++) {
        const bool tang = group_tangential<COUPLED, XFACE>(G);
        const float4 a = *reinterpret_cast<const float4 *>(rec + A * RS + 4 * G);
        const float4 b = *reinterpret_cast<const float4 *>(rec + B * RS + 4 * G);
        float4 an = a, bn = b, as = a, bs = b;
        if (tang) {
            if (tmode >= 0) {
                an = *reinterpret_cast<const float4 *>(rec + (A + tstride) * RS + 4 * G);
                bn = *reinterpret_cast<const float4 *>(rec + (B + tstride) * RS + 4 * G);
            }
            if (tmode <= 0) {
                as = *reinterpret_cast<const float4 *>(rec + (A - tstride) * RS + 4 * G);
                bs = *reinterpret_cast<const float4 *>(rec + (B - tstride) * RS + 4 * G);
            }
        }
#pragma unroll
        for (int P = 0; P < 2; P++) {
            const int s0 = 4 * G + 2 * P, s1 = s0 + 1;
            const bool n0 = Rec<COUPLED>::used(s0) && !(Rec<COUPLED>::model(s0) == 1 && Rec<COUPLED>::dir(s0) == 0);
            const bool n1 = Rec<COUPLED>::used(s1) && !(Rec<COUPLED>::model(s1) == 1 && Rec<COUPLED>::dir(s1) == 0);
            if (!n0 && !n1) continue;
            const int k0 = Rec<COUPLED>::dir(s0), k1 = Rec<COUPLED>::dir(s1);
            const int cn0 = XFACE ? cx(k0) : cy(k0), cn1 = XFACE ? cx(k1) : cy(k1);
            const int ct0 = XFACE ? cy(k0) : cx(k0), ct1 = XFACE ? cy(k1) : cx(k1);
            const float2 A2 = P == 0 ? f2(a.x, a.y) : f2(a.z, a.w);
            const float2 B2 = P == 0 ? f2(b.x, b.y) : f2(b.z, b.w);
            const float2 ca = f2(cn0 == 0 ? 0.5f : (cn0 > 0 ? cp : cm), cn1 == 0 ? 0.5f : (cn1 > 0 ? cp : cm));
            const float2 cb = f2(cn0 == 0 ? 0.5f : (cn0 > 0 ? cm : cp), cn1 == 0 ? 0.5f : (cn1 > 0 ? cm : cp));
            float2 V = fma2(cb, B2, mul2(ca, A2));
            if (tang && (ct0 != 0 || ct1 != 0)) {
                const float2 Pn = tmode >= 0 ? add2(P == 0 ? f2(an.x, an.y) : f2(an.z, an.w),
                                                    P == 0 ? f2(bn.x, bn.y) : f2(bn.z, bn.w))
                                             : add2(A2, B2);
                const float2 Ps = tmode <= 0 ? add2(P == 0 ? f2(as.x, as.y) : f2(as.z, as.w),
                                                    P == 0 ? f2(bs.x, bs.y) : f2(bs.z, bs.w))
                                             : add2(A2, B2);
                const float2 hv = f2(ct0 > 0 ? -ht : (ct0 < 0 ? ht : 0.0f), ct1 > 0 ? -ht : (ct1 < 0 ? ht : 0.0f));
                V = fma2(hv, sub2(Pn, Ps), V);
            }
            if (n0) { if (Rec<COUPLED>::model(s0) == 0) fb[k0] = V.x; else gb[k0] = V.x; }
            if (n1) { if (Rec<COUPLED>::model(s1) == 0) fb[k1] = V.y; else gb[k1] = V.y; }
        }
    }
}

template <typename Real, bool COUPLED, bool XFACE, int RS>
__device__ __forceinline__ void recon_face(const Real *__restrict__ rec, int A, int B, int tstride, int tmode, Real h,
                                           Real fb[9], Real gb[9]) {
    if constexpr (DUGKS_PACKED_F32 && std::is_same<Real, float>::value) {
        recon_face_f2<COUPLED, XFACE, RS>(rec, A, B, tstride, tmode, h, fb, gb);
    } else {
        // value - h xi.slope = (1/2 + h c_n) a + (1/2 - h c_n) b - h c_t s_t
        const Real cp = Real(0.5) + h, cm = Real(0.5) - h;
        const Real ht = tmode == 0 ? Real(0.25) * h : Real(0.5) * h;
#pragma unroll
        for (int G = 0; G < Rec<COUPLED>::NG; G++) {
            Real a[4], b[4], an[4], as[4], bn[4], bs[4];
            ld4(rec + A * RS + 4 * G, a);
            ld4(rec + B * RS + 4 * G, b);
            const bool tang = group_tangential<COUPLED, XFACE>(G);
            if (tang) {
                if (tmode >= 0) {
                    ld4(rec + (A + tstride) * RS + 4 * G, an);
                    ld4(rec + (B + tstride) * RS + 4 * G, bn);
                }
                if (tmode <= 0) {
                    ld4(rec + (A - tstride) * RS + 4 * G, as);
                    ld4(rec + (B - tstride) * RS + 4 * G, bs);
                }
            }
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int s = 4 * G + j;
                if (!Rec<COUPLED>::used(s)) continue;
                const int k = Rec<COUPLED>::dir(s), m = Rec<COUPLED>::model(s);
                if (m == 1 && k == 0) continue;
                const int cn = XFACE ? cx(k) : cy(k), ct = XFACE ? cy(k) : cx(k);
                Real v;
                if (cn == 0) v = Real(0.5) * (a[j] + b[j]);
                else if (cn > 0) v = cp * a[j] + cm * b[j];
                else v = cm * a[j] + cp * b[j];
                if (ct != 0) {
                    Real T;  // 4 s_t (central) or 2 s_t (one-sided)
                    if (tmode == 0) T = (an[j] + bn[j]) - (as[j] + bs[j]);
                    else if (tmode > 0) T = (an[j] + bn[j]) - (a[j] + b[j]);
                    else T = (a[j] + b[j]) - (as[j] + bs[j]);
                    v = ct > 0 ? v - ht * T : v + ht * T;
                }
                if (m == 0) fb[k] = v; else gb[k] = v;
            }
        }
    }
}

// van Leer's limiter of two one-sided differences: their harmonic mean, or 0
// at an extremum (R14).
template <typename Real>
__device__ __forceinline__ Real van_leer(Real s1, Real s2) {
    return s1 * s2 > Real(0) ? Real(2) * s1 * s2 * rcp_r(s1 + s2) : Real(0);
}

// van Leer's limiter on two lanes: the products, sums and scaling packed, the
// reciprocal and the extremum test per lane (as van_leer does for one).
__device__ __forceinline__ float2 van_leer2(float2 s1, float2 s2) {
    const float2 p = mul2(s1, s2), q = add2(s1, s2);
    const float2 v = mul2(mul2(f2(2.0f), p), f2(rcp_r(q.x), rcp_r(q.y)));
    return f2(p.x > 0.0f ? v.x : 0.0f, p.y > 0.0f ? v.y : 0.0f);
}

// FP32 form of recon_face_upwind: the two lanes of each half of a record
// group in one packed instruction.  A lane crossing the face reads the
// profile of the cell it leaves (centre, its normal neighbours, its
// tangential neighbours, chosen per lane at compile time); in the groups of
// directions along the face both lanes take the mean of both profiles.
template <bool COUPLED, bool XFACE, int RS>
__device__ __forceinline__ void recon_face_upwind_f2(const float *__restrict__ rec, int A, int B, int nstride,
                                                     int tstride, float h, float fb[9], float gb[9], int tmode = 0,
                                                     bool a_wall = false, bool b_wall = false) {
    auto ld = [&](int c, int G) { return *reinterpret_cast<const float4 *>(rec + c * RS + 4 * G); };
    auto half = [](const float4 &v, int P) { return P == 0 ? f2(v.x, v.y) : f2(v.z, v.w); };
#pragma unroll
    for (int G = 0; G < Rec<COUPLED>::NG; G++) {
        const bool tang = group_tangential<COUPLED, XFACE>(G);
        const float4 a = ld(A, G), b = ld(B, G), am = ld(A - nstride, G), bp = ld(B + nstride, G);
        float4 an = a, as = a, bn = b, bs = b;
        if (tang) {
            an = ld(A + tstride, G);
            as = ld(A - tstride, G);
            bn = ld(B + tstride, G);
            bs = ld(B - tstride, G);
        }
#pragma unroll
        for (int P = 0; P < 2; P++) {
            const int s0 = 4 * G + 2 * P, s1 = s0 + 1;
            const bool n0 = Rec<COUPLED>::used(s0) && !(Rec<COUPLED>::model(s0) == 1 && Rec<COUPLED>::dir(s0) == 0);
            const bool n1 = Rec<COUPLED>::used(s1) && !(Rec<COUPLED>::model(s1) == 1 && Rec<COUPLED>::dir(s1) == 0);
            if (!n0 && !n1) continue;
            const int k0 = Rec<COUPLED>::dir(s0), k1 = Rec<COUPLED>::dir(s1);
            const int cn0 = XFACE ? cx(k0) : cy(k0), cn1 = XFACE ? cx(k1) : cy(k1);
            const int ct0 = XFACE ? cy(k0) : cx(k0), ct1 = XFACE ? cy(k1) : cx(k1);
            const float2 A2 = half(a, P), B2 = half(b, P);
            // profile of the cell on side `up` (+1: A, -1: B) of each lane at x_f - xi h
            auto profile = [&](int up0, int up1, float2 coef) {
                const float2 c = f2(up0 > 0 ? A2.x : B2.x, up1 > 0 ? A2.y : B2.y);
                const float2 m = f2(up0 > 0 ? half(am, P).x : A2.x, up1 > 0 ? half(am, P).y : A2.y);
                const float2 q = f2(up0 > 0 ? B2.x : half(bp, P).x, up1 > 0 ? B2.y : half(bp, P).y);
                float2 sn = van_leer2(sub2(c, m), sub2(q, c));
                // R17: a cell next to a wall takes its one-sided difference into the fluid
                if (a_wall || b_wall) {
                    const float2 one = sub2(B2, A2);
                    sn = f2((up0 > 0 ? a_wall : b_wall) ? one.x : sn.x, (up1 > 0 ? a_wall : b_wall) ? one.y : sn.y);
                }
                float2 v = fma2(sn, coef, c);
                if (tang && (ct0 != 0 || ct1 != 0)) {
                    const float2 tn = f2(up0 > 0 ? half(an, P).x : half(bn, P).x, up1 > 0 ? half(an, P).y : half(bn, P).y);
                    const float2 ts = f2(up0 > 0 ? half(as, P).x : half(bs, P).x, up1 > 0 ? half(as, P).y : half(bs, P).y);
                    const float2 ht = f2(ct0 > 0 ? -h : (ct0 < 0 ? h : 0.0f), ct1 > 0 ? -h : (ct1 < 0 ? h : 0.0f));
                    const float2 st = tmode == 0 ? van_leer2(sub2(c, ts), sub2(tn, c))
                                                 : (tmode > 0 ? sub2(tn, c) : sub2(c, ts));
                    v = fma2(ht, st, v);
                }
                return v;
            };
            float2 V;
            if (cn0 != 0 && cn1 != 0) {
                V = profile(cn0, cn1, f2(cn0 > 0 ? 0.5f - h : h - 0.5f, cn1 > 0 ? 0.5f - h : h - 0.5f));
            } else {   // a lane along the face: both profiles, their mean there
                const float2 vA = profile(1, 1, f2(cn0 > 0 ? 0.5f - h : 0.5f, cn1 > 0 ? 0.5f - h : 0.5f));
                const float2 vB = profile(-1, -1, f2(cn0 < 0 ? h - 0.5f : -0.5f, cn1 < 0 ? h - 0.5f : -0.5f));
                const float2 M = mul2(f2(0.5f), add2(vA, vB));
                V = f2(cn0 > 0 ? vA.x : (cn0 < 0 ? vB.x : M.x), cn1 > 0 ? vA.y : (cn1 < 0 ? vB.y : M.y));
            }
            if (n0) { if (Rec<COUPLED>::model(s0) == 0) fb[k0] = V.x; else gb[k0] = V.x; }
            if (n1) { if (Rec<COUPLED>::model(s1) == 0) fb[k1] = V.y; else gb[k1] = V.y; }
        }
    }
}

// Upwind reconstruction (R14) at the face between cells A and B (record
// indices; B = A + nstride along the face normal): each cell carries a linear
// profile with van Leer slopes along the normal (cells A - nstride .. B +
// nstride) and the tangent (A +- tstride, B +- tstride); a direction crossing
// the face takes the upwind cell's profile at x_f - xi h, one along the face
// the mean of both.  The rest direction of g is not needed and is skipped.
// With walls (R17): tmode +1 / -1 takes the one-sided tangential difference
// towards +t / -t (a cell row next to a wall), and a_wall / b_wall give cell A
// / B the one-sided normal difference b - a into the fluid (A in the first
// row above a wall, B in the last row below one).
template <typename Real, bool COUPLED, bool XFACE, int RS>
__device__ __forceinline__ void recon_face_upwind(const Real *__restrict__ rec, int A, int B, int nstride,
                                                  int tstride, Real h, Real fb[9], Real gb[9], int tmode = 0,
                                                  bool a_wall = false, bool b_wall = false) {
    if constexpr (DUGKS_PACKED_F32 && std::is_same<Real, float>::value) {
        recon_face_upwind_f2<COUPLED, XFACE, RS>(rec, A, B, nstride, tstride, h, fb, gb, tmode, a_wall, b_wall);
    } else {
#pragma unroll
        for (int G = 0; G < Rec<COUPLED>::NG; G++) {
            Real a[4], b[4], am[4], bp[4], an[4], as[4], bn[4], bs[4];
            ld4(rec + A * RS + 4 * G, a);
            ld4(rec + B * RS + 4 * G, b);
            ld4(rec + (A - nstride) * RS + 4 * G, am);
            ld4(rec + (B + nstride) * RS + 4 * G, bp);
            if (group_tangential<COUPLED, XFACE>(G)) {
                ld4(rec + (A + tstride) * RS + 4 * G, an);
                ld4(rec + (A - tstride) * RS + 4 * G, as);
                ld4(rec + (B + tstride) * RS + 4 * G, bn);
                ld4(rec + (B - tstride) * RS + 4 * G, bs);
            }
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int s = 4 * G + j;
                if (!Rec<COUPLED>::used(s)) continue;
                const int k = Rec<COUPLED>::dir(s), m = Rec<COUPLED>::model(s);
                if (m == 1 && k == 0) continue;
                const int cn = XFACE ? cx(k) : cy(k), ct = XFACE ? cy(k) : cx(k);
                // A's profile at x_f - xi h: normal offset 1/2 - h cn, tangential -h ct; B's: -1/2 - h cn
                Real vA = Real(0), vB = Real(0);
                auto tslope = [&](Real c, Real sv, Real nv) {
                    return tmode == 0 ? van_leer(c - sv, nv - c) : (tmode > 0 ? nv - c : c - sv);
                };
                if (cn >= 0) {
                    const Real sA = a_wall ? b[j] - a[j] : van_leer(a[j] - am[j], b[j] - a[j]);
                    vA = a[j] + sA * (cn > 0 ? Real(0.5) - h : Real(0.5));
                    if (ct != 0) vA -= sgnmul(ct, h * tslope(a[j], as[j], an[j]));
                }
                if (cn <= 0) {
                    const Real sB = b_wall ? b[j] - a[j] : van_leer(b[j] - a[j], bp[j] - b[j]);
                    vB = b[j] + sB * (cn < 0 ? h - Real(0.5) : Real(-0.5));
                    if (ct != 0) vB -= sgnmul(ct, h * tslope(b[j], bs[j], bn[j]));
                }
                const Real v = cn > 0 ? vA : (cn < 0 ? vB : Real(0.5) * (vA + vB));
                if (m == 0) fb[k] = v; else gb[k] = v;
            }
        }
    }
}

// Wall face, bottom (TOP == false) or top: linear extrapolation from cell c0
// (next cell into the fluid at c0 + inward) for directions leaving the fluid
// or tangential, bounce-back for directions entering it.
// UPW (R17): the tangential slope is van Leer's limited one instead of the
// central difference.
template <typename Real, bool COUPLED, bool TOP, int RS, bool UPW = false>
__device__ __forceinline__ void recon_wall(const Real *__restrict__ rec, int c0, int inward, Real h, Real fb[9],
                                           Real gb[9]) {
    const Real dyw = TOP ? Real(0.5) : Real(-0.5);
#pragma unroll
    for (int m = 0; m < (COUPLED ? 2 : 1); m++) {
        Real *out = m == 0 ? fb : gb;
#pragma unroll
        for (int k = 0; k < 9; k++) {
            const bool keep = TOP ? (cy(k) >= 0) : (cy(k) <= 0);
            if (!keep) continue;
            const int sl = Rec<COUPLED>::slot(m, k);
            const Real b0 = rec[c0 * RS + sl];
            const Real sy = TOP ? (b0 - rec[(c0 + inward) * RS + sl]) : (rec[(c0 + inward) * RS + sl] - b0);
            Real v = b0 + (cy(k) == 0 ? dyw : (cy(k) > 0 ? dyw - h : dyw + h)) * sy;
            if (cx(k) != 0) {
                const Real e = rec[(c0 + 1) * RS + sl], w = rec[(c0 - 1) * RS + sl];
                const Real sx = UPW ? van_leer(b0 - w, e - b0) : Real(0.5) * (e - w);
                v -= h * sgnmul(cx(k), sx);
            }
            out[k] = v;
        }
#pragma unroll
        for (int k = 0; k < 9; k++) {
            const bool enters = TOP ? (cy(k) < 0) : (cy(k) > 0);
            if (enters) out[k] = out[opp(k)];
        }
    }
}

// First moments and non-rest sum of the g distributions (Eqs. 32-33).
template <typename Real>
__device__ __forceinline__ void moments9(const Real g[9], Real &mx, Real &my, Real &sn) {
    // directions 1..8: (1,0) (1,1) (0,1) (-1,1) (-1,0) (-1,-1) (0,-1) (1,-1)
    mx = ((g[1] + g[2]) + g[8]) - ((g[4] + g[5]) + g[6]);
    my = ((g[2] + g[3]) + g[4]) - ((g[6] + g[7]) + g[8]);
    sn = ((g[1] + g[2]) + (g[3] + g[4])) + ((g[5] + g[6]) + (g[7] + g[8]));
}

// Face state from f_bar, g_bar and the face values of the aux fields, then
// the original distributions (Eq. 28) of the directions crossing the face,
// in flux-slot order: out[slot] for f, out[6 + slot] for g.
template <typename Real, bool COUPLED, bool XFACE>
__device__ __forceinline__ void face_flux(const Phys<Real> &ph, const Real fb[9], const Real gb[9], Real dpx,
                                          Real dpy, Real lap, Real Dx, Real Dy, bool wall, Real out[12], Real xf = Real(0),
                                          Real yf = Real(0), double tf = 0.0, const Real *uf = nullptr) {
    Pt<Real> s;
    Real sphi = fb[0];
#pragma unroll
    for (int k = 1; k < 9; k++) sphi += fb[k];
    s.phi = ph.phi_ref + sphi;
    s.dpx = dpx;
    s.dpy = dpy;
    s.lap = lap;
    s.Dx = Dx;
    s.Dy = Dy;
    closures<Real, COUPLED>(ph, s, ph.h);
    if constexpr (COUPLED) {
        Real mx, my, sn;
        moments9(gb, mx, my, sn);
        if (wall) {
            s.ux = Real(0);
            s.uy = Real(0);
            s.pd = Real(0.6) * sn;
        } else {
            velocity_pressure(mx, my, sn, ph.half_h, s);
        }
    } else if (wall) {
        s.ux = Real(0);
        s.uy = Real(0);
    } else if (uf) {   // sampled field, evaluated by the caller
        s.ux = uf[0];
        s.uy = uf[1];
    } else {
        prescribed_velocity(ph, xf, yf, tf, s.ux, s.uy);
    }
    const FLin<Real> lf = f_lin(ph, s, ph.ff_b, ph.ff_c);
#pragma unroll
    for (int k = 1; k < 9; k++) {
        const int slot = XFACE ? xslot(k) : yslot(k);
        if (slot >= 0) out[slot] = ph.ff_a * fb[k] + f_lin_k(k, lf);
    }
    if (COUPLED) {
        const Real inv = sizeof(Real) == 8 ? s.inv : rcp_r(Real(2) * s.taug + ph.h);
        const Real a = Real(2) * s.taug * inv, bb = ph.h * inv, c = s.taug * ph.h * inv;
        const GLin<Real> gl = g_lin(s, bb, c);
#pragma unroll
        for (int k = 1; k < 9; k++) {
            const int slot = XFACE ? xslot(k) : yslot(k);
            if (slot >= 0) out[6 + slot] = a * gb[k] + g_lin_k(k, gl);
        }
    }
}

template <typename Real, bool COUPLED, int FS>
__device__ __forceinline__ void store_flux(Real *p, const Real v[12]) {
    if (COUPLED) {
        st4(p, v[0], v[1], v[2], v[3]);
        st4(p + 4, v[4], v[5], v[6], v[7]);
        st4(p + 8, v[8], v[9], v[10], v[11]);
    } else {
        st2(p, v[0], v[1]);
        st2(p + 2, v[2], v[3]);
        st2(p + 4, v[4], v[5]);
    }
}
template <typename Real, bool COUPLED, int FS>
__device__ __forceinline__ void load_flux(const Real *p, Real v[12]) {
    if (COUPLED) {
        ld4(p, v);
        ld4(p + 4, v + 4);
        ld4(p + 8, v + 8);
    } else {
        ld2(p, v);
        ld2(p + 2, v + 2);
        ld2(p + 4, v + 4);
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

// Macros, equilibria, sources and psi-bar-plus (Eq. 29) of one cell of the
// halo-1 region (record index c1, box index e), from the staged box.  For a
// tile cell (TILE) also psi~+ partials tp = 4/3 psi-bar-plus - 1/3 psi~
// (Eq. 30) and the new (phi u) history.
template <typename Real, int TX, int TY, bool COUPLED, bool WALLY, bool UPW, bool TILE>
__device__ __forceinline__ void cell_item(const StepArgs<Real> &a, const Phys<Real> &ph, const Real *__restrict__ box,
                                          const Real *__restrict__ sphi, Real *__restrict__ rec, Real *__restrict__ aux,
                                          Real *__restrict__ sdy, int hx, int hy, int x0, int y0, Real tp[18]) {
    using S = TileShape<Real, TX, TY, COUPLED, UPW>;
    using R = Rec<COUPLED>;
    constexpr int RS = S::RS, AS = S::AS, BXY = S::BXY;
    constexpr int H = S::H;
    const int c1 = hy * S::HX1 + hx;
    const int yraw = y0 + hy - H;
    if (!in_bounds(hx >= 0 && hx < S::HX1 && hy >= 0 && hy < S::HY1, a.status)) return;
    if (WALLY && (yraw < 0 || yraw >= a.ny)) {
        // outside the walls: never read by a face; keep the smem defined
#pragma unroll
        for (int G = 0; G < R::NG; G++) st4(rec + c1 * RS + 4 * G, Real(0), Real(0), Real(0), Real(0));
        st4(aux + c1 * AS, Real(0), Real(0), Real(0), Real(0));
        if (S::F64) aux[c1 * AS + 4] = Real(0); else sdy[c1] = Real(0);
        return;
    }
    const int e = (hy + 1) * S::BX + hx + 4 - H;
    if (!in_bounds(e >= 0 && e < BXY && hx + 4 - H >= 1 && hx + 5 - H < S::BX, a.status)) return;
    Pt<Real> s;
    const int c2 = (hy + 1) * S::HX2 + (hx + 1);
    phi_stencils(sphi, c2, S::HX2, s.dpx, s.dpy, s.lap);
    s.phi = ph.phi_ref + sphi[c2];
    closures<Real, COUPLED>(ph, s, ph.dt);
    Real dg[9];
    if (COUPLED) {
#pragma unroll
        for (int k = 0; k < 9; k++) dg[k] = box[(9 + k) * BXY + e];
        Real mx, my, sn;
        moments9(dg, mx, my, sn);
        velocity_pressure(mx, my, sn, ph.half_dt, s);
    } else if (ph.vel_kind == 0) {
        s.ux = ph.u0x;
        s.uy = ph.u0y;
    } else if (ph.vel_kind == 4) {
        const int gx = a.small ? wrap(x0 + hx - H, a.nx) : wrap1(x0 + hx - H, a.nx);
        const int gy = WALLY ? yraw : (a.small ? wrap(yraw, a.ny) : wrap1(yraw, a.ny));
        const long long gv = (long long)gy * a.pitch + gx;
        s.ux = a.vel[gv];
        s.uy = a.vel[a.plane + gv];
    } else {
        const int gx = a.small ? wrap(x0 + hx - H, a.nx) : wrap1(x0 + hx - H, a.nx);
        const int gy = WALLY ? yraw : (a.small ? wrap(yraw, a.ny) : wrap1(yraw, a.ny));
        prescribed_velocity(ph, Real(gx) + Real(0.5), Real(gy) + Real(0.5), a.t_n, s.ux, s.uy);
    }
    const Real phux = s.phi * s.ux, phuy = s.phi * s.uy;
    if (a.first_step) {
        s.Dx = Real(0);
        s.Dy = Real(0);
    } else {
        s.Dx = (phux - box[S::off_hbox + e]) * ph.inv_dt;
        s.Dy = (phuy - box[S::off_hbox + BXY + e]) * ph.inv_dt;
    }
    st4(aux + c1 * AS, s.dpx, s.dpy, s.lap, s.Dx);
    if (S::F64) aux[c1 * AS + 4] = s.Dy; else sdy[c1] = s.Dy;

    Real r[4 * R::NG];
    // psi-bar-plus of f (Eq. 29) and psi~+ = bp + (bp - d) / 3 (Eq. 30).  FP32:
    // bp is formed as a relaxation of d towards the equilibrium plus the
    // source, bp = d + (pf_b f_eq + pf_c S - pf_b d) (pf_a = 1 - pf_b), and the
    // rest direction takes phi' minus the other eight (the nine add up to phi'
    // in exact arithmetic), so that rounded coefficients cannot bias the phi
    // mass from step to step.  FP64 rounding is far below any such drift and
    // keeps the shorter form pf_a d + pf_b f_eq + pf_c S.
    const FLin<Real> lf = f_lin(ph, s, ph.pf_b, ph.pf_c);
    if constexpr (DUGKS_PACKED_F32 && !S::F64) {
        // opposite directions (k, k + 4) in the two lanes of one instruction
        float2 bsum2 = f2(0.0f);
        auto fpair = [&](auto kc) {
            constexpr int K = decltype(kc)::value, O = K + 4;
            const float2 d = f2(box[K * BXY + e], box[O * BXY + e]);
            const float2 bp = add2(d, fma2(f2(-ph.pf_b), d, f_lin_pair<K>(lf)));
            r[R::slot(0, K)] = bp.x;
            r[R::slot(0, O)] = bp.y;
            bsum2 = add2(bsum2, bp);
            if (TILE) {
                const float2 t = fma2(f2(1.0f / 3.0f), sub2(bp, d), bp);
                tp[K] = t.x;
                tp[O] = t.y;
            }
        };
        fpair(std::integral_constant<int, 1>{});
        fpair(std::integral_constant<int, 2>{});
        fpair(std::integral_constant<int, 3>{});
        fpair(std::integral_constant<int, 4>{});
        const Real d = box[e];
        const Real bp = sphi[c2] - (bsum2.x + bsum2.y);
        r[R::slot(0, 0)] = bp;
        if (TILE) tp[0] = bp + (bp - d) * Real(1.0 / 3.0);
    } else if (!S::F64) {
        Real bsum = Real(0);
#pragma unroll
        for (int k = 1; k < 9; k++) {
            const Real d = box[k * BXY + e];
            const Real bp = d + (f_lin_k(k, lf) - ph.pf_b * d);
            r[R::slot(0, k)] = bp;
            bsum += bp;
            if (TILE) tp[k] = bp + (bp - d) * Real(1.0 / 3.0);
        }
        const Real d = box[e];
        const Real bp = sphi[c2] - bsum;
        r[R::slot(0, 0)] = bp;
        if (TILE) tp[0] = bp + (bp - d) * Real(1.0 / 3.0);
    } else {
#pragma unroll
        for (int k = 0; k < 9; k++) {
            const Real d = box[k * BXY + e];
            const Real bp = ph.pf_a * d + f_lin_k(k, lf);
            r[R::slot(0, k)] = bp;
            if (TILE) tp[k] = bp + (bp - d) * Real(1.0 / 3.0);
        }
    }
    if (COUPLED) {
        const Real inv = S::F64 ? s.inv : rcp_r(Real(2) * s.taug + ph.dt);
        const Real ca = (Real(2) * s.taug - ph.h) * inv, cb = Real(3) * ph.h * inv, cc = Real(3) * s.taug * ph.h * inv;
        const GLin<Real> gl = g_lin(s, cb, cc);
        if constexpr (DUGKS_PACKED_F32 && !S::F64) {
            auto gpair = [&](auto kc) {
                constexpr int K = decltype(kc)::value, O = K + 4;
                const float2 d = f2(dg[K], dg[O]);
                const float2 bp = add2(d, fma2(f2(-cb), d, g_lin_pair<K>(gl)));
                r[R::slot(1, K)] = bp.x;
                r[R::slot(1, O)] = bp.y;
                if (TILE) {
                    const float2 t = fma2(f2(1.0f / 3.0f), sub2(bp, d), bp);
                    tp[9 + K] = t.x;
                    tp[9 + O] = t.y;
                }
            };
            gpair(std::integral_constant<int, 1>{});
            gpair(std::integral_constant<int, 2>{});
            gpair(std::integral_constant<int, 3>{});
            gpair(std::integral_constant<int, 4>{});
            const Real bp = dg[0] + (g_lin_k(0, gl) - cb * dg[0]);
            r[R::slot(1, 0)] = bp;
            if (TILE) tp[9] = bp + (bp - dg[0]) * Real(1.0 / 3.0);
        } else {
#pragma unroll
            for (int k = 0; k < 9; k++) {
                const Real bp = S::F64 ? ca * dg[k] + g_lin_k(k, gl) : dg[k] + (g_lin_k(k, gl) - cb * dg[k]);
                r[R::slot(1, k)] = bp;
                if (TILE) tp[9 + k] = bp + (bp - dg[k]) * Real(1.0 / 3.0);
            }
        }
    }
#pragma unroll
    for (int j = 4 * R::NG - 3; j < 4 * R::NG; j++)
        if (!R::used(j)) r[j] = Real(0);
#pragma unroll
    for (int G = 0; G < R::NG; G++) st4(rec + c1 * RS + 4 * G, r[4 * G], r[4 * G + 1], r[4 * G + 2], r[4 * G + 3]);

    if (TILE && x0 + hx - H < a.nx && yraw < a.ny &&
        in_bounds(x0 + hx - H >= 0 && yraw >= 0, a.status)) {
        const long long g = (long long)yraw * a.pitch + (x0 + hx - H);
        a.hdst[g] = phux;
        a.hdst[a.plane + g] = phuy;
        const bool bad = !finite_r(s.phi) || !finite_r(s.ux) || !finite_r(s.uy);
        const bool nonphys = COUPLED && !(s.rho > Real(0) && s.taug > Real(0));
        if (bad || nonphys) atomicOr(a.status, (bad ? STATUS_NONFINITE : 0u) | (nonphys ? STATUS_NONPHYSICAL : 0u));
    }
}

// Bound on mbarrier polls before a TMA wait gives up (well under a second).
// After one CTA has timed out the status word carries STATUS_TIMEOUT and
// later CTAs stage their box with plain loads instead.
constexpr long kPollLimit = 1l << 16;

// ---------------------------------------------------------------------------
// The fused step: one CTA per TX x TY tile, one thread per tile cell (plus
// two warps for halo cells and faces).
//   0. stage the input box (distributions and history, tile + halo) in smem:
//      one TMA load per array; a tile touching the domain edge then reloads
//      its out-of-domain cells with plain loads (periodic wrap / wall mirror)
//   1. phi' = sum_i d^f_i on the tile + 2-cell halo
//   2. cell macros, equilibria, sources and psi-bar-plus (Eq. 29) on the tile
//      + 1-cell halo (smem records); psi~+ partials of the tile cells stay in
//      registers; (phi u)^n of the tile to global
//   3. every face of the tile: reconstruction (Eq. 27), face macros, Eq. 28
//      (face records reuse the box)
//   4. the flux update (Eq. 24) of the tile to global
// ---------------------------------------------------------------------------
template <typename Real, int TX, int TY, bool COUPLED, bool WALLY, bool UPW>
__device__ __forceinline__ void tile_compute(const StepArgs<Real> &a, const Phys<Real> &ph, int x0, int y0,
                                             Real *__restrict__ box, Real *__restrict__ sphi, Real *__restrict__ rec,
                                             Real *__restrict__ aux, Real *__restrict__ sdy);

// A load of the stored state that bypasses L1 and the read-only path: the
// persistent batched kernel reads, in a later step of the same launch, state
// that other CTAs have written, which only L2 holds coherently.
template <typename Real>
__device__ __forceinline__ Real ld_state(const Real *p) { return __ldcg(p); }

// Stages the input box [NQ + 2][BY][BX] of the tile at (x0, y0) with plain
// loads (periodic wrap / wall mirror); no barrier.
template <typename Real, int TX, int TY, bool COUPLED, bool WALLY, bool UPW>
__device__ __forceinline__ void stage_plain(const StepArgs<Real> &a, int x0, int y0, Real *__restrict__ box) {
    using S = TileShape<Real, TX, TY, COUPLED, UPW>;
    constexpr int BX = S::BX, BXY = S::BXY, H = S::H;
    for (int e = threadIdx.x; e < (S::NQ + 2) * BXY; e += S::NT) {
        const int z = e / BXY, r = e - z * BXY, by = r / BX, bx = r - by * BX;
        const int gx = wrap(x0 - 4 + bx, a.nx);
        const int gy = map_row<WALLY>(y0 - H - 1 + by, a.ny, true);
        if (!in_bounds(gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny, a.status)) continue;
        const long long g = (long long)gy * a.pitch + gx;
        constexpr int HG = int(S::off_hbox) - S::NQ * BXY;   // alignment gap before the history planes
        box[(HG != 0 && z >= S::NQ) ? e + HG : e] = z < S::NQ ? ld_state(a.src + z * a.plane + g)
                                                               : ld_state(a.hsrc + (z - S::NQ) * a.plane + g);
    }
}

// Stages the cells of an edge tile's box that lie outside the domain
// (periodic wrap / wall mirror) with plain loads, once TMA has placed the
// rest of the box (those cells hold its out-of-range fill until overwritten
// here): whole rows below y = 0 and at y >= ny, then the columns left of
// x = 0 and at x >= nx in the other rows.  Grids of at least a tile plus
// halo only (one wrap correction suffices); no barrier.
template <typename Real, int TX, int TY, bool COUPLED, bool WALLY, bool UPW>
__device__ __forceinline__ void stage_edges(const StepArgs<Real> &a, int x0, int y0, Real *__restrict__ box) {
    using S = TileShape<Real, TX, TY, COUPLED, UPW>;
    constexpr int BX = S::BX, BY = S::BY, BXY = S::BXY, H = S::H;
    constexpr int HG = int(S::off_hbox) - S::NQ * BXY;   // alignment gap before the history planes
    const int lc = x0 < 4 ? 4 - x0 : 0;                   // box columns left of x = 0
    const int rc = max(0, x0 + TX + 4 - a.nx);            // box columns at x >= nx
    const int tr = max(0, H + 1 - y0);                    // box rows below y = 0
    const int br = max(0, y0 + TY + H + 1 - a.ny);        // box rows at y >= ny
    const int nrow = (tr + br) * BX;
    const int w = lc + rc;
    const int ncell = nrow + (BY - tr - br) * w;
    for (int e = threadIdx.x; e < (S::NQ + 2) * ncell; e += S::NT) {
        const int z = e / ncell, c = e - z * ncell;
        int bx, by;
        if (c < nrow) {
            const int r = c / BX;
            bx = c - r * BX;
            by = r < tr ? r : BY - br + (r - tr);
        } else {
            const int r = (c - nrow) / w, k = c - nrow - r * w;
            by = tr + r;
            bx = k < lc ? k : BX - rc + (k - lc);
        }
        const int gx = wrap1(x0 - 4 + bx, a.nx);
        const int gy = map_row<WALLY>(y0 - H - 1 + by, a.ny, false);
        if (!in_bounds(gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny && bx >= 0 && bx < BX && by >= 0 && by < BY,
                       a.status))
            continue;
        const long long g = (long long)gy * a.pitch + gx;
        const int b = z * BXY + by * BX + bx;
        box[(HG != 0 && z >= S::NQ) ? b + HG : b] = z < S::NQ ? ld_state(a.src + z * a.plane + g)
                                                               : ld_state(a.hsrc + (z - S::NQ) * a.plane + g);
    }
}

// Phase 0 of a tile: stages the input box [NQ + 2][BY][BX] at `box`, one TMA
// load per array (an edge tile's out-of-domain cells then overwritten by
// stage_edges), or plain loads throughout on grids smaller than a tile plus
// halo.  Ends with the box visible to every thread of the CTA.  Returns false
// if the CTA gave up on a TMA copy that timed out (STATUS_TIMEOUT is set; the
// tile must not be computed).
template <typename Real, int TX, int TY, bool COUPLED, bool WALLY, bool UPW>
__device__ __forceinline__ bool stage_box(const CUtensorMap *tm_state_p, const CUtensorMap *tm_hist_p,
                                          const StepArgs<Real> &a, int x0, int y0, Real *__restrict__ box,
                                          uint64_t *bar, int *staged_ok, bool *bar_live = nullptr) {
    using S = TileShape<Real, TX, TY, COUPLED, UPW>;
    constexpr int BXY = S::BXY;
    constexpr int H = S::H;
    const int tid = threadIdx.x;
    const int nx = a.nx, ny = a.ny;
    const bool interior = x0 >= 4 && x0 + TX + 4 <= nx && y0 >= H + 1 && y0 + TY + H + 1 <= ny;
    if (tid == 0) {
        int mode = 0;  // 0: plain loads, 1: staged by TMA, 2: TMA timed out
        if (a.use_tma && !a.small && !(*((volatile unsigned *)a.status) & STATUS_TIMEOUT)) {
            if (bar_live) {   // a CTA that stages several tiles: re-arm the barrier of the last one
                if (*bar_live) mbar_inval(bar);
                *bar_live = true;
            }
            mbar_init(bar, 1);
            mbar_expect_tx(bar, (uint32_t)((S::NQ + 2) * BXY * sizeof(Real)));
            tma_load_3d(box, tm_state_p, x0 - 4, y0 - H - 1, 0, bar);
            tma_load_3d(box + S::off_hbox, tm_hist_p, x0 - 4, y0 - H - 1, 0, bar);
            mode = 1;
            if (!mbar_wait(bar, 0, kPollLimit)) {
                atomicOr(a.status, STATUS_TIMEOUT);
                mbar_wait(bar, 0, kPollLimit);  // let copies in flight land before the CTA exits
                mode = 2;
            }
        }
        *staged_ok = mode;
    }
    __syncthreads();
    const int mode = *staged_ok;
    if (mode == 2) return false;
    if (mode == 1) {
        mbar_wait(bar, 0, 1);  // completed phase: makes the TMA writes visible to this thread
        if (!interior) {
            stage_edges<Real, TX, TY, COUPLED, WALLY, UPW>(a, x0, y0, box);
            __syncthreads();
        }
    } else {
        stage_plain<Real, TX, TY, COUPLED, WALLY, UPW>(a, x0, y0, box);
        __syncthreads();
    }
    return true;
}

template <typename Real, int TX, int TY, bool COUPLED, bool WALLY, bool UPW>
__device__ __forceinline__ void step_tile(const CUtensorMap *tm_state_p, const CUtensorMap *tm_hist_p,
                                          const StepArgs<Real> &a, const Phys<Real> &ph, int x0, int y0,
                                          bool *bar_live = nullptr) {
    using S = TileShape<Real, TX, TY, COUPLED, UPW>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // 128-byte aligned base for the TMA destinations, whatever the runtime gives
    Real *sm = reinterpret_cast<Real *>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
    Real *box = sm + S::off_box;
    Real *sphi = sm + S::off_phi;
    Real *rec = sm + S::off_rec;
    Real *aux = sm + S::off_aux;
    Real *sdy = sm + S::off_dy;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + S::off_bar);
    int *staged_ok = reinterpret_cast<int *>(bar + 1);

    // 0. stage the input box [NQ + 2][BY][BX]
    if (!stage_box<Real, TX, TY, COUPLED, WALLY, UPW>(tm_state_p, tm_hist_p, a, x0, y0, box, bar, staged_ok,
                                                       bar_live))
        return;

    tile_compute<Real, TX, TY, COUPLED, WALLY, UPW>(a, ph, x0, y0, box, sphi, rec, aux, sdy);
}

// Phases 1-4 of one tile whose input box is staged at `box` (the face
// records reuse it); sphi, rec, aux, sdy: the tile's other shared arrays.
template <typename Real, int TX, int TY, bool COUPLED, bool WALLY, bool UPW>
__device__ __forceinline__ void tile_compute(const StepArgs<Real> &a, const Phys<Real> &ph, int x0, int y0,
                                             Real *__restrict__ box, Real *__restrict__ sphi, Real *__restrict__ rec,
                                             Real *__restrict__ aux, Real *__restrict__ sdy) {
    using S = TileShape<Real, TX, TY, COUPLED, UPW>;
    constexpr int RS = S::RS, AS = S::AS, FS = S::FS, BX = S::BX, BXY = S::BXY;
    constexpr int H = S::H;
    Real *sfx = box + S::off_fx;
    Real *sfy = box + S::off_fy;
    const int tid = threadIdx.x;
    const int nx = a.nx, ny = a.ny, pitch = a.pitch;
    const long long plane = a.plane;

    // 1. phi' on the halo-(H+1) region; FP32 with the central scheme: two
    //    neighbouring cells per thread (8-byte aligned pairs, one packed add
    //    per plane, the same summation order per cell)
    if constexpr (DUGKS_PACKED_F32 && !S::F64 && (3 - H) % 2 == 0 && S::HX2 % 2 == 0) {
        for (int t = tid; t < S::N2 / 2; t += S::NT) {
            const int lx = (t % (S::HX2 / 2)) * 2, ly = t / (S::HX2 / 2);
            const float *p = reinterpret_cast<const float *>(box) + ly * BX + lx + 3 - H;
            float2 s = *reinterpret_cast<const float2 *>(p);
#pragma unroll
            for (int k = 1; k < 9; k++) s = add2(s, *reinterpret_cast<const float2 *>(p + k * BXY));
            *reinterpret_cast<float2 *>(reinterpret_cast<float *>(sphi) + ly * S::HX2 + lx) = s;
        }
    } else {
        for (int t = tid; t < S::N2; t += S::NT) {
            const int lx = t % S::HX2, ly = t / S::HX2;
            const Real *p = box + ly * BX + lx + 3 - H;
            Real s = p[0];
#pragma unroll
            for (int k = 1; k < 9; k++) s += p[k * BXY];
            sphi[t] = s;
        }
    }
    __syncthreads();

    // 2. items t < NC are the tile cells (their psi~+ partials stay in the
    //    registers of threads 0..NC-1), items t >= NC the halo ring
    Real tp[18];
    if (tid < S::NC)
        cell_item<Real, TX, TY, COUPLED, WALLY, UPW, true>(a, ph, box, sphi, rec, aux, sdy, tid % TX + H,
                                                           tid / TX + H, x0, y0, tp);
    for (int t = tid < S::NC ? tid + S::NT : tid; t < S::N1; t += S::NT) {
        const int r = t - S::NC;
        int hx, hy;
        if (H == 1) {   // ring: top row, bottom row, left column, right column
            if (r < S::HX1) { hx = r; hy = 0; }
            else if (r < 2 * S::HX1) { hx = r - S::HX1; hy = S::HY1 - 1; }
            else if (r < 2 * S::HX1 + TY) { hx = 0; hy = r - 2 * S::HX1 + 1; }
            else { hx = S::HX1 - 1; hy = r - 2 * S::HX1 - TY + 1; }
        } else {        // H top rows, H bottom rows, then H cells on each side of every tile row
            if (r < H * S::HX1) { hx = r % S::HX1; hy = r / S::HX1; }
            else if (r < 2 * H * S::HX1) { hx = (r - H * S::HX1) % S::HX1; hy = S::HY1 - H + (r - H * S::HX1) / S::HX1; }
            else {
                const int r3 = r - 2 * H * S::HX1, k = r3 % (2 * H);
                hy = H + r3 / (2 * H);
                hx = k < H ? k : TX + k;
            }
        }
        cell_item<Real, TX, TY, COUPLED, WALLY, UPW, false>(a, ph, box, sphi, rec, aux, sdy, hx, hy, x0, y0, nullptr);
    }
    __syncthreads();

    // 3. faces: x-faces (west face of local cell (fx, fy)), then y-faces (south face)
    //    (the y-face items start on a warp boundary, so no warp mixes both
    //    kinds: 0.333 -> 0.324 ms per FP32 2048^2 step on GB300)
    for (int t = tid; t < S::NFXP + S::NFY; t += S::NT) {
        Real fb[9], gb[9], out[12];
        Real au[4], bu[4], ady, bdy;
        if (t < S::NFXP) {
            if (t >= S::NFX) continue;
            const int fx = t % (TX + 1), fy = t / (TX + 1);
            const int gyr = y0 + fy;
            if (gyr >= ny || x0 + fx - 1 >= nx) continue;
            const int L = (fy + H) * S::HX1 + fx + H - 1, Rr = L + 1;
            // records read: L, Rr and their tangential neighbours (+- one row); upwind also L - 1, Rr + 1
            if (!in_bounds(L - S::HX1 >= 0 && Rr + S::HX1 < S::N1 && (!UPW || (L - 1 >= 0 && Rr + 1 < S::N1)),
                           a.status))
                continue;
            int tmode = 0;
            if (WALLY) tmode = (gyr == 0) ? 1 : ((gyr == ny - 1) ? -1 : 0);
            if (UPW)
                recon_face_upwind<Real, COUPLED, true, RS>(rec, L, Rr, 1, S::HX1, ph.h, fb, gb, tmode);
            else
                recon_face<Real, COUPLED, true, RS>(rec, L, Rr, S::HX1, tmode, ph.h, fb, gb);
            ld4(aux + L * AS, au);
            ld4(aux + Rr * AS, bu);
            ady = S::F64 ? aux[L * AS + 4] : sdy[L];
            bdy = S::F64 ? aux[Rr * AS + 4] : sdy[Rr];
            const Real hf = Real(0.5);
            const int gxf = x0 + fx >= nx ? x0 + fx - nx : x0 + fx;   // face coordinate in [0, nx)
            Real uf[2];
            if (!COUPLED && ph.vel_kind == 4) {   // R15: face i+1/2 of row gyr between columns gxl and gxf
                const int gxl = x0 + fx - 1 < 0 ? x0 + fx - 1 + nx : x0 + fx - 1;
                const long long kl = (long long)gyr * pitch + gxl, kr = (long long)gyr * pitch + gxf;
                if (!in_bounds(gxl >= 0 && gxl < nx && gxf >= 0 && gxf < nx && gyr >= 0 && gyr < ny, a.status)) continue;
                uf[0] = a.vel_faces ? a.vel[2 * plane + kl] : hf * (a.vel[kl] + a.vel[kr]);
                uf[1] = hf * (a.vel[plane + kl] + a.vel[plane + kr]);
            }
            face_flux<Real, COUPLED, true>(ph, fb, gb, hf * (au[0] + bu[0]), hf * (au[1] + bu[1]), hf * (au[2] + bu[2]),
                                           hf * (au[3] + bu[3]), hf * (ady + bdy), false, out, Real(gxf),
                                           Real(gyr) + Real(0.5), a.t_n + double(ph.h),
                                           (!COUPLED && ph.vel_kind == 4) ? uf : nullptr);
            store_flux<Real, COUPLED, FS>(sfx + t * FS, out);
        } else {
            const int u = t - S::NFXP;
            const int fx = u % TX, fy = u / TX;
            const int gyf = y0 + fy;  // face below row gyf
            if (x0 + fx >= nx || gyf - 1 >= ny) continue;
            const int D = (fy + H - 1) * S::HX1 + fx + H, U = D + S::HX1;
            // records read: D, U and their tangential neighbours (+- 1); upwind also D - HX1, U + HX1
            if (!in_bounds(D - 1 >= 0 && U + 1 < S::N1 && (!UPW || (D - S::HX1 >= 0 && U + S::HX1 < S::N1)),
                           a.status))
                continue;
            if (WALLY && (gyf == 0 || gyf == ny)) {
                const bool top = (gyf == ny);
                const int c0 = top ? D : U;
                if (!in_bounds(c0 - S::HX1 >= 0 && c0 + S::HX1 < S::N1, a.status)) continue;
                if (top)
                    recon_wall<Real, COUPLED, true, RS, UPW>(rec, c0, -S::HX1, ph.h, fb, gb);
                else
                    recon_wall<Real, COUPLED, false, RS, UPW>(rec, c0, S::HX1, ph.h, fb, gb);
                ld4(aux + c0 * AS, au);
                face_flux<Real, COUPLED, false>(ph, fb, gb, au[0], Real(0), au[2], au[3], Real(0), true, out);
            } else {
                if (UPW)
                    recon_face_upwind<Real, COUPLED, false, RS>(rec, D, U, S::HX1, 1, ph.h, fb, gb, 0,
                                                                WALLY && gyf - 1 == 0, WALLY && gyf == ny - 1);
                else
                    recon_face<Real, COUPLED, false, RS>(rec, D, U, 1, 0, ph.h, fb, gb);
                ld4(aux + D * AS, au);
                ld4(aux + U * AS, bu);
                ady = S::F64 ? aux[D * AS + 4] : sdy[D];
                bdy = S::F64 ? aux[U * AS + 4] : sdy[U];
                const Real hf = Real(0.5);
                const int gyw = (!WALLY && gyf >= ny) ? gyf - ny : gyf;   // face coordinate in [0, ny)
                Real uf[2];
                if (!COUPLED && ph.vel_kind == 4) {   // R15: face below row gyw of column x0 + fx
                    const int gyd = gyw - 1 < 0 ? gyw - 1 + ny : gyw - 1;
                    const long long kd = (long long)gyd * pitch + x0 + fx, ku = (long long)gyw * pitch + x0 + fx;
                    if (!in_bounds(gyd >= 0 && gyd < ny && gyw >= 0 && gyw < ny, a.status)) continue;
                    uf[0] = hf * (a.vel[kd] + a.vel[ku]);
                    uf[1] = a.vel_faces ? a.vel[3 * plane + ku] : hf * (a.vel[plane + kd] + a.vel[plane + ku]);
                }
                face_flux<Real, COUPLED, false>(ph, fb, gb, hf * (au[0] + bu[0]), hf * (au[1] + bu[1]),
                                                hf * (au[2] + bu[2]), hf * (au[3] + bu[3]), hf * (ady + bdy), false, out,
                                                Real(x0 + fx) + Real(0.5), Real(gyw), a.t_n + double(ph.h),
                                                (!COUPLED && ph.vel_kind == 4) ? uf : nullptr);
            }
            store_flux<Real, COUPLED, FS>(sfy + u * FS, out);
        }
    }
    __syncthreads();

    // 4. the flux update of the tile
    if (tid < S::NC) {
        const int lx = tid % TX, ly = tid / TX;
        const int gx = x0 + lx, gy = y0 + ly;
        if (gx < nx && gy < ny && in_bounds(gx >= 0 && gy >= 0 && gx < pitch, a.status)) {
            const long long g = (long long)gy * pitch + gx;
            const Real dt = ph.dt;
            // Each axis adds dt (psi_in - psi_out): the difference first, so a
            // cell with equal fluxes on both sides (a flat region) keeps its value.
            Real v[12], u[12];
            // west (+) and east (-) x-faces
            load_flux<Real, COUPLED, FS>(sfx + (ly * (TX + 1) + lx) * FS, v);
            load_flux<Real, COUPLED, FS>(sfx + (ly * (TX + 1) + lx + 1) * FS, u);
#pragma unroll
            for (int q = 0; q < S::NQ; q++) {
                const int m = q / 9, k = q % 9;
                if (cx(k) != 0) tp[q] += dt * sgnmul(cx(k), v[6 * m + xslot(k)] - u[6 * m + xslot(k)]);
            }
            // south (+) and north (-) y-faces
            load_flux<Real, COUPLED, FS>(sfy + (ly * TX + lx) * FS, v);
            load_flux<Real, COUPLED, FS>(sfy + ((ly + 1) * TX + lx) * FS, u);
#pragma unroll
            for (int q = 0; q < S::NQ; q++) {
                const int m = q / 9, k = q % 9;
                if (cy(k) != 0) tp[q] += dt * sgnmul(cy(k), v[6 * m + yslot(k)] - u[6 * m + yslot(k)]);
            }
#pragma unroll
            for (int q = 0; q < S::NQ; q++) a.dst[q * plane + g] = tp[q];
        }
    }
}

// ---------------------------------------------------------------------------
// The batched step kernel: a batch of independent problems of the same
// precision, model and y-boundary.  CTA b runs the (problem, tile) item
// work[b]; the problem's buffers, constants, tensor maps, buffer parity and
// step count come from its descriptor (parity and count advanced on the
// device by advance_kernel after each batched step).  solo_step_kernel below
// runs the same tile code for one problem.
// ---------------------------------------------------------------------------
template <typename Real>
struct InstDesc {
    CUtensorMap tm_state[2], tm_hist[2];  // 64-byte aligned maps of both ping-pong buffers
    Real *state[2];
    Real *hist[2];
    unsigned *status;
    Phys<Real> ph;
    long long plane;
    long long steps;                       // step count (batched use)
    int nx, ny, pitch, tiles_x;
    int ntiles;                            // tiles of one step of this problem
    int cur;                               // buffer holding psi~^n (batched use)
    int use_tma;
    const Real *vel;                       // sampled velocity field, or null
    int vel_faces;
};

template <typename Real, int TX, int TY, bool COUPLED, bool WALLY, bool UPW = false>
__global__ void __launch_bounds__((TileShape<Real, TX, TY, COUPLED, UPW>::NT),
                                  (TileShape<Real, TX, TY, COUPLED, UPW>::MINB))
step_kernel(const InstDesc<Real> *__restrict__ descs, const int2 *__restrict__ work) {
    const int2 item = work[blockIdx.x];   // (problem, tile)
    const InstDesc<Real> *d = descs + item.x;
    const int cur = d->cur;
    const long long steps = d->steps;
    StepArgs<Real> a;
    a.src = d->state[cur];
    a.dst = d->state[cur ^ 1];
    a.hsrc = d->hist[cur];
    a.hdst = d->hist[cur ^ 1];
    a.nx = d->nx;
    a.ny = d->ny;
    a.pitch = d->pitch;
    a.plane = d->plane;
    a.first_step = steps == 0;
    a.t_n = double(steps) * double(d->ph.dt);
    a.small = (a.nx < TX + 4 || a.ny < TY + 4) ? 1 : 0;
    a.use_tma = d->use_tma;
    a.vel = d->vel;
    a.vel_faces = d->vel_faces;
    a.status = d->status;
    const Phys<Real> &ph = d->ph;   // read-only: reloaded on demand rather than pinned in registers
    const int tx = item.y % d->tiles_x, ty = item.y / d->tiles_x;
    step_tile<Real, TX, TY, COUPLED, WALLY, UPW>(&d->tm_state[cur], &d->tm_hist[cur], a, ph, tx * TX, ty * TY);
}

// One step of a single problem.  Tensor maps, arguments and constants arrive
// in the kernel's parameter space, which the arithmetic instructions read as
// constant-bank operands without occupying registers; the tile code is the
// same inlined function the batched kernel runs (which loads the constants
// from its descriptor, so the compiler may contract multiply-adds differently
// and the two agree to round-off).
#ifndef DUGKS_SOLO_MINB
#define DUGKS_SOLO_MINB 0   // 0: the occupancy the shared memory allows
#endif
template <typename Real, int TX, int TY, bool COUPLED, bool WALLY, bool UPW = false>
__global__ void __launch_bounds__((TileShape<Real, TX, TY, COUPLED, UPW>::NT),
                                  (DUGKS_SOLO_MINB > 0 ? DUGKS_SOLO_MINB : TileShape<Real, TX, TY, COUPLED, UPW>::MINB))
solo_step_kernel(const __grid_constant__ CUtensorMap tm_state, const __grid_constant__ CUtensorMap tm_hist,
                 const __grid_constant__ StepArgs<Real> a, const __grid_constant__ Phys<Real> ph, int tiles_x) {
    const int tile = (int)blockIdx.x;
    step_tile<Real, TX, TY, COUPLED, WALLY, UPW>(&tm_state, &tm_hist, a, ph, (tile % tiles_x) * TX,
                                                 (tile / tiles_x) * TY);
}

// K steps of a batch group in one persistent launch.  The CTAs (as many as
// fit on the GPU) take items from one queue, in order: the items of step 0
// of every member, then those of step 1, and so on; item i is step i / nwork
// of the (problem, tile) pair work[i % nwork].  A tile of step s + 1 of a
// problem waits only until every tile of step s of that problem is done
// (its counter, ctr[1 + problem], has reached (s + 1) x its tile count), so
// a small member runs ahead of a large one instead of waiting at a step
// boundary of the whole batch.  Progress does not depend on the CTAs being
// resident together: an item is taken only by a running CTA that has
// finished its previous one, and every item it waits for comes earlier in the
// queue, so the earliest unfinished item is being worked on and never waits.
// (Claiming the next item while computing the current one made a CTA hold
// two items of consecutive steps, which serialised them: FP64 steps of two
// 128^2 members took 136 us instead of 97.)  Each
// wait is bounded (about 2 s of sleeps): on running out it flags the problem's
// status word (STATUS_TIMEOUT) and goes on, so a fault cannot hang the
// launch.  The counters start at zero (the launcher clears them); the
// descriptors' buffer parity and step count advance after the launch.
constexpr unsigned long long kItemWaitNs = 2000000000ull;   // sleep budget of one wait (about 2 s)

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
    unsigned v = 0;
#ifdef __CUDA_ARCH__
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
#endif
    return v;
}
// Adds 1 with release semantics at GPU scope: the CTA's writes that a barrier
// ordered before this are visible to whoever acquires the new count.
__device__ __forceinline__ void red_release_gpu_add1(unsigned *p) {
#ifdef __CUDA_ARCH__
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(p) : "memory");
#endif
}
// Orders this thread's earlier (generic) observations before its later TMA
// (async proxy) reads of global memory.
__device__ __forceinline__ void fence_proxy_async_global() {
#ifdef __CUDA_ARCH__
    asm volatile("fence.proxy.async.global;" ::: "memory");
#endif
}

// Waits until *done >= need (a member's counter; nt of its tiles per step),
// sleeping in proportion to how many steps the member is behind, so that
// CTAs waiting many steps ahead do not crowd the counter.  Returns false if
// budget_ns of sleeps pass first.
__device__ __forceinline__ bool member_wait(const unsigned *done, unsigned need, unsigned nt,
                                            unsigned long long budget_ns) {
    unsigned long long slept = 0;
    for (unsigned have; (have = ld_acquire_gpu(done)) < need;) {
        if (slept > budget_ns) return false;
        const unsigned behind = (need - have + nt - 1) / nt;
        const unsigned ns = behind > 1 ? (behind < 16 ? 1000u * (behind - 1) : 15000u) : 100u;
        __nanosleep(ns);
        slept += ns;
    }
    return true;
}

template <typename Real, int TX, int TY, bool COUPLED, bool WALLY, bool UPW = false>
__global__ void __launch_bounds__((TileShape<Real, TX, TY, COUPLED, UPW>::NT),
                                  (TileShape<Real, TX, TY, COUPLED, UPW>::MINB))
persistent_step_kernel(const InstDesc<Real> *__restrict__ descs, const int2 *__restrict__ work, int nwork,
                       int ksteps, unsigned *ctr) {
    using S = TileShape<Real, TX, TY, COUPLED, UPW>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Real *sm = reinterpret_cast<Real *>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
    // the queue position, in the spare word after the barrier and the staging flag
    volatile int *slot = reinterpret_cast<int *>(reinterpret_cast<uint64_t *>(sm + S::off_bar) + 1) + 1;
    const int tid = threadIdx.x;
    const unsigned total = (unsigned)ksteps * (unsigned)nwork;
    bool bar_live = false;
    if (tid == 0) *slot = (int)atomicAdd(ctr, 1u);
    __syncthreads();
    for (;;) {
        const unsigned i = (unsigned)*slot;
        if (i >= total) break;
        const unsigned s = i / (unsigned)nwork;
        const int2 item = work[i - s * (unsigned)nwork];
        const InstDesc<Real> *d = descs + item.x;
        if (tid == 0) {
            const unsigned *done = ctr + 1 + item.x;
            const unsigned nt = (unsigned)d->ntiles;
            if (s > 0 && !member_wait(done, s * nt, nt, kItemWaitNs)) atomicOr(d->status, STATUS_TIMEOUT);
            fence_proxy_async_global();
        }
        __syncthreads();
        const int cur = d->cur ^ (int)(s & 1u);
        const long long steps = d->steps + (long long)s;
        StepArgs<Real> a;
        a.src = d->state[cur];
        a.dst = d->state[cur ^ 1];
        a.hsrc = d->hist[cur];
        a.hdst = d->hist[cur ^ 1];
        a.nx = d->nx;
        a.ny = d->ny;
        a.pitch = d->pitch;
        a.plane = d->plane;
        a.first_step = steps == 0;
        a.t_n = double(steps) * double(d->ph.dt);
        a.small = (a.nx < TX + 4 || a.ny < TY + 4) ? 1 : 0;
        a.use_tma = d->use_tma;
        a.vel = d->vel;
        a.vel_faces = d->vel_faces;
        a.status = d->status;
        const Phys<Real> &ph = d->ph;
        const int tx = item.y % d->tiles_x, ty = item.y / d->tiles_x;
        step_tile<Real, TX, TY, COUPLED, WALLY, UPW>(&d->tm_state[cur], &d->tm_hist[cur], a, ph, tx * TX, ty * TY,
                                                     &bar_live);
        __syncthreads();   // every store of the tile is issued before the release below
        if (tid == 0) {
            // the member is looked up again rather than kept in registers through the tile
            const unsigned j = (unsigned)*slot;
            red_release_gpu_add1(ctr + 1 + work[j % (unsigned)nwork].x);
            *slot = (int)atomicAdd(ctr, 1u);
        }
        __syncthreads();   // the next position is visible; the tile's shared memory is free
    }
}

// After k batched steps: every instance's buffers swap k times and its step count grows by k.
template <typename Real>
__global__ void advance_kernel(InstDesc<Real> *descs, int n, int k) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        descs[i].cur ^= (k & 1);
        descs[i].steps += k;
    }
}

}  // namespace dugks
