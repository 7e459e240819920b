/*
 * dugks_oracle.c -- plain FP64 restatement of one time step of the
 * phase-field DUGKS of Yang, Zhong & Zhuo (arXiv:1810.07802), Sec. II.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * bench's CPU-baseline leg; never by the product path.  It is written to be
 * checked against the paper by eye: one whole-grid loop per stage of the
 * scheme, in the paper's order, with whole-grid temporaries and no fusion.
 * Compiled with -O2 -ffp-contract=off.
 *
 * Readings of passages the paper leaves open (the CUDA path takes the same):
 *  R1  RT = 1/3, so sqrt(3RT) = 1, xi_i = e_i and dt = CFL (delta_x = 1,
 *      Eq. 37); Fig. 1's caption pairs CFL 0.5 with dt 0.5.
 *  R2  Central reconstruction of psi-bar-plus at x_f - xi h (Eq. 27, "central
 *      scheme" of Sec. II.B): linear profile through the face with
 *        value            = mean of the two cells sharing the face,
 *        normal slope     = difference of those two cells,
 *        tangential slope = mean of their central differences,
 *      psi_bar(x_f, t+h) = value - h (xi . slope).
 *  R3  Face macros: phi_f = sum_i f_bar_i; u_f and p_f from g_bar by Eqs.
 *      32-33 with h in place of dt (psi_bar is psi shifted by h/2 of
 *      collision and source, as psi~ is by dt/2); grad phi, lap phi and
 *      d_t(phi u) at the face are the means of the two adjacent cells.
 *  R4  "Six-point" gradient = isotropic D2Q9 gradient
 *      (1/RT) sum_i w_i xi_i phi(x + xi_i); "nine-point" Laplacian
 *      = [4 (E+W+N+S) + (NE+NW+SE+SW) - 20 C] / 6.
 *  R5  d_t(phi u) in Eq. 16 by the explicit difference
 *      ((phi u)^n - (phi u)^{n-1}) / dt, and 0 on the first step.
 *  R6  n = grad phi / sqrt(|grad phi|^2 + 1e-16): the unit normal wherever an
 *      interface is resolved (|grad phi| >> 1e-8), and a continuous function
 *      of grad phi where it vanishes, so that round-off in a flat region
 *      cannot flip n between 0 and a unit vector.
 *  R7  Initial state psi~ = psi_eq - dt/2 S (Eq. 23a with psi = psi_eq) and
 *      d_t(phi u) = 0; (phi u)^{-1} = phi0 u0.
 *  R8  Gravity G = (gx, gy), or (rho - rho_ref)(gx, gy).
 *  R9  No-slip walls on the faces y = 0 and y = ny: phi mirrored into ghost
 *      rows (phi(-1) = phi(0), phi(ny) = phi(ny-1)); x-faces in the first and
 *      last row take a one-sided y-slope (into the fluid); at a wall face a
 *      direction that leaves the fluid or runs along the wall is
 *      extrapolated linearly from the adjacent cell, and one that enters
 *      the fluid takes the value of its opposite direction (bounce-back);
 *      the wall face has u = 0, and its grad phi and d_t(phi u) are the
 *      adjacent cell's with the normal component removed (the mean of the
 *      cell and its mirror image), its lap phi is the adjacent cell's.
 *  R10 No clamping of phi, rho or mu.
 *  R12 Prescribed velocity fields of the A-C-only model are evaluated
 *      analytically: at cell centres at t_n = n dt, at face centres at
 *      t_n + h (the time of the face distributions), with face coordinates
 *      taken in [0, nx) x [0, ny) on periodic axes.  The reversing shear
 *      (Eq. 42) changes sign for t >= L0/U0.
 *  R15 Sampled velocity field (velocity_field 4, the boundary's
 *      dugks_set_velocity_field): u at cell centres from a [ny][nx] pair of
 *      arrays (initially the ux0, uy0 given at creation), steady between
 *      updates; at a face, the normal component from an optional face array
 *      (x-face i+1/2 of row j at [j][i], y-face below row j at [j][i]), else
 *      the mean of the two cells, and the tangential component the mean of
 *      the two cells (as R3 takes face values of cell quantities); wall faces
 *      keep u = 0.
 *  R16 Sec. IV.A keeps one kinematic viscosity for the whole field of the
 *      stationary bubble: tau_g = nu / RT everywhere, which is Eq. 36 (visc
 *      = 1) with mu_H / mu_L = rho_H / rho_L; the bubble workloads select it.
 *  R14 Upwind reconstruction (recon = 1; Sec. II.B names the upwind scheme
 *      as the alternative to the central one, and Sec. III.A the fix for
 *      its high-Peclet error, without printing it): each of the two cells
 *      sharing the face carries a linear profile of psi-bar-plus with
 *      per-axis slopes from van Leer's limiter of its two one-sided
 *      differences, sigma = 2 s1 s2 / (s1 + s2) if s1 s2 > 0 else 0; the
 *      value at x_f - xi h is taken from the profile of the upwind cell
 *      (the one xi . n points away from), and for xi . n = 0 it is the mean
 *      of the two profiles.
 *  R17 The upwind reconstruction with no-slip walls (R9 for the profiles of
 *      R14): a cell of the first or last row takes its one-sided y-difference
 *      into the fluid as its y-slope; at a wall face a direction leaving the
 *      fluid or running along the wall takes the adjacent cell's profile at
 *      x_f - xi h, one entering the fluid bounces back.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "dugks_oracle.h"

#define Q 9
#define RT (1.0 / 3.0)

/* D2Q9 velocities in the paper's order and weights (Eq. 14). */
static const int EX[Q] = {0, 1, 1, 0, -1, -1, -1, 0, 1};
static const int EY[Q] = {0, 0, 1, 1, 1, 0, -1, -1, -1};
static const double WQ[Q] = {4.0 / 9.0,  1.0 / 9.0, 1.0 / 36.0,
                             1.0 / 9.0,  1.0 / 36.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 9.0, 1.0 / 36.0};

static int opposite(int i) { return i == 0 ? 0 : ((i + 3) % 8) + 1; }

struct oracle_ctx {
    oracle_params P;
    long n;            /* steps taken */
    double *vel;       /* velocity_field 4: ux, uy at cells, ux at x-faces, uy at y-faces ([4][ny][nx]) */
    int vel_faces;     /* the face planes of vel are set (else faces take the mean of their cells) */
    double *f, *g;     /* psi~ : [9][ny][nx] each */
    double *phiu;      /* (phi u)^{n-1} : [2][ny][nx] */
    double *snap;      /* phi, ux, uy at the previous oracle_reduce call */
    int have_snap;
};

/* Everything the scheme needs at one point (cell centre or face). */
typedef struct {
    double phi, dphix, dphiy, lap;
    double rho, drhox, drhoy;
    double muphi, mu, tau_g;
    double theta, nx, ny;
    double Fx, Fy;
    double ux, uy, p;
    double Dx, Dy;
} point_state;

void oracle_lattice(int *ex, int *ey, double *w)
{
    for (int i = 0; i < Q; i++) {
        ex[i] = EX[i];
        ey[i] = EY[i];
        w[i] = WQ[i];
    }
}

/* Gamma_i(u), Eq. 18. */
static double gamma_i(int i, double ux, double uy)
{
    double eu = EX[i] * ux + EY[i] * uy;
    return WQ[i] * (1.0 + eu / RT + eu * eu / (2.0 * RT * RT) - (ux * ux + uy * uy) / (2.0 * RT));
}

/* Eq. 15 with c_s^2 = RT. */
void oracle_feq(double phi, double ux, double uy, double *feq)
{
    for (int i = 0; i < Q; i++)
        feq[i] = WQ[i] * phi * (1.0 + (EX[i] * ux + EY[i] * uy) / RT);
}

/* Eq. 16: S^f_i = w_i theta xi_i.n + w_i xi_i . d_t(phi u) / RT. */
void oracle_sf(double theta, double nx, double ny, double Dx, double Dy, double *sf)
{
    for (int i = 0; i < Q; i++)
        sf[i] = WQ[i] * theta * (EX[i] * nx + EY[i] * ny) + WQ[i] * (EX[i] * Dx + EY[i] * Dy) / RT;
}

/* Eq. 17. */
void oracle_geq(double p, double rho, double ux, double uy, double *geq)
{
    for (int i = 0; i < Q; i++) {
        double rest = (i == 0) ? (WQ[i] - 1.0) : WQ[i];
        geq[i] = p / RT * rest + rho * (gamma_i(i, ux, uy) - gamma_i(i, 0.0, 0.0));
    }
}

/* Eq. 19 with grad(rho RT) = RT grad rho (RT is constant). */
void oracle_sg(double drhox, double drhoy, double Fx, double Fy,
               double ux, double uy, double *sg)
{
    for (int i = 0; i < Q; i++) {
        double gu = gamma_i(i, ux, uy);
        double g0 = gamma_i(i, 0.0, 0.0);
        double ax = (gu - g0) * RT * drhox + Fx * gu;
        double ay = (gu - g0) * RT * drhoy + Fy * gu;
        sg[i] = ((EX[i] - ux) * ax + (EY[i] - uy) * ay) / RT;
    }
}

/* Eqs. 29-30. */
void oracle_prestep(double tau, double dt, const double *tilde, const double *eq,
                    const double *src, double *bar_plus, double *tilde_plus)
{
    double h = 0.5 * dt;
    for (int i = 0; i < Q; i++) {
        bar_plus[i] = (2.0 * tau - h) / (2.0 * tau + dt) * tilde[i]
                    + 3.0 * h / (2.0 * tau + dt) * eq[i]
                    + 3.0 * tau * h / (2.0 * tau + dt) * src[i];
        tilde_plus[i] = 4.0 / 3.0 * bar_plus[i] - 1.0 / 3.0 * tilde[i];
    }
}

/* Eq. 28. */
void oracle_face_psi(double tau, double h, const double *bar, const double *eq,
                     const double *src, double *psi)
{
    for (int i = 0; i < Q; i++)
        psi[i] = 2.0 * tau / (2.0 * tau + h) * bar[i]
               + h / (2.0 * tau + h) * eq[i]
               + tau * h / (2.0 * tau + h) * src[i];
}

/* phi at cell (i, j): periodic in x; periodic or mirrored (R9) in y. */
static double phi_at(int nx, int ny, int wall_y, const double *phi, int i, int j)
{
    i = ((i % nx) + nx) % nx;
    if (wall_y) {
        if (j < 0) j = -1 - j;
        if (j >= ny) j = 2 * ny - 1 - j;
    } else {
        j = ((j % ny) + ny) % ny;
    }
    return phi[(long)j * nx + i];
}

/* R4. */
void oracle_grad_lap(int nx, int ny, int wall_y, const double *phi,
                     double *dphix, double *dphiy, double *lap)
{
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            double gx = 0.0, gy = 0.0;
            for (int q = 0; q < Q; q++) {
                double v = phi_at(nx, ny, wall_y, phi, i + EX[q], j + EY[q]);
                gx += WQ[q] * EX[q] * v;
                gy += WQ[q] * EY[q] * v;
            }
            double C = phi_at(nx, ny, wall_y, phi, i, j);
            double E = phi_at(nx, ny, wall_y, phi, i + 1, j);
            double Wv = phi_at(nx, ny, wall_y, phi, i - 1, j);
            double N = phi_at(nx, ny, wall_y, phi, i, j + 1);
            double S = phi_at(nx, ny, wall_y, phi, i, j - 1);
            double NE = phi_at(nx, ny, wall_y, phi, i + 1, j + 1);
            double NW = phi_at(nx, ny, wall_y, phi, i - 1, j + 1);
            double SE = phi_at(nx, ny, wall_y, phi, i + 1, j - 1);
            double SW = phi_at(nx, ny, wall_y, phi, i - 1, j - 1);
            long k = (long)j * nx + i;
            dphix[k] = gx / RT;
            dphiy[k] = gy / RT;
            lap[k] = (4.0 * (E + Wv + N + S) + (NE + NW + SE + SW) - 20.0 * C) / 6.0;
        }
}

/* Prescribed velocity of the A-C-only model at (x, y), time t (R12). */
static void prescribed_velocity(const oracle_params *P, double x, double y, double t, double *ux, double *uy)
{
    const double pi = 3.14159265358979323846;
    double U = P->vel_u0, L = P->vel_length;
    switch (P->velocity_field) {
    case 1:  /* rotation about the box centre, Eq. 41 */
        *ux = -U * pi / L * (y - 0.5 * L);
        *uy = U * pi / L * (x - 0.5 * L);
        break;
    case 2: {  /* shear, reversed after L0 / U0, Eq. 42 */
        double sgn = (t < L / U) ? 1.0 : -1.0;
        *ux = sgn * U * pi * sin(pi * x / L) * cos(pi * y / L);
        *uy = -sgn * U * pi * cos(pi * x / L) * sin(pi * y / L);
        break;
    }
    case 3: {  /* smoothed deformation with period T = L0 / U0, Eq. 43 */
        double c = cos(pi * t / (L / U));
        *ux = -U * sin(4.0 * pi * x / L) * sin(4.0 * pi * y / L) * c;
        *uy = -U * cos(4.0 * pi * x / L) * cos(4.0 * pi * y / L) * c;
        break;
    }
    default:  /* uniform, Eq. 40 */
        *ux = P->u0x;
        *uy = P->u0y;
    }
}

/* rho, grad rho, mu_phi, mu, tau_g, theta, n and F at a point whose phi,
 * grad phi and lap phi are set (Eqs. 3, 4, 6, 10, 34-36, R6, R8). */
static void closures(const oracle_params *P, point_state *s)
{
    double phi = s->phi;
    s->theta = -4.0 * (phi - 1.0) * (phi - 0.0) / (P->width * (1.0 - 0.0));   /* Eq. 6 */
    double gn = sqrt(s->dphix * s->dphix + s->dphiy * s->dphiy + 1e-16);   /* R6 */
    s->nx = s->dphix / gn;
    s->ny = s->dphiy / gn;
    if (P->model != 0) return;   /* A-C only: no hydrodynamics */

    double beta = 12.0 * P->sigma / P->width;     /* Eq. 3 */
    double kappa = 1.5 * P->sigma * P->width;     /* Eq. 3 */
    s->rho = (P->rho_h - P->rho_l) * phi + P->rho_l;        /* Eq. 10 */
    s->drhox = (P->rho_h - P->rho_l) * s->dphix;
    s->drhoy = (P->rho_h - P->rho_l) * s->dphiy;
    s->muphi = 4.0 * beta * (phi - 1.0) * (phi - 0.0) * (phi - 0.5) - kappa * s->lap;  /* Eq. 4 */
    if (P->visc == 0)
        s->mu = 1.0 / (phi * (1.0 / P->mu_h - 1.0 / P->mu_l) + 1.0 / P->mu_l);    /* Eq. 35 */
    else
        s->mu = phi * (P->mu_h - P->mu_l) + P->mu_l;                           /* Eq. 36 */
    s->tau_g = s->mu / (s->rho * RT);                                           /* Eq. 34 */
    double Gx = P->gx, Gy = P->gy;
    if (P->gravity_mode == 1) {
        Gx = (s->rho - P->rho_ref) * P->gx;
        Gy = (s->rho - P->rho_ref) * P->gy;
    }
    s->Fx = s->muphi * s->dphix + Gx;   /* F = F_s + G, F_s = mu_phi grad phi (Eq. 9) */
    s->Fy = s->muphi * s->dphiy + Gy;
}

/* Eq. 33 (half = dt/2 at a cell centre, h/2 at a face) with the point's u. */
static void pressure(double sum_nonrest, double half, point_state *s)
{
    double gamma0_shift = gamma_i(0, s->ux, s->uy) - gamma_i(0, 0.0, 0.0);
    s->p = RT / (1.0 - WQ[0]) * (sum_nonrest + half * (s->ux * s->drhox + s->uy * s->drhoy)
                                 + s->rho * gamma0_shift);
}

/* Eqs. 32-33 from the moments of g (psi~ at a cell, psi_bar at a face). */
static void velocity_pressure(const double *g9, double half, point_state *s)
{
    double mx = 0.0, my = 0.0, sum_nonrest = 0.0;
    for (int i = 0; i < Q; i++) {
        mx += EX[i] * g9[i];
        my += EY[i] * g9[i];
        if (i != 0) sum_nonrest += g9[i];
    }
    s->ux = (mx + half * s->Fx) / s->rho;
    s->uy = (my + half * s->Fy) / s->rho;
    pressure(sum_nonrest, half, s);
}

/* Macros at every cell centre (Eqs. 31-33) plus d_t(phi u) (R5). */
static void cell_states(const oracle_ctx *c, point_state *cs)
{
    const oracle_params *P = &c->P;
    int nx = P->nx, ny = P->ny;
    long N = (long)nx * ny;
    double dt = P->cfl;
    double *phi = calloc((size_t)N, sizeof(double));
    double *gx = calloc((size_t)N, sizeof(double));
    double *gy = calloc((size_t)N, sizeof(double));
    double *lp = calloc((size_t)N, sizeof(double));
    for (long k = 0; k < N; k++) {              /* Eq. 31 */
        double s = 0.0;
        for (int i = 0; i < Q; i++) s += c->f[i * N + k];
        phi[k] = s;
    }
    oracle_grad_lap(nx, ny, P->wall_y, phi, gx, gy, lp);
    for (long k = 0; k < N; k++) {
        point_state *s = &cs[k];
        memset(s, 0, sizeof *s);
        s->phi = phi[k];
        s->dphix = gx[k];
        s->dphiy = gy[k];
        s->lap = lp[k];
        closures(P, s);
        if (P->model == 0) {
            double g9[Q];
            for (int i = 0; i < Q; i++) g9[i] = c->g[i * N + k];
            velocity_pressure(g9, 0.5 * dt, s);
        } else if (P->velocity_field == 4) {
            s->ux = c->vel[k];
            s->uy = c->vel[N + k];
        } else {
            prescribed_velocity(P, (double)(k % nx) + 0.5, (double)(k / nx) + 0.5, (double)c->n * dt,
                                &s->ux, &s->uy);
        }
        if (c->n == 0) {
            s->Dx = 0.0;
            s->Dy = 0.0;
        } else {
            s->Dx = (s->phi * s->ux - c->phiu[k]) / dt;
            s->Dy = (s->phi * s->uy - c->phiu[N + k]) / dt;
        }
    }
    free(phi); free(gx); free(gy); free(lp);
}

/* R15: velocity of the sampled field (velocity_field 4) at a face between
 * cells ka and kb (axis 0: x-face, 1: y-face; kf the face's index): the
 * normal component from the face plane when one was given, else the mean of
 * the two cells; the tangential component the mean of the two cells. */
static void sampled_face_velocity(const oracle_ctx *c, int axis, long ka, long kb, long kf, double *uf)
{
    long N = (long)c->P.nx * c->P.ny;
    const double *v = c->vel;
    double ux = 0.5 * (v[ka] + v[kb]), uy = 0.5 * (v[N + ka] + v[N + kb]);
    if (c->vel_faces) {
        if (axis == 0) ux = v[2 * N + kf];
        else uy = v[3 * N + kf];
    }
    uf[0] = ux;
    uf[1] = uy;
}

/* Face state from the reconstructed psi_bar and the face means of grad phi,
 * lap phi and d_t(phi u) (R3), then the original distributions (Eq. 28). */
static void face_distributions(const oracle_ctx *c, const double *fbar, const double *gbar,
                               double dphix, double dphiy, double lap, double Dx, double Dy,
                               int wall_face, double xf, double yf, const double *uf,
                               double *fpsi, double *gpsi)
{
    const oracle_params *P = &c->P;
    double dt = P->cfl, h = 0.5 * dt;
    double tau_f = P->mobility / RT;   /* Eq. 34 */
    point_state s;
    memset(&s, 0, sizeof s);
    s.phi = 0.0;
    for (int i = 0; i < Q; i++) s.phi += fbar[i];
    s.dphix = dphix;
    s.dphiy = dphiy;
    s.lap = lap;
    s.Dx = Dx;
    s.Dy = Dy;
    closures(P, &s);
    if (P->model == 0) {
        velocity_pressure(gbar, 0.5 * h, &s);
        if (wall_face) {
            double sum_nonrest = 0.0;
            for (int i = 1; i < Q; i++) sum_nonrest += gbar[i];
            s.ux = 0.0;
            s.uy = 0.0;
            pressure(sum_nonrest, 0.5 * h, &s);
        }
    } else if (wall_face) {
        s.ux = 0.0;
        s.uy = 0.0;
    } else if (P->velocity_field == 4) {
        s.ux = uf[0];
        s.uy = uf[1];
    } else {
        prescribed_velocity(P, xf, yf, (double)c->n * dt + h, &s.ux, &s.uy);
    }
    double eq[Q], src[Q];
    oracle_feq(s.phi, s.ux, s.uy, eq);
    oracle_sf(s.theta, s.nx, s.ny, s.Dx, s.Dy, src);
    oracle_face_psi(tau_f, h, fbar, eq, src, fpsi);
    if (P->model == 0) {
        oracle_geq(s.p, s.rho, s.ux, s.uy, eq);
        oracle_sg(s.drhox, s.drhoy, s.Fx, s.Fy, s.ux, s.uy, src);
        oracle_face_psi(s.tau_g, h, gbar, eq, src, gpsi);
    }
}

/* R2 (and R9 for the first/last row with walls) at the x-face i+1/2 of row j. */
static void recon_xface(const oracle_params *P, const double *B, int i, int j, double *out)
{
    int nx = P->nx, ny = P->ny;
    long N = (long)nx * ny;
    double h = 0.5 * P->cfl;
    int ip = (i + 1) % nx;
    for (int q = 0; q < Q; q++) {
        const double *b = B + q * N;
        double L = b[(long)j * nx + i], R = b[(long)j * nx + ip];
        double sy;
        if (!P->wall_y) {
            int jp = (j + 1) % ny, jm = (j - 1 + ny) % ny;
            sy = 0.25 * ((b[(long)jp * nx + i] - b[(long)jm * nx + i])
                       + (b[(long)jp * nx + ip] - b[(long)jm * nx + ip]));
        } else if (j == 0) {
            sy = 0.5 * ((b[(long)1 * nx + i] - b[i]) + (b[(long)1 * nx + ip] - b[ip]));
        } else if (j == ny - 1) {
            sy = 0.5 * ((b[(long)(ny - 1) * nx + i] - b[(long)(ny - 2) * nx + i])
                      + (b[(long)(ny - 1) * nx + ip] - b[(long)(ny - 2) * nx + ip]));
        } else {
            sy = 0.25 * ((b[(long)(j + 1) * nx + i] - b[(long)(j - 1) * nx + i])
                       + (b[(long)(j + 1) * nx + ip] - b[(long)(j - 1) * nx + ip]));
        }
        double v = 0.5 * (L + R);
        double sx = R - L;
        out[q] = v - h * (EX[q] * sx + EY[q] * sy);
    }
}

/* R2 at the interior (or periodic) y-face between rows jm and jc of column i. */
static void recon_yface(const oracle_params *P, const double *B, int i, int jm, int jc, double *out)
{
    int nx = P->nx, ny = P->ny;
    long N = (long)nx * ny;
    double h = 0.5 * P->cfl;
    int ip = (i + 1) % nx, im = (i - 1 + nx) % nx;
    for (int q = 0; q < Q; q++) {
        const double *b = B + q * N;
        double D = b[(long)jm * nx + i], U = b[(long)jc * nx + i];
        double sx = 0.25 * ((b[(long)jm * nx + ip] - b[(long)jm * nx + im])
                          + (b[(long)jc * nx + ip] - b[(long)jc * nx + im]));
        double v = 0.5 * (D + U);
        double sy = U - D;
        out[q] = v - h * (EX[q] * sx + EY[q] * sy);
    }
}

/* van Leer's limiter of two one-sided differences: their harmonic mean, or 0
 * at an extremum (R14). */
static double van_leer(double s1, double s2)
{
    return s1 * s2 > 0.0 ? 2.0 * s1 * s2 / (s1 + s2) : 0.0;
}

/* y-slope of the upwind profile of cell (i, j) (R14): van Leer's limiter of
 * its two one-sided differences; with walls (R17) a cell of the first or last
 * row takes its one-sided difference into the fluid instead. */
static double upwind_yslope(const oracle_params *P, const double *b, int i, int j)
{
    int nx = P->nx, ny = P->ny;
    double c = b[(long)j * nx + i];
    if (P->wall_y && j == 0) return b[(long)1 * nx + i] - c;
    if (P->wall_y && j == ny - 1) return c - b[(long)(ny - 2) * nx + i];
    int jm = (j - 1 + ny) % ny, jp = (j + 1) % ny;
    return van_leer(c - b[(long)jm * nx + i], b[(long)jp * nx + i] - c);
}

/* R14 at the x-face between columns i and i+1 of row j (periodic x). */
static void recon_xface_upwind(const oracle_params *P, const double *B, int i, int j, double *out)
{
    int nx = P->nx, ny = P->ny;
    long N = (long)nx * ny;
    double h = 0.5 * P->cfl;
    int im = (i - 1 + nx) % nx, ip = (i + 1) % nx, ipp = (i + 2) % nx;
    for (int q = 0; q < Q; q++) {
        const double *b = B + q * N;
        double L = b[(long)j * nx + i], R = b[(long)j * nx + ip];
        double sxL = van_leer(L - b[(long)j * nx + im], R - L);
        double sxR = van_leer(R - L, b[(long)j * nx + ipp] - R);
        double syL = upwind_yslope(P, b, i, j);
        double syR = upwind_yslope(P, b, ip, j);
        /* x_f - xi h relative to the centre of L is (1/2 - h ex, -h ey), of R (-1/2 - h ex, -h ey) */
        double vL = L + sxL * (0.5 - h * EX[q]) + syL * (-h * EY[q]);
        double vR = R + sxR * (-0.5 - h * EX[q]) + syR * (-h * EY[q]);
        out[q] = EX[q] > 0 ? vL : (EX[q] < 0 ? vR : 0.5 * (vL + vR));
    }
}

/* R14 at the interior (or periodic) y-face between rows jm (below) and jc of
 * column i. */
static void recon_yface_upwind(const oracle_params *P, const double *B, int i, int jm, int jc, double *out)
{
    int nx = P->nx;
    long N = (long)nx * P->ny;
    double h = 0.5 * P->cfl;
    int im = (i - 1 + nx) % nx, ip = (i + 1) % nx;
    for (int q = 0; q < Q; q++) {
        const double *b = B + q * N;
        double D = b[(long)jm * nx + i], U = b[(long)jc * nx + i];
        double syD = upwind_yslope(P, b, i, jm);
        double syU = upwind_yslope(P, b, i, jc);
        double sxD = van_leer(D - b[(long)jm * nx + im], b[(long)jm * nx + ip] - D);
        double sxU = van_leer(U - b[(long)jc * nx + im], b[(long)jc * nx + ip] - U);
        /* x_f - xi h relative to the centre of D is (-h ex, 1/2 - h ey), of U (-h ex, -1/2 - h ey) */
        double vD = D + sxD * (-h * EX[q]) + syD * (0.5 - h * EY[q]);
        double vU = U + sxU * (-h * EX[q]) + syU * (-0.5 - h * EY[q]);
        out[q] = EY[q] > 0 ? vD : (EY[q] < 0 ? vU : 0.5 * (vD + vU));
    }
}

void oracle_face_bar(const oracle_params *P, const double *B, int i, int j, int xface, double *out)
{
    if (xface) {
        if (P->recon == 1) recon_xface_upwind(P, B, i, j, out);
        else recon_xface(P, B, i, j, out);
    } else {
        int jm = (j - 1 + P->ny) % P->ny;
        if (P->recon == 1) recon_yface_upwind(P, B, i, jm, j, out);
        else recon_yface(P, B, i, jm, j, out);
    }
}

/* R9 at a wall face of column i: bottom (y = 0, top == 0) or top (y = ny). */
static void recon_wall(const oracle_params *P, const double *B, int i, int top, double *out)
{
    int nx = P->nx, ny = P->ny;
    long N = (long)nx * ny;
    double h = 0.5 * P->cfl;
    int ip = (i + 1) % nx, im = (i - 1 + nx) % nx;
    int j0 = top ? ny - 1 : 0;         /* cell adjacent to the wall */
    int j1 = top ? ny - 2 : 1;         /* next cell into the fluid */
    double dyw = top ? 0.5 : -0.5;     /* wall position minus cell centre */
    for (int q = 0; q < Q; q++) {
        int leaves_fluid_or_tangent = top ? (EY[q] >= 0) : (EY[q] <= 0);
        if (!leaves_fluid_or_tangent) continue;
        const double *b = B + q * N;
        double b0 = b[(long)j0 * nx + i];
        double sx = 0.5 * (b[(long)j0 * nx + ip] - b[(long)j0 * nx + im]);
        double sy = top ? (b[(long)j0 * nx + i] - b[(long)j1 * nx + i])
                        : (b[(long)j1 * nx + i] - b[(long)j0 * nx + i]);
        out[q] = b0 + (-h * EX[q]) * sx + (dyw - h * EY[q]) * sy;
    }
    for (int q = 0; q < Q; q++) {
        int enters_fluid = top ? (EY[q] < 0) : (EY[q] > 0);
        if (enters_fluid) out[q] = out[opposite(q)];
    }
}

/* R17 at a wall face of column i with the upwind reconstruction: a direction
 * leaving the fluid or running along the wall takes the upwind profile of
 * the adjacent cell (its limited x-slope, its one-sided y-slope into the
 * fluid) at x_f - xi h; a direction entering the fluid takes the value of
 * its opposite direction (bounce-back). */
static void recon_wall_upwind(const oracle_params *P, const double *B, int i, int top, double *out)
{
    int nx = P->nx, ny = P->ny;
    long N = (long)nx * ny;
    double h = 0.5 * P->cfl;
    int ip = (i + 1) % nx, im = (i - 1 + nx) % nx;
    int j0 = top ? ny - 1 : 0;         /* cell adjacent to the wall */
    double dyw = top ? 0.5 : -0.5;     /* wall position minus cell centre */
    for (int q = 0; q < Q; q++) {
        int leaves_fluid_or_tangent = top ? (EY[q] >= 0) : (EY[q] <= 0);
        if (!leaves_fluid_or_tangent) continue;
        const double *b = B + q * N;
        double b0 = b[(long)j0 * nx + i];
        double sx = van_leer(b0 - b[(long)j0 * nx + im], b[(long)j0 * nx + ip] - b0);
        double sy = upwind_yslope(P, b, i, j0);
        out[q] = b0 + (-h * EX[q]) * sx + (dyw - h * EY[q]) * sy;
    }
    for (int q = 0; q < Q; q++) {
        int enters_fluid = top ? (EY[q] < 0) : (EY[q] > 0);
        if (enters_fluid) out[q] = out[opposite(q)];
    }
}

void oracle_wall_face_bar(const oracle_params *P, const double *B, int i, int top, double *out)
{
    if (P->recon == 1) recon_wall_upwind(P, B, i, top, out);
    else recon_wall(P, B, i, top, out);
}

static void one_step(oracle_ctx *c)
{
    const oracle_params *P = &c->P;
    int nx = P->nx, ny = P->ny, coupled = (P->model == 0);
    long N = (long)nx * ny;
    double dt = P->cfl;
    double tau_f = P->mobility / RT;    /* Eq. 34 */
    int nyf = P->wall_y ? ny + 1 : ny;  /* y-faces: index j = face below row j */

    point_state *cs = malloc(sizeof(point_state) * N);
    double *fbp = malloc(sizeof(double) * Q * N), *ftp = malloc(sizeof(double) * Q * N);
    double *gbp = calloc((size_t)Q * N, sizeof(double)), *gtp = calloc((size_t)Q * N, sizeof(double));
    double *fxf = malloc(sizeof(double) * Q * N), *gxf = calloc((size_t)Q * N, sizeof(double));
    double *fyf = malloc(sizeof(double) * Q * nx * nyf);
    double *gyf = calloc((size_t)Q * nx * nyf, sizeof(double));

    /* 1. cell macros at t_n (Eqs. 31-33, 3-10, 34-36) */
    cell_states(c, cs);

    /* 2. equilibria, sources and the pre-step distributions (Eqs. 15-19, 29-30) */
    for (long k = 0; k < N; k++) {
        const point_state *s = &cs[k];
        double tl[Q], eq[Q], src[Q], bp[Q], tp[Q];
        for (int i = 0; i < Q; i++) tl[i] = c->f[i * N + k];
        oracle_feq(s->phi, s->ux, s->uy, eq);
        oracle_sf(s->theta, s->nx, s->ny, s->Dx, s->Dy, src);
        oracle_prestep(tau_f, dt, tl, eq, src, bp, tp);
        for (int i = 0; i < Q; i++) { fbp[i * N + k] = bp[i]; ftp[i * N + k] = tp[i]; }
        if (coupled) {
            for (int i = 0; i < Q; i++) tl[i] = c->g[i * N + k];
            oracle_geq(s->p, s->rho, s->ux, s->uy, eq);
            oracle_sg(s->drhox, s->drhoy, s->Fx, s->Fy, s->ux, s->uy, src);
            oracle_prestep(s->tau_g, dt, tl, eq, src, bp, tp);
            for (int i = 0; i < Q; i++) { gbp[i * N + k] = bp[i]; gtp[i * N + k] = tp[i]; }
        }
    }

    /* 3. x-faces: face i+1/2 of row j stored at index (j, i) (Eqs. 27-28, R2, R3) */
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            long kl = (long)j * nx + i, kr = (long)j * nx + (i + 1) % nx;
            double fb[Q], gb[Q] = {0}, fp[Q], gp[Q] = {0};
            if (P->recon == 1) {
                recon_xface_upwind(P, fbp, i, j, fb);
                if (coupled) recon_xface_upwind(P, gbp, i, j, gb);
            } else {
                recon_xface(P, fbp, i, j, fb);
                if (coupled) recon_xface(P, gbp, i, j, gb);
            }
            double uf[2] = {0.0, 0.0};
            if (P->velocity_field == 4) sampled_face_velocity(c, 0, kl, kr, kl, uf);
            face_distributions(c, fb, gb,
                               0.5 * (cs[kl].dphix + cs[kr].dphix), 0.5 * (cs[kl].dphiy + cs[kr].dphiy),
                               0.5 * (cs[kl].lap + cs[kr].lap),
                               0.5 * (cs[kl].Dx + cs[kr].Dx), 0.5 * (cs[kl].Dy + cs[kr].Dy),
                               0, (double)((i + 1) % nx), (double)j + 0.5, uf, fp, gp);
            for (int q = 0; q < Q; q++) { fxf[q * N + kl] = fp[q]; gxf[q * N + kl] = gp[q]; }
        }

    /* 4. y-faces: face j is the one below row j (Eqs. 27-28, R2, R3, R9) */
    long NF = (long)nx * nyf;
    for (int j = 0; j < nyf; j++)
        for (int i = 0; i < nx; i++) {
            double fb[Q], gb[Q] = {0}, fp[Q], gp[Q] = {0};
            long kf = (long)j * nx + i;
            if (P->wall_y && (j == 0 || j == ny)) {
                int top = (j == ny);
                long k0 = (long)(top ? ny - 1 : 0) * nx + i;
                if (P->recon == 1) {
                    recon_wall_upwind(P, fbp, i, top, fb);
                    if (coupled) recon_wall_upwind(P, gbp, i, top, gb);
                } else {
                    recon_wall(P, fbp, i, top, fb);
                    if (coupled) recon_wall(P, gbp, i, top, gb);
                }
                face_distributions(c, fb, gb, cs[k0].dphix, 0.0, cs[k0].lap, cs[k0].Dx, 0.0,
                                   1, (double)i + 0.5, (double)j, NULL, fp, gp);
            } else {
                int jm = (j - 1 + ny) % ny, jc = j % ny;
                long kd = (long)jm * nx + i, ku = (long)jc * nx + i;
                if (P->recon == 1) {
                    recon_yface_upwind(P, fbp, i, jm, jc, fb);
                    if (coupled) recon_yface_upwind(P, gbp, i, jm, jc, gb);
                } else {
                    recon_yface(P, fbp, i, jm, jc, fb);
                    if (coupled) recon_yface(P, gbp, i, jm, jc, gb);
                }
                double uf[2] = {0.0, 0.0};
                if (P->velocity_field == 4) sampled_face_velocity(c, 1, kd, ku, kf, uf);
                face_distributions(c, fb, gb,
                                   0.5 * (cs[kd].dphix + cs[ku].dphix), 0.5 * (cs[kd].dphiy + cs[ku].dphiy),
                                   0.5 * (cs[kd].lap + cs[ku].lap),
                                   0.5 * (cs[kd].Dx + cs[ku].Dx), 0.5 * (cs[kd].Dy + cs[ku].Dy),
                                   0, (double)i + 0.5, (double)j, uf, fp, gp);
            }
            for (int q = 0; q < Q; q++) { fyf[q * NF + kf] = fp[q]; gyf[q * NF + kf] = gp[q]; }
        }

    /* 5. cell update psi~^{n+1} = psi~+ - dt/|V| J (Eqs. 22, 24; |V| = 1, |S| = 1) */
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            long k = (long)j * nx + i;
            long kw = (long)j * nx + (i - 1 + nx) % nx;     /* face i-1/2 */
            long ks = (long)j * nx + i;                     /* face below row j */
            long kn = (long)((P->wall_y ? j + 1 : (j + 1) % ny)) * nx + i;
            for (int q = 0; q < Q; q++) {
                double jf = EX[q] * (fxf[q * N + k] - fxf[q * N + kw])
                          + EY[q] * (fyf[q * NF + kn] - fyf[q * NF + ks]);
                c->f[q * N + k] = ftp[q * N + k] - dt * jf;
                if (coupled) {
                    double jg = EX[q] * (gxf[q * N + k] - gxf[q * N + kw])
                              + EY[q] * (gyf[q * NF + kn] - gyf[q * NF + ks]);
                    c->g[q * N + k] = gtp[q * N + k] - dt * jg;
                }
            }
        }

    /* 6. history for d_t(phi u) (R5) */
    for (long k = 0; k < N; k++) {
        c->phiu[k] = cs[k].phi * cs[k].ux;
        c->phiu[N + k] = cs[k].phi * cs[k].uy;
    }
    c->n++;

    free(cs); free(fbp); free(ftp); free(gbp); free(gtp);
    free(fxf); free(gxf); free(fyf); free(gyf);
}

static int params_valid(const oracle_params *P)
{
    if (P->nx < 3 || P->ny < 3) return 0;
    if (!(P->cfl > 0.0) || !(P->mobility > 0.0) || !(P->width > 0.0)) return 0;
    if (P->model != 0 && P->model != 1) return 0;
    if (P->velocity_field < 0 || P->velocity_field > 4) return 0;
    if (P->recon < 0 || P->recon > 1) return 0;
    if (P->model == 1 && P->velocity_field >= 1 && P->velocity_field <= 3 &&
        (!(P->vel_u0 > 0.0) || !(P->vel_length > 0.0))) return 0;
    if (P->model == 0) {
        if (!(P->rho_h > 0.0) || !(P->rho_l > 0.0)) return 0;
        if (!(P->mu_h > 0.0) || !(P->mu_l > 0.0)) return 0;
    }
    return 1;
}

oracle_ctx *oracle_create(const oracle_params *p, const double *phi0,
                          const double *ux0, const double *uy0, const double *p0)
{
    if (!p || !phi0 || !params_valid(p)) return NULL;
    oracle_ctx *c = calloc(1, sizeof *c);
    c->P = *p;
    int nx = p->nx, ny = p->ny;
    long N = (long)nx * ny;
    double dt = p->cfl;
    c->f = calloc((size_t)Q * N, sizeof(double));
    c->g = calloc((size_t)Q * N, sizeof(double));
    c->phiu = calloc((size_t)2 * N, sizeof(double));
    c->snap = calloc((size_t)3 * N, sizeof(double));
    if (p->model == 1 && p->velocity_field == 4) {
        /* the sampled field starts as the cell velocity given at creation */
        c->vel = calloc((size_t)4 * N, sizeof(double));
        for (long k = 0; k < N; k++) {
            c->vel[k] = ux0 ? ux0[k] : 0.0;
            c->vel[N + k] = uy0 ? uy0[k] : 0.0;
        }
    }

    double *gx = malloc(sizeof(double) * N), *gy = malloc(sizeof(double) * N);
    double *lp = malloc(sizeof(double) * N);
    oracle_grad_lap(nx, ny, p->wall_y, phi0, gx, gy, lp);
    for (long k = 0; k < N; k++) {
        point_state s;
        memset(&s, 0, sizeof s);
        s.phi = phi0[k];
        s.dphix = gx[k];
        s.dphiy = gy[k];
        s.lap = lp[k];
        closures(p, &s);
        if (p->model == 0) {
            s.ux = ux0 ? ux0[k] : 0.0;
            s.uy = uy0 ? uy0[k] : 0.0;
            s.p = p0 ? p0[k] : 0.0;
        } else if (p->velocity_field == 4) {
            s.ux = c->vel[k];
            s.uy = c->vel[N + k];
        } else {
            prescribed_velocity(p, (double)(k % nx) + 0.5, (double)(k / nx) + 0.5, 0.0, &s.ux, &s.uy);
        }
        double eq[Q], src[Q];
        oracle_feq(s.phi, s.ux, s.uy, eq);             /* R7 */
        oracle_sf(s.theta, s.nx, s.ny, 0.0, 0.0, src);
        for (int i = 0; i < Q; i++) c->f[i * N + k] = eq[i] - 0.5 * dt * src[i];
        if (p->model == 0) {
            oracle_geq(s.p, s.rho, s.ux, s.uy, eq);
            oracle_sg(s.drhox, s.drhoy, s.Fx, s.Fy, s.ux, s.uy, src);
            for (int i = 0; i < Q; i++) c->g[i * N + k] = eq[i] - 0.5 * dt * src[i];
        }
        c->phiu[k] = s.phi * s.ux;
        c->phiu[N + k] = s.phi * s.uy;
    }
    free(gx); free(gy); free(lp);
    c->n = 0;
    return c;
}

int oracle_set_velocity(oracle_ctx *c, const double *ux_cell, const double *uy_cell,
                        const double *ux_xface, const double *uy_yface)
{
    if (!c || !c->vel || !ux_cell || !uy_cell || (!ux_xface) != (!uy_yface)) return 0;
    long N = (long)c->P.nx * c->P.ny;
    for (long k = 0; k < N; k++) {
        c->vel[k] = ux_cell[k];
        c->vel[N + k] = uy_cell[k];
        c->vel[2 * N + k] = ux_xface ? ux_xface[k] : 0.0;
        c->vel[3 * N + k] = uy_yface ? uy_yface[k] : 0.0;
    }
    c->vel_faces = ux_xface != NULL;
    return 1;
}

void oracle_destroy(oracle_ctx *c)
{
    if (!c) return;
    free(c->f); free(c->g); free(c->phiu); free(c->snap); free(c->vel);
    free(c);
}

void oracle_step(oracle_ctx *c, long nsteps)
{
    for (long s = 0; s < nsteps; s++) one_step(c);
}

long oracle_step_count(const oracle_ctx *c) { return c->n; }

void oracle_macros(oracle_ctx *c, double *phi, double *p, double *ux, double *uy)
{
    long N = (long)c->P.nx * c->P.ny;
    point_state *cs = malloc(sizeof(point_state) * N);
    cell_states(c, cs);
    for (long k = 0; k < N; k++) {
        if (phi) phi[k] = cs[k].phi;
        if (p) p[k] = cs[k].p;
        if (ux) ux[k] = cs[k].ux;
        if (uy) uy[k] = cs[k].uy;
    }
    free(cs);
}

void oracle_get_state(const oracle_ctx *c, double *f, double *g, double *phiu_prev)
{
    long N = (long)c->P.nx * c->P.ny;
    if (f) memcpy(f, c->f, sizeof(double) * Q * N);
    if (g) memcpy(g, c->g, sizeof(double) * Q * N);
    if (phiu_prev) memcpy(phiu_prev, c->phiu, sizeof(double) * 2 * N);
}

void oracle_set_state(oracle_ctx *c, const double *f, const double *g,
                      const double *phiu_prev, long step_count)
{
    long N = (long)c->P.nx * c->P.ny;
    if (f) memcpy(c->f, f, sizeof(double) * Q * N);
    if (g) memcpy(c->g, g, sizeof(double) * Q * N);
    if (phiu_prev) memcpy(c->phiu, phiu_prev, sizeof(double) * 2 * N);
    c->n = step_count;
}

/* Mass, Eq. 44 residuals of phi and u against the previous call, max |u|. */
void oracle_reduce(oracle_ctx *c, double *mass, double *resid_phi,
                   double *resid_u, double *umax)
{
    long N = (long)c->P.nx * c->P.ny;
    double *phi = malloc(sizeof(double) * N), *ux = malloc(sizeof(double) * N);
    double *uy = malloc(sizeof(double) * N);
    oracle_macros(c, phi, NULL, ux, uy);
    double m = 0.0, dphi = 0.0, nphi = 0.0, du = 0.0, nu = 0.0, um = 0.0;
    for (long k = 0; k < N; k++) {
        m += phi[k];
        double u2 = ux[k] * ux[k] + uy[k] * uy[k];
        if (sqrt(u2) > um) um = sqrt(u2);
        nphi += phi[k] * phi[k];
        nu += u2;
        if (c->have_snap) {
            double a = phi[k] - c->snap[k];
            double bx = ux[k] - c->snap[N + k], by = uy[k] - c->snap[2 * N + k];
            dphi += a * a;
            du += bx * bx + by * by;
        }
    }
    if (mass) *mass = m;
    if (umax) *umax = um;
    if (resid_phi) *resid_phi = c->have_snap ? (nphi > 0.0 ? dphi / nphi : 0.0) : 1.0;
    if (resid_u) *resid_u = c->have_snap ? (nu > 0.0 ? du / nu : 0.0) : 1.0;
    memcpy(c->snap, phi, sizeof(double) * N);
    memcpy(c->snap + N, ux, sizeof(double) * N);
    memcpy(c->snap + 2 * N, uy, sizeof(double) * N);
    c->have_snap = 1;
    free(phi); free(ux); free(uy);
}
