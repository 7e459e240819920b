/*
 * dugks_oracle.h -- plain, slow FP64 CPU oracle for the phase-field DUGKS step.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the bench's
 * CPU-baseline leg may load this library. The product path (the CUDA library
 * under paper_1810_07802_gb300/) never calls it and shares no code with it.
 *
 * What it computes: Yang, Zhong & Zhuo, "A phase-field model for
 * large-density-ratio two-phase flows based on discrete unified gas-kinetic
 * scheme" (arXiv:1810.07802), Sec. II: two D2Q9 kinetic models, one for the
 * conservative Allen-Cahn order parameter phi (Eqs. 5-6, 12, 15-16) and one for
 * the incompressible hydrodynamics p, u (Eqs. 8-10, 13, 17-19), advanced by
 * the DUGKS finite-volume scheme (Eqs. 20-30) with the macroscopic closures of
 * Eqs. 31-37.  Every reading of a passage the paper leaves open is listed at
 * the top of dugks_oracle.c.
 *
 * Layout of every field: row-major [ny][nx], x fastest, no padding.
 * Distributions: [9][ny][nx] per model, direction index first.
 */
#ifndef DUGKS_ORACLE_H
#define DUGKS_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int nx, ny;          /* cells; delta_x = 1 (Sec. III)                      */
    int model;           /* 0: coupled A-C + hydrodynamics;
                            1: A-C only with a prescribed uniform velocity     */
    int wall_y;          /* 0: periodic in y; 1: no-slip walls at y=0, y=ny    */
    int visc;            /* 0: reciprocal interpolation (Eq. 35); 1: linear (Eq. 36) */
    int gravity_mode;    /* 0: G = (gx, gy); 1: G = (rho - rho_ref)(gx, gy)     */
    double cfl;          /* dt = CFL * dx / sqrt(3RT) (Eq. 37)                  */
    double mobility;     /* M_phi; tau_f = M_phi / RT (Eq. 34)                 */
    double width;        /* interface width W (Eq. 3)                          */
    double rho_h, rho_l; /* Eq. 10                                             */
    double mu_h, mu_l;   /* dynamic viscosities of the phi=1 / phi=0 phases    */
    double sigma;        /* surface tension (Eq. 3)                            */
    double gx, gy;       /* body force, see gravity_mode                      */
    double rho_ref;
    double u0x, u0y;     /* prescribed velocity for model 1, velocity_field 0  */
    int velocity_field;  /* model 1: 0 uniform (u0x, u0y) (Eq. 40); 1 rotation (Eq. 41);
                            2 reversing shear (Eq. 42); 3 smoothed deformation (Eq. 43);
                            4 sampled arrays (R15; see oracle_set_velocity) */
    int reserved;
    double vel_u0;       /* U0 of fields 1-3                                   */
    double vel_length;   /* L0 of fields 1-3                                   */
    int recon;           /* 0 central (R2), 1 upwind with van Leer slopes (R14; walls: R17) */
    int reserved2;
} oracle_params;

typedef struct oracle_ctx oracle_ctx;

/* Builds the initial state psi~0 = psi_eq - dt/2 S (D = 0) from host fields.
 * ux0, uy0, p0 may be NULL (zero).  Returns NULL on invalid parameters. */
oracle_ctx *oracle_create(const oracle_params *p, const double *phi0,
                          const double *ux0, const double *uy0, const double *p0);
void oracle_destroy(oracle_ctx *c);
/* velocity_field 4: replaces the sampled velocity (R15) for the next steps:
 * [ny][nx] cell arrays (required) and optional face arrays (both or neither).
 * Returns 0 if the run has no sampled field or the arguments are invalid. */
int oracle_set_velocity(oracle_ctx *c, const double *ux_cell, const double *uy_cell,
                        const double *ux_xface, const double *uy_yface);
void oracle_step(oracle_ctx *c, long nsteps);
long oracle_step_count(const oracle_ctx *c);
/* Cell-centre macros (Eqs. 31-33) of the current state; any pointer may be NULL. */
void oracle_macros(oracle_ctx *c, double *phi, double *p, double *ux, double *uy);
/* Raw state: f~ [9][ny][nx], g~ [9][ny][nx] (zero in model 1), (phi u)^{n-1} [2][ny][nx]. */
void oracle_get_state(const oracle_ctx *c, double *f, double *g, double *phiu_prev);
void oracle_set_state(oracle_ctx *c, const double *f, const double *g,
                      const double *phiu_prev, long step_count);
/* Domain sums: phi mass; relative residuals of phi and |u| against
 * the snapshot taken at the previous call (Eq. 44; 1.0 on the first call); max |u|. */
void oracle_reduce(oracle_ctx *c, double *mass, double *resid_phi,
                   double *resid_u, double *umax);

/* ---- the pieces of one step, exposed so the tests can pin each one ---- */
void oracle_lattice(int *ex, int *ey, double *w);          /* Eq. 14           */
void oracle_feq(double phi, double ux, double uy, double *feq);           /* Eq. 15 */
void oracle_sf(double theta, double nx, double ny, double Dx, double Dy,
               double *sf);                                               /* Eq. 16 */
void oracle_geq(double p, double rho, double ux, double uy, double *geq); /* Eqs. 17-18 */
void oracle_sg(double drhox, double drhoy, double Fx, double Fy,
               double ux, double uy, double *sg);                         /* Eq. 19 */
/* Eqs. 29-30: psi-bar-plus and psi-tilde-plus from psi-tilde at a cell centre. */
void oracle_prestep(double tau, double dt, const double *tilde, const double *eq,
                    const double *src, double *bar_plus, double *tilde_plus);
/* Eq. 28: original distribution at a face from psi-bar. */
void oracle_face_psi(double tau, double h, const double *bar, const double *eq,
                     const double *src, double *psi);
/* Stencils of Sec. II.B: six-point isotropic gradient and nine-point
 * Laplacian of phi, with periodic x and periodic-or-mirrored y. */
void oracle_grad_lap(int nx, int ny, int wall_y, const double *phi,
                     double *dphix, double *dphiy, double *lap);

/* Face value psi_bar(x_f, t + h) of every direction reconstructed from the
 * grid B ([Q][ny][nx], psi-bar-plus) by the scheme params->recon selects, at
 * the interior or periodic x-face i+1/2 of row j (xface != 0) or the y-face
 * below row j of column i (xface == 0). */
void oracle_face_bar(const oracle_params *params, const double *B, int i, int j, int xface, double *out);
/* Face value psi_bar(x_f, t + h) of every direction at the wall face of
 * column i (walled grids): the bottom wall y = 0 (top == 0) or the top wall
 * y = ny, by R9 (central) or R17 (upwind). */
void oracle_wall_face_bar(const oracle_params *params, const double *B, int i, int top, double *out);

#ifdef __cplusplus
}
#endif
#endif
