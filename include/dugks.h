/*
 * dugks.h -- C ABI of the GB300 (sm_103a) phase-field DUGKS library.
 *
 * The library advances the two coupled D2Q9 kinetic models of Yang, Zhong &
 * Zhuo, "A phase-field model for large-density-ratio two-phase flows based on
 * discrete unified gas-kinetic scheme" (arXiv:1810.07802), Sec. II.B: the
 * conservative Allen-Cahn model for the order parameter phi (Eqs. 12, 15, 16)
 * and the incompressible hydrodynamic model for p and u (Eqs. 13, 17-19), by
 * the DUGKS finite-volume step (Eqs. 20-30) with the closures of Eqs. 3-10
 * and 31-37.  Every step runs in CUDA kernels on the device; there is no CPU
 * fallback.
 *
 * Conventions shared by every call
 *  - Grid: nx * ny square cells of unit size (delta_x = 1, Sec. III); cell
 *    (i, j) has its centre at (i + 1/2, j + 1/2).  Host fields are row-major
 *    [ny][nx] arrays of double, x fastest, no padding.
 *  - Lattice: D2Q9 with RT = 1/3, so xi_i = e_i and dt = CFL (Eq. 37).
 *  - Streams: every call enqueues work on the stream given to dugks_create
 *    (a cudaStream_t passed as void*; NULL = the legacy default stream).
 *    Calls marked "synchronises" wait for that stream before returning.
 *  - Errors: every call returns a dugks_status.  Invalid arguments return
 *    DUGKS_ERR_ARG and change nothing.  The step kernels record non-finite
 *    values (DUGKS_ERR_NONFINITE) and rho <= 0 or mu <= 0
 *    (DUGKS_ERR_NONPHYSICAL) in a device status word; asynchronous calls
 *    cannot see it, and the next synchronising call returns it.  The status
 *    is sticky until dugks_destroy.
 *  - Ownership: the library owns the handle and any device memory it
 *    allocates.  A caller-supplied workspace stays the caller's and must
 *    outlive the handle.  Host arrays are only read or written during the call.
 *  - Thread safety: one handle must not be used from two host threads at once;
 *    distinct handles are independent (their parameters are passed to the
 *    kernels by value; no global device state).
 */
#ifndef DUGKS_H
#define DUGKS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DUGKS_OK = 0,
    DUGKS_ERR_ARG = -1,          /* invalid parameter or argument              */
    DUGKS_ERR_OOM = -2,          /* device allocation failed / workspace small */
    DUGKS_ERR_CUDA = -3,         /* a CUDA runtime call failed                 */
    DUGKS_ERR_NONFINITE = -4,    /* a step produced NaN or Inf                 */
    DUGKS_ERR_NONPHYSICAL = -5,  /* a step met rho <= 0 or mu <= 0             */
    DUGKS_ERR_TIMEOUT = -6,      /* a bounded device wait ran out: in a step,
                                    the wait for a tile's TMA copy.  A CTA
                                    that gives up leaves its tile of the
                                    step's output unwritten, so the state
                                    after that step is undefined (stale cells);
                                    restore a checkpoint (dugks_set_state)
                                    before stepping on.  Later CTAs of the
                                    same and following steps stage with plain
                                    loads, and the flag stays set           */
    DUGKS_ERR_UNSUPPORTED = -7,  /* valid request this build does not provide  */
    DUGKS_ERR_BOUNDS = -8        /* a bounds-checked build (DUGKS_BOUNDS_CHECK)
                                    met an out-of-range index; the access was
                                    skipped                                    */
} dugks_status;

typedef enum { DUGKS_BC_PERIODIC = 0, DUGKS_BC_WALL = 1 } dugks_bc;
typedef enum { DUGKS_FP64 = 0, DUGKS_FP32_SHIFTED = 1 } dugks_precision;
typedef enum { DUGKS_COUPLED = 0, DUGKS_AC_PRESCRIBED_U = 1 } dugks_model;
typedef enum { DUGKS_VISC_RECIPROCAL = 0, DUGKS_VISC_LINEAR = 1 } dugks_visc;
/* Reconstruction of psi-bar-plus at x_f - xi h (Eq. 27).  Central: linear
 * profile through the face (Sec. II.B's choice).  Upwind: each cell of the
 * face carries a linear profile with van Leer-limited slopes, and a direction
 * takes the profile of the cell it leaves (the mean of both when it runs
 * along the face); the scheme Sec. II.B names as the alternative and Sec.
 * III.A as the remedy for the error growth at high Peclet number. */
typedef enum { DUGKS_RECON_CENTRAL = 0, DUGKS_RECON_UPWIND = 1 } dugks_recon;

/*
 * Problem statement (Sec. II.A-B).  phi_H = 1 is the heavy phase, phi_L = 0
 * the light one (Eq. 7).
 */
typedef struct {
    int32_t nx, ny;        /* cells, each >= 3                                     */
    int32_t lattice;       /* must be 9 (D2Q9, Eq. 14)                             */
    int32_t model;         /* dugks_model: coupled (default) or Allen-Cahn only
                              with the uniform velocity (u0x, u0y) (Sec. III)      */
    int32_t precision;     /* dugks_precision: FP64 arithmetic and storage, or
                              FP32 arithmetic with distributions stored in FP32
                              as deviations from the rest state (phi_ref, p_ref) */
    int32_t bc_x;          /* must be DUGKS_BC_PERIODIC                            */
    int32_t bc_y;          /* periodic, or no-slip walls on y = 0 and y = ny       */
    int32_t visc_interp;   /* dugks_visc: 1/mu linear in phi (Eq. 35) or mu (Eq. 36) */
    int32_t gravity_mode;  /* 0: G = (gx, gy); 1: G = (rho - rho_ref)(gx, gy)      */
    int32_t tile_shape;    /* step-kernel tile: 0 the library default, k >= 1 the
                              k-th compiled shape of the precision (see
                              dugks_tile_shapes, dugks_autotune).  Every shape
                              computes the same scheme                             */
    double cfl;            /* dt = cfl (Eq. 37 with delta_x = 1, RT = 1/3), > 0    */
    double mobility;       /* M_phi > 0; tau_f = M_phi / RT (Eq. 34)               */
    double width;          /* interface width W > 0 (Eq. 3)                        */
    double rho_h, rho_l;   /* phase densities > 0 (Eq. 10); coupled model only     */
    double mu_h, mu_l;     /* dynamic viscosities > 0 (Eqs. 35-36); coupled only   */
    double sigma;          /* surface tension >= 0 (Eq. 3)                         */
    double gx, gy;         /* body force (see gravity_mode), coupled model only    */
    double rho_ref;        /* reference density for gravity_mode 1                 */
    double phi_ref, p_ref; /* rest state subtracted before FP32 storage            */
    double u0x, u0y;       /* uniform velocity of the Allen-Cahn-only model (Eq. 40) */
    int32_t velocity_field; /* Allen-Cahn-only model: 0 uniform (u0x, u0y); 1 rotation
                              about the box centre (Eq. 41); 2 shear reversed at
                              t = L0/U0 (Eq. 42); 3 smoothed deformation with period
                              L0/U0 (Eq. 43).  Evaluated at cell centres at t_n and
                              at faces at t_n + dt/2.  4: sampled arrays, steady
                              between dugks_set_velocity_field calls (initially the
                              ux0, uy0 given to dugks_create)                      */
    int32_t reserved2;     /* must be 0                                            */
    double vel_u0;         /* U0 > 0 of velocity fields 1-3                        */
    double vel_length;     /* L0 > 0 of velocity fields 1-3                        */
    int32_t recon;         /* dugks_recon: reconstruction of psi-bar-plus at
                              x_f - xi h (Eq. 27): central (default, Sec. II.B) or
                              upwind with van Leer-limited slopes (the default
                              tile shape only; with walls a cell next to a wall
                              takes its one-sided y-difference into the fluid and
                              the wall face bounces back entering directions)     */
    int32_t reserved3;     /* must be 0                                            */
} dugks_params;

typedef struct dugks_ctx *dugks_handle;

/* Device bytes the solver needs for these parameters (state, ping-pong
 * buffers, macro staging, reduction scratch), or 0 if the parameters are
 * invalid.  Used for admission by HBM footprint. */
size_t dugks_workspace_bytes(const dugks_params *params);

/* Sampled velocity field of the Allen-Cahn-only model (velocity_field 4),
 * used from the next step on.  ux_cell, uy_cell: [ny][nx] host doubles at
 * the cell centres (required).  ux_xface: the x-component at x-face i+1/2 of
 * row j ([j][i], the face between columns i and i+1, periodic) and uy_yface:
 * the y-component at the y-face below row j ([j][i]); both or neither.  A
 * face without its array takes the mean of the two cells; the tangential
 * component is always the mean of the two cells; wall faces keep u = 0.
 * Stored in the solver's workspace in the storage precision; synchronises the
 * solver's stream.  DUGKS_ERR_UNSUPPORTED if the solver has no sampled field,
 * DUGKS_ERR_ARG for missing arrays. */
dugks_status dugks_set_velocity_field(dugks_handle h, const double *ux_cell, const double *uy_cell,
                                      const double *ux_xface, const double *uy_yface);

/* Self-check of the bounded device waits (failure detection without a
 * fault): launches one CTA that waits, with the step kernel's wait function,
 * on a shared-memory barrier that no copy ever completes, giving up after
 * max_polls polls (<= 0: the step kernel's own limit, well under a second).
 * Returns DUGKS_ERR_TIMEOUT when the wait ran out as designed (the CUDA
 * context stays usable), DUGKS_OK if it unexpectedly completed, or a CUDA
 * error.  Synchronises cuda_stream; allocates and frees 4 device bytes. */
dugks_status dugks_check_bounded_wait(int64_t max_polls, void *cuda_stream);

/* Self-check of the persistent batched launch's wait for a member's previous
 * step (failure detection without a fault): launches one CTA that waits, with
 * that kernel's wait function, on a step counter that nothing raises, giving
 * up after budget_ns nanoseconds of sleeps (<= 0: the kernel's own budget,
 * about 2 s).  Returns DUGKS_ERR_TIMEOUT when the wait ran out as designed
 * (the CUDA context stays usable), DUGKS_OK if it unexpectedly completed, or
 * a CUDA error.  Synchronises cuda_stream; allocates and frees 8 device
 * bytes. */
dugks_status dugks_check_batch_wait(int64_t budget_ns, void *cuda_stream);

/* Tile shapes the step kernels are compiled for, for one precision: writes
 * up to `cap` (tx, ty) cell counts (tx may be NULL, likewise ty) and returns
 * how many there are (tile_shape k >= 1 selects entry k - 1), or -1 for an
 * unknown precision.  Shape 1 is the library default.  No device work. */
int32_t dugks_tile_shapes(int32_t precision, int32_t *tx, int32_t *ty, int32_t cap);

/* Autotuner of the step kernel's tile shape for one problem.  For every
 * compiled shape it creates the problem (params, with tile_shape replaced,
 * and the host fields as for dugks_create) in a library-allocated workspace,
 * runs 2 warm-up steps, times trial_steps (>= 1) steps with CUDA events on
 * cuda_stream and destroys it; one shape at a time, so the device memory
 * needed is one workspace.  Writes the fastest tile_shape value (>= 1) to
 * *best and, if ms_per_step is not NULL, the milliseconds per step of shape
 * k to ms_per_step[k - 1] (-1 where a shape failed; as many entries as
 * dugks_tile_shapes returns).  Synchronises.  Returns DUGKS_OK if at least
 * one shape ran, else the first failure. */
dugks_status dugks_autotune(const dugks_params *params, const double *phi0, const double *ux0, const double *uy0,
                            const double *p0, int32_t trial_steps, void *cuda_stream, int32_t *best,
                            double *ms_per_step);

/* Creates a solver and builds the initial state psi~0 = psi_eq - dt/2 S with
 * d_t(phi u) = 0 (Eq. 23a with psi = psi_eq) from host fields phi0, ux0, uy0,
 * p0 ([ny][nx] doubles; ux0, uy0, p0 may be NULL for zero; ignored in the
 * Allen-Cahn-only model, which uses (u0x, u0y)).
 * device_workspace: NULL to let the library cudaMalloc its workspace, or a
 * caller-owned device buffer of at least dugks_workspace_bytes(params) bytes,
 * 256-byte aligned.  cuda_stream: cudaStream_t or NULL.  Synchronises. */
dugks_status dugks_create(const dugks_params *params, const double *phi0,
                          const double *ux0, const double *uy0, const double *p0,
                          void *device_workspace, size_t ws_bytes,
                          void *cuda_stream, dugks_handle *out);

/* Enqueues nsteps >= 0 DUGKS time steps (Eqs. 20-30; one fused kernel launch
 * per step).  Asynchronous. */
dugks_status dugks_step(dugks_handle h, int64_t nsteps);

/* Cell-centre macros of the current state (Eqs. 31-33): phi, p, ux, uy as
 * [ny][nx] doubles; any pointer may be NULL.  dst_is_device != 0: pointers
 * are device memory written on the solver's stream (asynchronous);
 * otherwise host memory, and the call synchronises. */
dugks_status dugks_macros(dugks_handle h, double *phi, double *p, double *ux, double *uy,
                          int32_t dst_is_device);

/* FP64 reductions on the device: total phi (phi mass), the steady-state
 * residuals of Eq. 44 for phi and |u| against the fields at the previous
 * dugks_reduce call (1.0 on the first call), and max |u|.  Any pointer may
 * be NULL.  Synchronises. */
dugks_status dugks_reduce(dugks_handle h, double *phi_mass, double *resid_phi,
                          double *resid_u, double *umax);

/* The sums behind dugks_reduce over the rows [row0, row0 + nrows) only, for
 * combining several y-bands of one problem (sum the first five over bands,
 * take the maximum of the last, then form the Eq. 44 ratios sums[2]/sums[1]
 * and sums[4]/sums[3]): sums[0] = sum phi, sums[1] = sum phi^2, sums[2] =
 * sum (phi - phi_prev)^2, sums[3] = sum |u|^2, sums[4] = sum |u - u_prev|^2,
 * sums[5] = max |u|, in FP64 on the device, the previous fields being those
 * of the last dugks_reduce / dugks_reduce_rows call on the handle
 * (*had_snapshot = 0 and sums[2] = sums[4] = 0 on the first call;
 * had_snapshot may be NULL).  Like dugks_reduce it then keeps the whole
 * grid's fields as the next call's previous fields.  DUGKS_ERR_ARG for rows
 * outside the grid or a NULL sums; a failed step is reported as by
 * dugks_reduce, with the sums written.  Synchronises. */
dugks_status dugks_reduce_rows(dugks_handle h, int32_t row0, int32_t nrows, double *sums,
                               int32_t *had_snapshot);

/* The distributions as absolute FP64 values, in the oracle-comparable layout:
 * f [9][ny][nx], g [9][ny][nx] (zero for the Allen-Cahn-only model) and the
 * stored (phi u)^{n-1} [2][ny][nx], on the host; any pointer may be NULL.
 * Synchronises. */
dugks_status dugks_get_distributions(dugks_handle h, double *f, double *g, double *phiu_prev);

/* Rows of the state for domain decomposition into y-slabs (no counterpart
 * in the paper's single-domain runs; the halo a band needs follows from the
 * stencils of Eqs. 27 and 31-33 and the gradient and Laplacian of Sec. II.B:
 * two rows of f, one of g and one of (phi u)^{n-1} on each side).
 * dugks_get_rows copies rows [row0, row0 + nrows) (0 <= row0, row0 + nrows <=
 * ny) of the current state -- the distribution planes (9 for the
 * Allen-Cahn-only model, 18 coupled) followed by the 2 history planes,
 * exactly as stored (FP32 deviations from the rest state, or FP64), in
 * elements of dugks_state_element_bytes bytes -- into buf laid out
 * [planes][nrows][nx]; dugks_set_rows copies such a buffer back into those
 * rows.  buf is device memory (buf_is_device != 0: one kernel on the
 * solver's stream, no synchronisation) or host memory (synchronises).  Rows
 * written this way replace the state the next step reads; a band stepped
 * with its halo rows refreshed from its neighbours before every step gives
 * its own rows the bits of the single-domain step.  DUGKS_ERR_ARG for rows
 * outside the grid. */
size_t dugks_state_element_bytes(dugks_handle h);
dugks_status dugks_get_rows(dugks_handle h, int32_t row0, int32_t nrows, void *buf, int32_t buf_is_device);
dugks_status dugks_set_rows(dugks_handle h, int32_t row0, int32_t nrows, const void *buf, int32_t buf_is_device);

/* Checkpoint: size of, and copy of, the complete solver state (header,
 * stored distributions and history exactly as held on the device).
 * Restoring a checkpoint into a handle created with the same parameters
 * continues bit-identically.  Both synchronise. */
size_t dugks_state_bytes(dugks_handle h);
dugks_status dugks_get_state(dugks_handle h, void *host_buf, size_t bytes);
dugks_status dugks_set_state(dugks_handle h, const void *host_buf, size_t bytes);

/* Number of steps taken since creation (or since the restored checkpoint's). */
int64_t dugks_step_count(dugks_handle h);

/* Waits for the solver's stream and returns the device status word. */
dugks_status dugks_sync(dugks_handle h);

/* Frees the handle and the memory the library allocated.  Synchronises. */
dugks_status dugks_destroy(dugks_handle h);

/* ---- Batches: several independent problems advanced together ----
 * A batch advances every member by the same number of DUGKS steps.  Members
 * are grouped by kernel variant (precision x model x y-boundary x tile shape
 * x reconstruction).  By default each group and step is one grid launch over
 * the group's (problem, tile) items.  In the persistent mode
 * (dugks_batch_set_persistent(b, 1)) a group advances up to 16 steps in one
 * launch: CTAs (at most one step's items, at most as many as fit on the GPU)
 * take (step, problem, tile) items from one queue in step order, and a tile
 * of step s + 1 of a member waits only for that member's tiles of step s, so
 * members of uneven size advance without a batch-wide barrier between steps.
 * Either way the launches are captured once into CUDA graphs (16 steps, and
 * one step) and replayed until the membership changes.  The two modes run
 * separately compiled kernels and agree to round-off.  Each CTA runs the same tile code as
 * dugks_step, with the member's constants read from a device descriptor
 * instead of the kernel's parameter space, so the two agree to round-off.  A
 * member of 2048 tiles or more fills the GPU by itself: it is stepped by
 * dugks_step's kernel on the batch's stream and is bit-identical to stepping
 * it alone.  Which path a member takes depends on its own size only, so its
 * result does not depend on the rest of the batch.
 * Members may differ in size, physics and precision.  While a handle is in a
 * batch, advance it only through the batch; its other calls (dugks_macros,
 * dugks_reduce, ...) stay valid but run on the handle's own stream, so use
 * the batch's stream for the handle or call dugks_batch_sync first.  The
 * batch does not own its members: remove or keep them, then destroy them
 * with dugks_destroy. */
typedef struct dugks_batch_ctx *dugks_batch;

/* New empty batch enqueuing on cuda_stream (cudaStream_t or NULL). */
dugks_status dugks_batch_create(void *cuda_stream, dugks_batch *out);
/* Adds / removes a member (DUGKS_ERR_ARG if already in / not in the batch). */
dugks_status dugks_batch_add(dugks_batch b, dugks_handle h);
dugks_status dugks_batch_remove(dugks_batch b, dugks_handle h);
/* Number of members, or -1 for a NULL batch. */
int32_t dugks_batch_size(dugks_batch b);
/* Enqueues nsteps >= 0 steps of every member (asynchronous).  The first call
 * after a membership change uploads the work lists and captures the graph. */
dugks_status dugks_batch_step(dugks_batch b, int64_t nsteps);
/* Selects the persistent launch (on != 0) or one grid launch per step (on ==
 * 0, the default) for later dugks_batch_step calls; drops the captured graphs.
 * A persistent wait that runs out (a fault elsewhere; it does not happen in a
 * correct run) sets the member's status to DUGKS_ERR_TIMEOUT, reported by
 * dugks_batch_sync, and leaves that member's state undefined.  Returns
 * DUGKS_ERR_ARG for a NULL batch. */
dugks_status dugks_batch_set_persistent(dugks_batch b, int32_t on);
/* Waits for the batch's stream; returns the first member's error status. */
dugks_status dugks_batch_sync(dugks_batch b);
/* Frees the batch (not its members).  Synchronises. */
dugks_status dugks_batch_destroy(dugks_batch b);

/* Allocation-free FP64 reduction of macro fields (the paper has no
 * counterpart; this is a convenience for callers that cannot allocate).
 * Some callers cannot call cudaMalloc/cudaFree where they need a convergence
 * check: code being recorded into a CUDA graph (allocation is illegal while a
 * stream is captured), serving loops that plan all device memory up front,
 * or hosts without an allocator of their own.  This call takes device arrays
 * phi, ux, uy of n doubles (for example dugks_macros output with
 * dst_is_device = 1) and, optionally, snap = [3][n] doubles (phi, ux, uy of an
 * earlier time; NULL if none), and writes four doubles to the device array
 * out: the phi mass sum(phi); the relative residuals
 * sum((phi - snap_phi)^2) / sum(phi^2) and sum(|u - snap_u|^2) / sum(|u|^2)
 * (the same quantities dugks_reduce returns; 1.0 when snap is NULL); and
 * max |u|.  It is enqueued on cuda_stream (cudaStream_t or NULL) and does not
 * synchronise.
 * It allocates nothing: its per-block partial sums live in a fixed device
 * array inside this library (192 KiB, present on every GPU that loads the
 * library until the process exits), which bounds n to
 * DUGKS_STATIC_REDUCE_MAX_CELLS; larger n, n < 1 or a NULL phi/ux/uy/out
 * return DUGKS_ERR_ARG without launching anything.  The first call on each
 * device looks up that array's device address (cudaGetSymbolAddress) with
 * the device current, and so does the first call in a new context on it
 * (after cudaDeviceReset, say); a lookup that fails returns DUGKS_ERR_CUDA
 * and is tried again on the next call.  Make that first call before any
 * stream capture.  Every call shares the array: calls that can overlap on
 * the GPU (other streams or host threads) race and must be serialised by the
 * caller. */
#define DUGKS_STATIC_REDUCE_MAX_CELLS 16777216
dugks_status dugks_reduce_fields_static(const double *phi, const double *ux, const double *uy,
                                        const double *snap, int64_t n, double *out, void *cuda_stream);

/* Static description of a status code. */
const char *dugks_status_string(dugks_status s);

#ifdef __cplusplus
}
#endif
#endif
