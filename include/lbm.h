/*
 * lbm.h - C ABI of a GB300 (sm_103a) library for the streaming-collision
 * lattice Boltzmann scheme of Meng & Zhang, "Kinetic diffuse boundary
 * condition for high-order lattice Boltzmann model with streaming-collision
 * mechanism" (arXiv:1209.5201).
 *
 * What the library computes (one time step, every fluid cell x, velocity a):
 *   pull   f_in(x, a) = f~*(x - e_a, a)                      Eq. (5), left side
 *          or, where x - e_a lies beyond a wall, the diffuse re-emission
 *          M_in * g_a^eq(u_w, T_w) / sum_l sum_out g^eq(u_w, T_w)     Eq. (12)
 *   moments rho, u, T of f_in                                  Eq. (3)
 *   relax   f~* = f_in - dt/(tau + dt/2) (f_in - rho g^eq(u, T))  Eq. (4)-(5)
 * The stored state is the post-collision transformed distribution f~*.
 *
 * Conventions shared by every call:
 *  - Units are the paper's non-dimensional ones (Sec. II, Eq. (2)): speeds in
 *    sqrt(R T0), lengths in the channel height (= 1), time in L/sqrt(R T0).
 *  - Lattice velocities are c_a = r e_a with integer e_a, |e_a,y| <= 3; one
 *    step dt = 1/(r Ny) moves a population by e_a cells (Sec. II, after Eq. (5)).
 *  - Grid: Nx periodic columns x, Ny fluid rows j at y = (j + 1/2)/Ny; the
 *    walls sit half a cell outside rows 0 and Ny-1 (Sec. III).  The bottom
 *    wall (y = 0) moves with u_wall[0], the top one (y = 1) with u_wall[1],
 *    both tangentially (along x).
 *  - Host arrays of per-cell fields are row-major [Ny][Nx] FP64.  Host arrays
 *    of distributions are [Q][Ny][Nx] FP64 in the library's velocity order
 *    (query it with lbm_lattice_tables).
 *  - Every call returns an int status (LBM_OK = 0).  No C++ exception crosses
 *    the ABI.  On failure the thread-local message of lbm_last_error says why.
 *  - Handles are opaque and not thread-safe: one host thread at a time per
 *    handle.  Device work is enqueued on the caller's CUDA stream, given as a
 *    cudaStream_t cast to void* (NULL = the legacy default stream).
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define LBM_OK             0
#define LBM_EINVAL         1   /* bad argument, size or parameter            */
#define LBM_ENOMEM         2   /* host or device allocation failed           */
#define LBM_EBUDGET        3   /* request can never fit the memory budget    */
#define LBM_ENOTCONVERGED  4   /* max_steps reached, or residual stagnated   */
#define LBM_ENONFINITE     5   /* NaN / Inf met in a residual or state       */
#define LBM_ETIMEOUT       6   /* a bounded device or host wait ran out      */
#define LBM_ECUDA          7   /* a CUDA runtime call failed                 */
#define LBM_EBUSY          8   /* queue or slot table full; retry later      */
#define LBM_ECANCELLED     9   /* the request was cancelled by the caller    */

/* Text of a status code (static storage). */
const char *lbm_status_string(int status);
/* Copy the calling thread's last error message (NUL-terminated, truncated to
 * n bytes).  Returns LBM_OK. */
int lbm_last_error(char *buf, size_t n);
/* Library version. */
int lbm_version(int *major, int *minor);

/* ---- lattices: xi = {c_a, w_a} (Sec. II, after Eq. (3)) ---------------- */
#define LBM_LATTICE_D2Q17   17  /* Shan-Yuan-Chen D2Q17, degree 7 (Sec. IV)  */
#define LBM_LATTICE_D2Q25   25  /* D1Q5 {0,+-1,+-3}^2, root r^2=(5+sqrt10)/3 */
#define LBM_LATTICE_D2Q25B  26  /* same set, other root r^2=(5-sqrt10)/3     */
#define LBM_LATTICE_D2Q37   37  /* degree-9 D2Q37 (the paper's cited set)   */

typedef struct lbm_lattice lbm_lattice;

/* Build a lattice: the library solves the Gaussian moment conditions for the
 * weights and the scale r in extended precision (Sec. II: "the discrete
 * velocity set may be determined through several ways").  *out is owned by
 * the caller and released with lbm_lattice_destroy.
 * Errors: LBM_EINVAL (unknown kind), LBM_ENOMEM. */
int lbm_lattice_create(int kind, lbm_lattice **out);
/* A lattice xi = {c_a = r e_a, w_a} from caller tables (Sec. II: the velocity
 * set "may be determined through several ways"): e is Q x 2 int8 (x then y, any
 * order), w the Q weights in the same order, r the scale.  The velocities must
 * be one of the built-in sets (Q = 17, 25 or 37; the kernels are compiled for
 * them), the weights positive and equal within each shell of symmetric
 * velocities; the isotropy degree is measured (lbm_lattice_info).  The tables
 * are copied; *out is owned by the caller.  Errors: LBM_EINVAL (message says
 * which condition failed), LBM_ENOMEM. */
int lbm_lattice_create_custom(int Q, const int8_t *e, const double *w, double r,
                              lbm_lattice **out);
int lbm_lattice_destroy(lbm_lattice *lat);
/* Q, scale r, ghost depth N = max |e_y| (Sec. III) and isotropy degree. */
int lbm_lattice_info(const lbm_lattice *lat, int *Q, double *r, int *ghost_depth,
                     int *degree);
/* Copy the tables: e (Q x 2 int8, x then y) and w (Q doubles); either may be
 * NULL.  Order is the library's velocity order used by every [Q] array. */
int lbm_lattice_tables(const lbm_lattice *lat, int8_t *e, double *w);
/* Largest |sum_a w_a c_ax^p c_ay^q - E[c_x^p c_y^q]| over p + q <= degree,
 * E the unit Gaussian moment (the isotropy the quadrature must satisfy for
 * Eq. (4)).  Errors: LBM_EINVAL if degree < 0 or > 16. */
int lbm_lattice_verify(const lbm_lattice *lat, int degree, double *max_err);

/* ---- solver parameters -------------------------------------------------- */
#define LBM_FP64     0   /* FP64 storage and arithmetic                        */
#define LBM_FP32     1   /* FP32 storage and arithmetic                        */
#define LBM_BF16DEV  2   /* BF16 storage of d_a = f~*_a - w_a rho, FP32 rho
                            plane, FP32 arithmetic; the step kernels round
                            the stored d stochastically (unbiased, from a
                            counter-based hash of step, cell and velocity), so
                            results are reproducible run to run             */
#define LBM_BF16SHIFT 3  /* BF16 storage of d_a = f~*_a - w_a rho_0 (rho_0 = 1,
                            the reference density of the non-dimensional
                            variables, Sec. II), FP32 arithmetic on the
                            deviations (the collision of LBM_FP32), the same
                            stochastic rounding of the stored d as
                            LBM_BF16DEV; no density plane: 4 Q bytes per cell
                            and step move through HBM.  Kernels: DIRECT and
                            CELLWARP (STAGED is LBM_EINVAL)                  */

#define LBM_KERNEL_AUTO     0   /* library picks                             */
#define LBM_KERNEL_DIRECT   1   /* one-pass pull kernel, global loads         */
#define LBM_KERNEL_STAGED   2   /* TMA-staged tile kernel (shared memory)     */
#define LBM_KERNEL_CELLWARP 3   /* one warp per cell (grids of a few thousand
                                   cells; AUTO picks it up to 4096 cells)    */

typedef struct lbm_params {
    int32_t Nx;          /* periodic columns, >= 1                            */
    int32_t Ny;          /* fluid rows between the walls, >= 2 * ghost depth  */
    int32_t eq_order;    /* Hermite orders kept in Eq. (4): 2, 3 or 4         */
    int32_t thermal;     /* 0: T = 1 in the collision (isothermal, Sec. II)   */
    double Kn;           /* Knudsen number of Eq. (15); tau = sqrt(2/pi) Kn
                            mu/(rho T) with mu = T^mu_exp (Sec. II)            */
    double tau;          /* > 0 overrides Kn with a constant tau (units of t)  */
    double mu_exp;       /* viscosity law exponent, default 1                  */
    double u_wall[2];    /* x-velocity of bottom and top wall                  */
    double T_wall[2];    /* wall temperatures; isothermal runs use 1           */
    int32_t precision;   /* LBM_FP64 / LBM_FP32 / LBM_BF16DEV / LBM_BF16SHIFT  */
    int32_t kernel;      /* LBM_KERNEL_*                                       */
    double rho0;         /* initial density of lbm_solver_init                 */
    double noise_amp;    /* initial rho = rho0 (1 + noise_amp (2U - 1))        */
    uint64_t seed;       /* U = SplitMix64 draw at counter j*Nx + x            */
    double accom[2];     /* accommodation per wall (bottom, top) of the
                            scattering kernel R = a R_D + (1 - a) R_S of Sec.
                            III, Eq. (9)-(10): 1 = diffuse (Eq. (11)-(12)),
                            0 = specular (the incoming population of the
                            mirrored velocity at the same ghost node), in [0, 1] */
} lbm_params;

/* Defaults: Nx = 1, Ny = 64, eq_order 2, isothermal, Kn 0.1, tau 0, mu_exp 1,
 * walls -0.1 / +0.1 at T 1, FP64, AUTO kernel, rho0 1, no noise, seed 7,
 * diffuse walls (accom 1). */
void lbm_params_default(lbm_params *p);

/* ---- single-domain solver ----------------------------------------------- */
typedef struct lbm_solver lbm_solver;

/* Device bytes a solver needs (two state buffers plus reduction space). */
int lbm_solver_required_bytes(const lbm_lattice *lat, const lbm_params *p,
                              size_t *bytes);

/* Create a solver.  If device_mem is non-NULL it must point to at least
 * lbm_solver_required_bytes bytes of device memory, 256-byte aligned, that the
 * caller owns and keeps alive until lbm_solver_destroy (the Python binding
 * passes a torch allocation); if NULL the library allocates (and frees) its
 * own with cudaMallocAsync on `stream`.  The lattice may be destroyed after
 * this call.  Errors: LBM_EINVAL (parameters; Ny < 2 N, eq_order, precision,
 * or Q x Ny x stored row >= 2^31 elements per state buffer, a stored row
 * being the grid's x-tiles' segments: Nx + 8 rounded up to 128 bytes, or to a
 * pitch class of 1056 / 2112 / 4224 elements, 1088 / 2112 / 4224 for
 * BF16DEV, or tiles of 4224), LBM_ENOMEM,
 * LBM_ECUDA. */
int lbm_solver_create(const lbm_lattice *lat, const lbm_params *p, void *stream,
                      void *device_mem, size_t device_bytes, lbm_solver **out);
int lbm_solver_destroy(lbm_solver *s);

/* f~* = rho g^eq(0, 1) with rho = rho0 (1 + noise_amp (2U - 1)); U is the
 * SplitMix64 draw (Steele, Lea & Flood 2014) of counter j*Nx + x under seed:
 * first output of the stream seeded with seed XOR counter, top 53 bits.
 * Asynchronous on the solver's stream; resets the step counter. */
int lbm_solver_init(lbm_solver *s);
/* f~* = rho g^eq(u, T) (Eq. (4)) from host fields [Ny][Nx]; ux, uy, T may be
 * NULL (0, 0, 1).  Synchronous.  Resets the step counter. */
int lbm_solver_init_fields(lbm_solver *s, const double *rho, const double *ux,
                           const double *uy, const double *T);

/* Enqueue n >= 0 time steps on the stream (asynchronous; no host round trip
 * inside).  Errors: LBM_EINVAL, LBM_ECUDA (launch failure). */
int lbm_solver_step(lbm_solver *s, int64_t n);
/* Wait for the solver's stream.  Errors: LBM_ECUDA. */
int lbm_solver_sync(lbm_solver *s);

/* Copy the post-collision state f~* to / from host FP64 [Q][Ny][Nx]
 * (converted from / to the storage precision).  Synchronous. */
int lbm_solver_get_f(lbm_solver *s, double *f);
int lbm_solver_set_f(lbm_solver *s, const double *f);

/* Macroscopic fields of Eq. (3) of the current state, host FP64 [Ny][Nx]
 * each; any pointer may be NULL.  T is the kinetic temperature
 * sum f |c - u|^2 / (D rho) even for isothermal runs.  Synchronous. */
int lbm_solver_macros(lbm_solver *s, double *rho, double *ux, double *uy,
                      double *T);

/* Steady-state estimate of a noisy iteration: advance the solver by nsteps
 * steps (asynchronous launches, then a synchronisation) and return the time
 * mean of the Eq. (3) fields over those steps, accumulated in FP64 on the
 * device (host buffers of Nx*Ny, any may be NULL).  The paper's scheme is
 * deterministic; with BF16 deviation storage the stored values are rounded
 * stochastically, so a steady state carries zero-mean noise (about 4e-3 U_w
 * in u_x on the 64-row Couette column) and the mean over a few thousand steps
 * is the steady field to about a tenth of that.  Errors: LBM_EINVAL,
 * LBM_ECUDA, LBM_ETIMEOUT (staged kernel). */
int lbm_solver_macros_mean(lbm_solver *s, int64_t nsteps, double *rho, double *ux, double *uy,
                           double *T);

/* Stress and heat flux (Sec. II: f~ = f + dt/(2 tau) (f - f^eq), so
 * f = (f~ + dt/(2 tau) f^eq) / (1 + dt/(2 tau))) of the pre-collision f~ that
 * the next step's streaming and wall fill produce from the current state:
 *   sigma_ij = sum (c_i - u_i)(c_j - u_j) f - rho T delta_ij,
 *   q_i      = 1/2 sum |c - u|^2 (c_i - u_i) f,
 * T = 1 in an isothermal run.  Computed in FP64 on the device from the stored
 * state (any precision).  Host FP64 outputs [Ny][Nx] each, caller-owned; any
 * may be NULL.  Synchronous.  Errors: LBM_EINVAL (NULL solver), LBM_ECUDA. */
int lbm_solver_fluxes(lbm_solver *s, double *sxx, double *sxy, double *syy,
                      double *qx, double *qy);

/* Checkpoint: the exact stored bytes plus the step counter.  get_state
 * writes state_bytes bytes to host memory; set_state restores them; a resumed
 * run is bit-identical to an uninterrupted one.  Errors: LBM_EINVAL if bytes
 * is smaller than the size (get) or differs from it (set). */
int lbm_solver_state_bytes(lbm_solver *s, size_t *bytes);
int lbm_solver_get_state(lbm_solver *s, void *buf, size_t bytes);
int lbm_solver_set_state(lbm_solver *s, const void *buf, size_t bytes);

/* Steady-state driver (the paper's Couette solutions are steady, Sec. IV):
 * run chunks of check_every steps; after each chunk
 *   res = max( ||u_x - u_x'||_2 / ||u_x||_2 ,
 *              thermal: ||T - T'||_2 / ||T - T_ref||_2 )
 * over all cells, primes = previous check, T_ref = mean wall temperature,
 * reductions in FP64 on the device.  Returns LBM_OK when res <= tol,
 * LBM_ENOTCONVERGED after max_steps or when res has not decreased over 50
 * consecutive checks, LBM_ENONFINITE on a NaN/Inf.  *steps and *res receive
 * the steps run by this call and the last residual. */
int lbm_solver_run_to_residual(lbm_solver *s, double tol, int64_t max_steps,
                               int32_t check_every, int64_t *steps, double *res);
/* Residual history of the last lbm_solver_run_to_residual call: one entry per
 * check, the solver's step count and the residual at that check (the
 * definition above).  Copies min(max, count) entries; *n receives the count.
 * Errors: LBM_EINVAL (NULL argument, or max > 0 with NULL arrays). */
int lbm_solver_residual_history(lbm_solver *s, int64_t *steps, double *res, int32_t max,
                                int32_t *n);

typedef struct lbm_stats {
    int64_t steps;        /* steps since the last init                        */
    double mass0;         /* sum of rho at init                               */
    double mass;          /* sum of rho now                                   */
    double mass_drift;    /* |mass - mass0| / mass0                           */
    double residual;      /* last residual of run_to_residual (or -1)        */
    double wall_in[2];    /* sum over columns of M_in of the last step,
                             bottom / top (numerator of Eq. (12))             */
} lbm_stats;
/* Synchronous (one reduction over the state). */
int lbm_solver_stats(lbm_solver *s, lbm_stats *st);

/* Step-kernel selection.  LBM_KERNEL_DIRECT: one thread per cell, populations
 * pulled straight from global memory; its variants differ in block width,
 * register cap, rows per block and store cache policy.  LBM_KERNEL_STAGED: persistent tile
 * kernel whose producer warp stages each velocity's shifted source window
 * (tile plus the +-3-cell halo, rounded to 16 bytes in x) into shared memory
 * with TMA; `variant` picks one of the compiled tile shapes, 0 <= variant <
 * nvariants; it runs grids stored as one x-tile only (Nx + 8 columns within
 * the tile pitch: 1056 elements for FP32 and FP64, 1088 for BF16DEV; wider
 * grids are stored as several x-tiles of that pitch).  AUTO uses DIRECT
 * variant 0 until set_kernel or autotune picks another.  Both compute the
 * same step (Eq. (5) with Eq. (12)).  Errors: LBM_EINVAL (also STAGED on a
 * grid of several x-tiles). */
int lbm_solver_set_kernel(lbm_solver *s, int32_t kernel, int32_t variant);

/* Limit, in nanoseconds of the GPU's global timer, of each bounded wait of
 * the staged kernel (its mbarrier waits between the producer warp and the
 * consumer warps; default 2 s).  The paper has no counterpart: it is the
 * library's failure detection.  A wait that runs out records a device flag,
 * the CTA stops taking tiles and its producer waits for its copies in flight
 * (with a fixed 2 s limit of its own) before the CTA exits; the next
 * lbm_solver_sync (or a synchronous call) returns LBM_ETIMEOUT and clears the
 * flag.  The state of that step is then incomplete: reload one (set_state,
 * set_f or init) before stepping on.  0 makes every such wait give up at
 * once, met or not (the failure path on demand; the drain before exit still
 * waits).  The other kernels have no waits.  Errors: LBM_EINVAL. */
int lbm_solver_set_wait_limit(lbm_solver *s, uint64_t ns);
/* Number of compiled variants of `kernel` (DIRECT or STAGED) for this
 * solver's precision.  Errors: LBM_EINVAL. */
int lbm_solver_variant_count(lbm_solver *s, int32_t kernel, int32_t *n);
/* Kernel in effect (AUTO resolved), its variant, and the number of staged
 * variants. */
int lbm_solver_kernel_info(lbm_solver *s, int32_t *kernel, int32_t *variant,
                           int32_t *nvariants);
/* Autotuner: time trial_steps steps of every direct and every staged
 * variant on this solver's grid (CUDA events on the solver's stream), keep
 * the fastest, and cache the choice per (lattice, precision, order, Nx and Ny
 * rounded up to powers of two) for the process, and in the file named by the
 * environment variable LBM_AUTOTUNE_CACHE when set.  Overwrites the state:
 * on return the solver holds the lbm_solver_init state.  Synchronous.
 * Errors: LBM_EINVAL, LBM_ECUDA. */
int lbm_solver_autotune(lbm_solver *s, int32_t trial_steps, int32_t *kernel,
                        int32_t *variant, double *ms_per_step);

/* Diffuse-wall incoming mass per ghost column (numerator of Eq. (12)) of the
 * current state: m_in[2][Nx] host FP64, bottom row then top row.  M_in(x) sums
 * the post-collision populations that stream into ghost column x through all
 * N ghost layers (Sec. III).  Synchronous. */
int lbm_solver_wall_mass(lbm_solver *s, double *m_in);

/* ---- residual reduction without allocation -------------------------------
 * The paper has no counterpart to this call: it is a service of the library.
 * It computes the steady-state residual that lbm_solver_run_to_residual
 * checks,
 *   res = max( ||ux - ux_prev||_2 / ||ux||_2 ,
 *              thermal: ||T - T_prev||_2 / ||T - T_ref||_2 ),
 * on caller-owned device arrays of n FP64 values, writes res to the device
 * double *res (NaN if any value is not finite), and then copies ux into
 * ux_prev and T into T_prev, as the solver does at each check.  All pointers
 * are device pointers; the work is enqueued on `stream` (asynchronous).
 *
 * It allocates nothing, for callers that cannot: code running while a CUDA
 * stream is being captured into a graph (where allocation calls are not
 * allowed), hosts that hand the whole device memory to another allocator or
 * run under a fixed memory budget, and embedding frameworks that forbid
 * libraries from allocating on their own.  Its scratch (1024 block partials
 * of 5 FP64 sums plus the totals, 41 KB) is a file-scope device array of the
 * library, created on every GPU that loads the library and kept until the
 * process exits.  The first call in a CUDA context looks up that array's
 * device address there (cudaGetSymbolAddress); the address is cached with the
 * context's unique ID (cuCtxGetId), so a call in another context - one the
 * caller created and made current, or the primary context re-created after
 * cudaDeviceReset - looks it up again instead of using an address of a
 * context that no longer holds it.  Make the first call in each context
 * before any stream capture begins.  All calls on a device share the
 * array and it keeps the last call's contents: calls whose kernels overlap on
 * the GPU (different streams, no ordering between them) race and return
 * garbage; calls ordered on one stream are safe.
 * Errors: LBM_EINVAL for a NULL pointer or n outside [1, 2^31 - 1] (nothing
 * is launched), LBM_ECUDA if the address look-up or a launch fails. */
int lbm_residual_noalloc(const double *ux, const double *T, double *ux_prev, double *T_prev,
                         int64_t n, double T_ref, int32_t thermal, double *res, void *stream);

/* ---- batched steady-state solves and the continuous-batching server ------
 * Each request is one steady Couette solve on a single periodic column
 * (Nx = 1) between the paper's two diffuse walls (Sec. IV set-up): its own
 * lattice, height, Kn (or tau), wall speeds and temperatures, FP32 storage
 * and arithmetic, FP64 wall-flux and residual reductions.  The solve starts
 * from rest (rho = 1, u = 0, T = 1) and stops when the extrapolated distance
 * to the steady state, res q / (1 - q), is at most `tol` at two checks in a
 * row: res is the largest change of the column's fields over one check in
 * the units of the requested accuracy - over the column's 32-row blocks, the
 * largest change of a block's mean u_x divided by U = max |u_wall| and, when
 * thermal, of a block's mean T (u_x and T compared as FP32 values) - and q
 * the ratio of successive changes; so `tol` is the accuracy asked for, the
 * L-inf distance of u_x / U (and of T) from the steady state, e.g. 1e-5.
 * The stored FP32 values are rounded stochastically (unbiased), so that the
 * steady state carries no systematic round-off.
 * (This differs from lbm_solver_run_to_residual's relative L2 residual,
 * which keeps the solver's definition.)  Checks run about four times per
 * e-folding time of the slowest shear mode, 0.127 Ny r / Kn steps.  A change
 * that has stopped shrinking for 8 checks at no more than tol / 20 also
 * counts as converged (the FP32 round-off floor); one that has not shrunk for
 * 50 checks above that ends the request with LBM_ENOTCONVERGED. */
typedef struct lbm_request {
    int32_t lattice;      /* LBM_LATTICE_*                                     */
    int32_t Ny;           /* rows, 6 <= Ny <= 8192                             */
    int32_t eq_order;     /* 2, 3 or 4                                         */
    int32_t thermal;      /* 0: isothermal (T = 1 in the collision)            */
    double Kn;            /* Knudsen number (Eq. (15)); or tau > 0             */
    double tau;
    double mu_exp;        /* mu = T^mu_exp                                     */
    double u_wall[2];     /* bottom, top wall x-velocity                       */
    double T_wall[2];     /* bottom, top wall temperature (thermal only)       */
    double tol;           /* target L-inf distance to the steady state of u_x / U
                             (and T), e.g. 1e-5                                */
    int64_t max_steps;    /* give up after this many steps                     */
    uint64_t tag;         /* caller's tag, returned in the result              */
    double accom[2];      /* wall accommodation, as in lbm_params (1: diffuse) */
    int32_t rounding;     /* LBM_ROUND_*: how the FP32 collision rounds        */
    int32_t init;         /* LBM_INIT_*: the state the solve starts from       */
} lbm_request;

/* lbm_request.init.  REST: rho = 1, u = 0, T = 1 (T_w for a thermal lattice
 * at rest is not imposed: T = 1).  NS: the local equilibrium at rho = 1 of the
 * Navier-Stokes slip solution of the paper's Couette problem (Sec. IV,
 * Eq. (13)-(14)): u_x(y) = (u_b + u_t)/2 + (u_t - u_b)(y - 1/2)/(1 + 2 lambda)
 * with the slip length lambda = Kn (2 - a)/a (a the mean accommodation), and
 * for a thermal lattice T(y) = T_b + (T_t - T_b) y + the viscous heating
 * 2 Pr U^2 y (1 - y)/(C_p (1 + 2 lambda)^2) plus the temperature jump
 * [8 gamma/(gamma + 1)] lambda U^2/(2 C_p (1 + 2 lambda)^2), U = (u_t - u_b)/2,
 * C_p = 2, gamma = 2, Pr = 1.  The steady state does not depend on the start
 * (the column's mass is the same); a start close to it takes fewer steps,
 * most of all in the dense, tall columns that dominate the latency tail. */
#define LBM_INIT_REST  0
#define LBM_INIT_NS    1

/* lbm_request.rounding.  AUTO: round to nearest while the change per check
 * is above 5 tol, then increments that conserve mass, momentum (and energy)
 * added with stochastic rounding, the admission mass restored at the switch
 * (round-to-nearest at a steady state leaves the same round-off every step,
 * which the slowest relaxation time amplifies).  STOCHASTIC: the conserving,
 * stochastically rounded increments from the first step (e.g. for runs to a
 * fixed step count).  NEAREST: round to nearest throughout. */
#define LBM_ROUND_AUTO        0
#define LBM_ROUND_STOCHASTIC  1
#define LBM_ROUND_NEAREST     2

typedef struct lbm_result {
    uint64_t id, tag;
    int32_t status;       /* LBM_OK, LBM_ENOTCONVERGED (max_steps or residual
                             stagnation), LBM_ENONFINITE                       */
    int32_t Ny;
    int64_t steps;
    double residual;      /* last change over one check (units of tol)        */
    double err_est;       /* extrapolated distance to the steady state (units
                             of tol) at the last check: at most tol when the
                             request stopped by extrapolation; 1e30 while the
                             change does not contract (a stop at the
                             round-off floor)                                */
    double mass;          /* sum of rho over the column at the last check     */
    double t_submit, t_admit, t_done;   /* seconds since server creation      */
} lbm_result;

typedef struct lbm_server_cfg {
    size_t mem_budget_bytes; /* device pool for the requests' f-arrays        */
    int32_t max_slots;       /* CTAs the running requests may occupy at once
                                (1..4096): a column of Ny rows runs on a
                                cluster of CL = 1, 2, 4, 8 or 16 CTAs of 256
                                threads, the smallest CL with ceil(Ny / CL) <=
                                cluster_rows (the largest if none), at most
                                max_slots; 16-CTA clusters only where the
                                device schedules them (else at most 8)       */
    int32_t chunk_steps;     /* steps per chunk launch                         */
    int32_t precision;       /* LBM_FP32                                       */
    int32_t use_graph;       /* replay the chunk launch as a CUDA graph        */
    int32_t cluster_rows;    /* rows per CTA above which a column is split over
                                a cluster (>= 32; default 256): smaller gives
                                lower latency per request, larger more solves
                                per second when the GPU is full             */
    int32_t class_sub[5];    /* chunks per launch of a slot on a cluster of 1,
                                2, 4, 8, 16 CTAs (0..16; 0: the built-in rule
                                max(1, CL / 2)); a cluster runs a step faster
                                than one CTA, so it runs several chunks while
                                one-CTA slots run one.  lbm_server_autotune
                                measures them.  Results do not depend on it. */
} lbm_server_cfg;

typedef struct lbm_server_metrics {
    int64_t submitted, completed, running, queued, chunks;
    double p50_latency_s, p99_latency_s, mean_latency_s;  /* submit -> done  */
    double solves_per_s;     /* completed / (last completion - first submit)  */
    double mean_occupancy;   /* mean fraction of max_slots busy per chunk     */
    size_t pool_bytes, pool_used_bytes;
    int64_t promoted;        /* running requests moved to a larger cluster once
                                CTAs were spare (results unchanged)           */
    int64_t demoted;         /* ... to a smaller one to make room for queued
                                requests (results unchanged)                  */
} lbm_server_metrics;

typedef struct lbm_server lbm_server;

/* 40 GB budget, 256 CTAs, 100-step chunks, FP32, CUDA graph on, clusters
 * above 256 rows per CTA. */
void lbm_server_cfg_default(lbm_server_cfg *cfg);
/* Device bytes one request occupies while admitted (two f-arrays of Q x Ny
 * floats plus two rows of previous-check fields, 256-byte granules). */
int lbm_request_bytes(const lbm_request *req, size_t *bytes);
/* Start a server: allocates the pool (cudaMallocAsync on `stream`), the slot
 * table and a host worker thread that owns `stream`.  Errors: LBM_EINVAL,
 * LBM_ENOMEM, LBM_ECUDA. */
int lbm_server_create(const lbm_server_cfg *cfg, void *stream, lbm_server **out);
/* Queue a request (thread-safe, non-blocking); it is admitted as soon as a
 * slot and pool memory are free, while other requests keep running.  A long
 * request may run on a cluster of CTAs, and between chunks a running one may
 * move to a larger cluster (CTAs spare) or a smaller one (queued requests
 * lack CTAs); its result does not depend on where it ran.
 * Errors: LBM_EINVAL (bad request), LBM_EBUDGET (larger than the budget). */
int lbm_server_submit(lbm_server *srv, const lbm_request *req, uint64_t *id);
/* Non-blocking: copy up to max finished results (oldest first) to out. */
int lbm_server_poll(lbm_server *srv, lbm_result *out, int32_t max, int32_t *n);
/* Copy a finished request's profiles (host FP64 arrays of Ny, any may be
 * NULL) and release them.  Errors: LBM_EINVAL for an unknown / fetched id. */
int lbm_server_fetch(lbm_server *srv, uint64_t id, double *rho, double *ux,
                     double *uy, double *T);
/* Cancel request `id`: a queued request is dropped, a running one stops at
 * the end of its current launch (one or a few chunks).  Either completes with status LBM_ECANCELLED
 * (poll returns it, drain counts it); fetch then gives the fields where a
 * running request stopped, and zeros for one that never ran.  Thread-safe.
 * Errors: LBM_EINVAL (no queued or running request with this id). */
int lbm_server_cancel(lbm_server *s, uint64_t id);
/* Block until every submitted request has finished, or timeout_s seconds.
 * Errors: LBM_ETIMEOUT, or the worker's LBM_ECUDA. */
int lbm_server_drain(lbm_server *srv, double timeout_s);
/* Latency percentiles, throughput and occupancy so far. */
int lbm_server_stats(lbm_server *srv, lbm_server_metrics *st);
/* Stop the worker (running requests are abandoned) and free everything. */
int lbm_server_destroy(lbm_server *srv);
/* Step times the batched-path autotuner measured (lbm_server_autotune). */
typedef struct lbm_server_tuning {
    int32_t ny[3];              /* column heights timed: 256, 1024, 4096      */
    double lone_us[3][3][5];    /* us per step of one lone column: lattice
                                   D2Q17 / D2Q25 / D2Q37, height ny[i], on a
                                   cluster of 1, 2, 4, 8, 16 CTAs (0: that
                                   split is not usable or not schedulable)    */
    int32_t chunk_try[5];       /* chunk lengths timed on a full GPU          */
    double chunk_glups[5];      /* lattice updates per second (1e9) of
                                   max_slots one-CTA D2Q37 columns of 256 rows
                                   at each chunk length, launches included
                                   (best of two runs)                          */
    double seconds;             /* wall time of the autotuning                */
} lbm_server_tuning;

/* Autotuner of the batched path (the paper has no counterpart: it is a
 * service of the library).  Starting from *cfg (budget, max_slots, graph
 * use), it times on this device, through servers it creates and destroys:
 *  - one lone column of each lattice at heights 256, 1024 and 4096 on each
 *    usable cluster size (long runs, so launch overhead is negligible), and
 *  - max_slots one-CTA columns at chunk lengths 25, 50, 100, 200, 400,
 * then writes into *cfg: class_sub[c] = the step time of a lone D2Q37
 * column of CL x 256 rows (the tallest a CL-CTA cluster serves at 256 rows
 * per CTA) on one CTA over that on the class's cluster of CL CTAs (how many
 * chunks a cluster slot runs while a one-CTA slot runs one, 1..16);
 * cluster_rows = the median over lattices and heights of the rows per CTA
 * of the smallest cluster within 15 % of the fastest (32 .. 1024); and
 * chunk_steps = the longest chunk within 5 % of the best full-GPU rate
 * (fewer launches, each a host round trip).  Takes about half a minute;
 * the device must be otherwise idle for the times to mean anything.  `stream`
 * as for lbm_server_create; `report` (may be NULL) receives the times.
 * Results of a solve do not depend on cluster_rows or class_sub; chunk_steps
 * moves the steps at which its convergence checks fall.
 * Errors: LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA. */
int lbm_server_autotune(lbm_server_cfg *cfg, void *stream, lbm_server_tuning *report);

/* Batched solve: a server with `cfg`, all n requests submitted at once,
 * drained (timeout_s), results written to out[i] for reqs[i]. */
int lbm_batch_solve(const lbm_server_cfg *cfg, void *stream, const lbm_request *reqs,
                    int32_t n, lbm_result *out, double timeout_s);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
