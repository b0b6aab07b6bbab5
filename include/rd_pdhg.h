/*
 * rd_pdhg.h -- C ABI of the GB300 G-prox PDHG solver for implicit reaction-diffusion steps.
 *
 * Method (arxiv 2305.03945, "A first-order computational algorithm for reaction-diffusion type
 * equations via primal-dual hybrid gradient method"):
 *   one implicit (or semi-implicit) time step U^k -> U^{k+1} of a reaction-diffusion equation on
 *   a finite-difference grid is the root of a nonlinear map F (Section 2.1, eq. F(U) rd
 *   equation).  F(U) = 0 is rewritten as the saddle problem min_U max_P P^T F(U) (Section 2.1,
 *   eq. illustrate saddle) and solved by the linearised G-prox PDHG iteration
 *     P_{n+1} = P_n + tau_p G^{-1} F(U_n)                       (eq. G-prox ... dynamic 1)
 *     P~      = P_{n+1} + omega (P_{n+1} - P_n)                  (eq. G-prox ... dynamic 2)
 *     U_{n+1} = U_n - tau_u dF(U_n)^T P~                         (eq. G-prox ... dynamic 3)
 *   from U_0 = U^k, P_0 = 0, until ||Res(U_n)||_2 <= delta (Section 2.1, stopping criterion),
 *   with G = A_lin^2 inverted by 2-D FFT (periodic) or DCT-II (Neumann) (Section 2.1,
 *   "Choosing the matrix G", Remark 1).  Algorithm 1 is the outer time loop.
 *
 * Everything runs on ONE CUDA device in hand-written sm_103a kernels.  Unless stated otherwise
 * every pointer named "device" is a CUDA device pointer the CALLER owns; the handle owns all
 * internal workspaces, allocated once by rd_pdhg_create and freed by rd_pdhg_destroy (step and
 * solve never allocate).  No C++ exception crosses this ABI; every function returns an
 * rd_status and leaves a human-readable detail string for rd_last_error().
 *
 * Grid layout: an array of ncomp*ny*nx doubles, component-major, then y, then x (x contiguous):
 * element (c, i, j) is at c*ny*nx + i*nx + j.  This is the vectorisation l = i*N_x + j of
 * Section 2.1 (i the y index, j the x index).  Periodic nodes sit at (j h_x, i h_y); Neumann
 * nodes at cell centres ((j+1/2) h_x, (i+1/2) h_y) with the half-cell mirror ghost
 * U_{-1} = U_0 of Remark 1; in both cases h_x = length[0]/nx, h_y = length[1]/ny.
 */
#ifndef RD_PDHG_H
#define RD_PDHG_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define RD_API __attribute__((visibility("default")))
#else
#define RD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RD_OK = 0,
    RD_ERR_INVALID_ARG = 1,    /* a NULL handle/pointer, n < 2, dt <= 0, tau <= 0, a < 0, ...   */
    RD_ERR_UNSUPPORTED = 2,    /* valid but not built: e.g. non-power-of-two n, 3-D two species  */
    RD_ERR_OOM = 3,            /* cudaMalloc failed                                              */
    RD_ERR_CUDA = 4,           /* another CUDA runtime error (detail in rd_last_error)           */
    RD_ERR_NOT_CONVERGED = 5,  /* max_iter PDHG updates did not meet the stopping rule           */
    RD_ERR_DIVERGED = 6,       /* the stopping measure became non-finite or grew 1e8-fold        */
    RD_ERR_TIMEOUT = 7,        /* a bounded device or host wait ran out                          */
    RD_ERR_BUSY = 8            /* batch: no free slot / over the memory budget                   */
} rd_status;

typedef enum { RD_BC_PERIODIC = 0, RD_BC_NEUMANN = 1 } rd_bc;

/* Linear diffusion operator L of the equation u_t = L u + R(u) (Section 1, eq. rd equ). */
typedef enum {
    RD_OP_LAPLACIAN = 0,       /* L = a Lap            (Allen-Cahn, Gray-Scott, Schnakenberg)   */
    RD_OP_NEG_BIHARMONIC = 1,  /* L = -a Lap^2         (Cahn-Hilliard, Section 3.2)             */
    RD_OP_FUNCTIONALIZED = 2   /* sixth order, with RD_RX_FCH only (Section 3.3)               */
} rd_operator;

/* Reaction term R and the residual map F it defines (dt = h_t):
 *   RD_RX_NONE          F = (I - a dt Lap) U - U^k    or (I + a dt Lap^2) U - U^k
 *   RD_RX_ALLEN_CAHN    F = U - U^k - dt (a Lap U - b (U^3 - U))        (Section 3.1, eq. AC equ)
 *   RD_RX_CH_IMPLICIT   F = (I + a dt Lap^2) U - U^k - b dt Lap (U^3 - U)    (eq. F(U) CH)
 *   RD_RX_CH_SPLIT      F = (I + a dt Lap^2) U - U^k - b dt Lap U^3 + b dt Lap U^k
 *                       (convex-concave split: U^3 implicit, -U explicit)
 *   RD_RX_GRAY_SCOTT    ncomp = 2, p = {Du, Dv, F, k}:
 *                       F_u = U - U^k - dt (Du Lap U - U V^2 + F (1 - U))
 *                       F_v = V - V^k - dt (Dv Lap V + U V^2 - (F + k) V)
 *   RD_RX_SCHNAKENBERG  ncomp = 2, p = {D1, D2, kappa, a_s, b_s}       (Section 3.4.1)
 *                       F_u = U - U^k - dt (D1 Lap U + kappa (a_s - U + U^2 V))
 *                       F_v = V - V^k - dt (D2 Lap V + kappa (b_s - U^2 V))
 *   RD_RX_FCH           sixth-order functionalized Cahn-Hilliard (Section 3.3), a = eps^2:
 *                       F = U - U^k - dt Lap (a Lap - b W''(U) + a)(a Lap U - b W'(U)),
 *                       W' = U^3 - U, W'' = 3U^2 - 1; G = (I - dt Lap (a Lap - (2b - a)) a Lap)^2.
 *                       RD_PREC_FP64 only (RD_ERR_UNSUPPORTED otherwise), not batched.
 * The allowed operator is RD_OP_LAPLACIAN for AC / Gray-Scott / Schnakenberg,
 * RD_OP_NEG_BIHARMONIC for both Cahn-Hilliard kinds, RD_OP_FUNCTIONALIZED for RD_RX_FCH (and
 * only for it); RD_RX_NONE takes the first two. */
typedef enum {
    RD_RX_NONE = 0,
    RD_RX_ALLEN_CAHN = 1,
    RD_RX_CH_IMPLICIT = 2,
    RD_RX_CH_SPLIT = 3,
    RD_RX_GRAY_SCOTT = 4,
    RD_RX_SCHNAKENBERG = 5,
    RD_RX_FCH = 6
} rd_reaction_kind;

/* Grid.  2-D: sides nx, ny.  3-D (ndim = 3, not in the paper, which is 2-D: its scheme with a
 * third axis -- seven-point Laplacian, Lap^2 as its square, transforms along x, y and z; scalar
 * kinds RD_RX_NONE, Allen-Cahn and both Cahn-Hilliard forms; arrays [ncomp][nz][ny][nx]).
 * Every side is a power of two, at least 2; at most 2048 on 3-D grids and 8192 on 2-D grids.
 * 2-D grids with a side above 2048 (RD_PREC_FP32_DC) or 4096 (RD_PREC_FP64) run on the
 * line-transform kernels of 3-D grids (pointwise residual and update, one transform pass per
 * axis, the spectral scaling on the y pass) and take the scalar kinds only; longer sides, and
 * two-species or sixth-order equations on such grids, return RD_ERR_UNSUPPORTED. */
typedef struct {
    int ndim;            /* 2 or 3                                                             */
    int n[3];            /* n[0] = nx (contiguous), n[1] = ny, n[2] = nz (3-D)                 */
    double length[3];    /* side lengths; h_x = length[0]/nx, h_y = length[1]/ny, h_z = length[2]/nz */
} rd_grid;

typedef struct {
    int kind;            /* rd_reaction_kind                                                   */
    int ncomp;           /* 1, or 2 for the two-species kinds (must match the kind)            */
    double a, b;         /* diffusion and reaction scales (a >= 0, b >= 0)                     */
    double p[6];         /* kind-specific parameters, see rd_reaction_kind                     */
} rd_reaction;

/* Preconditioner G of the dual proximal step (Section 2.1, "Choosing the matrix G"). */
typedef enum {
    RD_PC_NONE = 0,      /* G = I: the plain linearised PDHG (eqs. illustrate pdhg dynamic 1-3) */
    RD_PC_LINEAR = 1,    /* G = A_lin^2, A_lin the constant-coefficient linear part of F:
                            (I - D dt Lap)^2 per species, or (I + a dt Lap^2)^2 (default)       */
    RD_PC_STABILIZED = 2 /* G = A_s^2, A_s the Jacobian of F with its nonlinear factor replaced by
                            the constant s (Section 3.3's construction of G, for any scalar
                            reaction): Allen-Cahn (1 + b dt s) I - a dt Lap; Cahn-Hilliard
                            I + a dt Lap^2 - b s dt Lap (s in place of W''(U), or of 3 U^2 for the
                            convex split: 2, resp. 3, at u = +-1, where G equals the square of the
                            exact Jacobian); sixth order with (s b - a) in place of (2b - a).
                            Scalar reactions only (else RD_ERR_UNSUPPORTED).  Near u = +-1 it keeps
                            PDHG convergent where RD_PC_LINEAR's iteration diverges (stiff
                            reaction terms b dt).                                             */
} rd_precond_kind;

typedef struct { int kind; double s; } rd_precond;   /* s: the RD_PC_STABILIZED constant (>= 0);
                                                         0 for the other kinds */

typedef enum {
    RD_TOL_RES_ABS = 0,  /* stop when sum_c ||F_c(U_n)||_2 / dt <= tol  (||Res||_2 <= delta)   */
    RD_TOL_F_REL = 1     /* stop when sum_c ||F_c(U_n)||_2 <= tol * ||U^k||_2                    */
} rd_tol_kind;

typedef enum {
    RD_PREC_FP64 = 0,    /* every PDHG sweep in FP64 (plain method)                             */
    RD_PREC_FP32_DC = 1  /* FP32 PDHG sweeps on the correction equation inside an FP64 defect-
                            correction loop: r = F(u) in FP64, solve F(u + d) = 0 for d in FP32
                            until ||F~(d)|| <= dc_inner_rtol ||r||, u += d in FP64, repeat until
                            the stopping rule above holds for F(u) evaluated in FP64             */
} rd_precision;

typedef enum {
    RD_LOOP_GRAPH = 0,    /* the PDHG iterations run in a WHILE node of the step's CUDA graph
                             (graph_k iterations per trip) that the kernels end themselves, and
                             the defect-correction outer rounds in a second WHILE node around
                             it: one graph launch per step                                    */
    RD_LOOP_HOST = 1      /* plain CUDA graphs of graph_k iterations (one outer round of defect
                             correction at a time), launched until the host reads a finished
                             state: the same kernels as ordinary graph kernel nodes (profilers
                             cannot attribute kernels inside conditional nodes)                */
} rd_solve_loop;

typedef struct {
    double tol;           /* stopping threshold (delta), default 1e-10                          */
    int tol_kind;         /* rd_tol_kind, default RD_TOL_RES_ABS                                */
    int max_iter;         /* PDHG updates per step (FP64) or per inner solve (DC); default 10000 */
    double omega;         /* extrapolation coefficient, default 1 (Section 3)                   */
    int precision;        /* rd_precision, default RD_PREC_FP64                                 */
    double dc_inner_rtol; /* DC inner tolerance factor, default 1e-5: the FP32 solve of a round
                             stops at max(dc_inner_rtol ||r||, half the outer threshold)        */
    int dc_max_outer;     /* DC outer rounds per step before RD_ERR_NOT_CONVERGED, default 64
                             (the paper's seven-circle Cahn-Hilliard example at tau = 0.5 takes
                             about 16 rounds of a few inner iterations each)                    */
    int graph_k;          /* PDHG iterations per trip of the device-side loop (a WHILE node of the
                             step's CUDA graph), default 2                                      */
    int band_rows;        /* rows per CTA of the stencil sweeps (k_res and k_upd); 0 = chosen at
                             create (occupancy planner, or measured with autotune)              */
    int col_width;        /* columns per CTA of the column transform; 0 = chosen at create      */
    int upd_rows;         /* rows per CTA of the update sweep k_upd when it differs from k_res;
                             0 (default) = band_rows                                            */
    int profile;          /* 1: time the three PDHG kernels of the first iteration of every graph
                             launch with CUDA events (read back by rd_pdhg_get_stats)            */
    int fft_buffers;      /* shared-memory transforms: 0 = chosen per kernel (two buffers where the
                             second costs no resident blocks), 1 = in place in one buffer,
                             2 = two buffers wherever they fit; default 0                       */
    int solve_loop;       /* rd_solve_loop, default RD_LOOP_GRAPH                               */
    int fft_unrolled;     /* 1 (default): transform passes unrolled per line length at compile
                             time; 0: one looped pass body for every pass                       */
    int autotune;         /* 1: at create, time each sweep kernel over a few PDHG iterations at
                             every tile that fits and keep the fastest per kernel (band rows of
                             k_res and of k_upd, column width of k_col; ignored when band_rows
                             or col_width is set); 0 (default): the occupancy-based planner.
                             Timing noise can change the choice between runs, and with it the
                             summation order of the stopping norm (results agree to rounding). */
    int dc_stall_window;  /* DC: the FP32 inner solve also stops (as converged) when its residual
                             has not halved for this many updates (its rounding floor); default
                             8                                                                   */
    int fused_update;     /* 1 (default): FP32 defect correction (either loop) runs the update
                             of each iteration fused with the next residual (k_col + k_updres
                             per iteration; k_res only before the first update) when its block
                             fits, and with autotune only where it measures faster; 0: never.
                             Fused and unfused inner iterates differ by FP32 rounding only.     */
    int small_solve;      /* 1 (default): FP32 defect correction on a 2-D grid small enough that
                             every array of the inner solve fits on chip runs each inner solve as
                             ONE kernel launch, its iterations separated by barriers: one block
                             below 16 points a side (up to 4 K points), a cluster of eight blocks
                             with distributed shared memory from 16 x 16 up to 16 K points; the
                             outer rounds then loop on the device too (one graph launch and one
                             host read per step); 0: never */
} rd_opts;

typedef struct {
    int iterations;       /* PDHG updates (DC: summed over inner solves)                        */
    int outer_rounds;     /* DC outer rounds (FP64 residual evaluations); 0 for plain FP64      */
    int converged;        /* 1 when the stopping rule held                                      */
    int status;           /* rd_status of this step                                             */
    double residual;      /* the stopping measure at the returned iterate                       */
    double mass;          /* h_x h_y sum of all components of U^{k+1}                           */
} rd_step_info;

/* Counters of a handle since creation (or the last rd_pdhg_reset_stats). */
typedef struct {
    long long kernel_launches;   /* kernels this library launched (graph nodes included)        */
    long long graph_launches;    /* CUDA graph launches of the PDHG iteration                   */
    long long pdhg_iterations;   /* PDHG updates (FP64 plain or FP32 inner)                     */
    long long residual_passes;   /* FP64 residual evaluations of defect correction              */
    long long host_syncs;        /* device -> host status reads                                 */
    double kernel_ms[3];         /* profile = 1: summed CUDA-event time of k_res, k_col, k_upd   */
    long long kernel_samples[3]; /* number of timed launches behind kernel_ms                    */
    int plan_band_rows;          /* rows per CTA of the sweeps chosen at create (planner/autotune) */
    int plan_col_width;          /* columns per CTA of the column transform chosen at create      */
    int plan_upd_rows;           /* rows per CTA of the update sweep (k_upd) chosen at create    */
    int fused_update;            /* 1 when the fused update + residual kernel (k_updres) runs      */
    int small_solve;             /* inner solves in one launch (rd_opts.small_solve): 1 one block,
                                    2 a cluster of eight blocks, 0 the multi-kernel sweeps        */
    int line_kernels;            /* 1 when the iteration runs on the line-transform kernels (3-D
                                    grids; 2-D grids with a side beyond the band / column sweeps) */
} rd_stats;

typedef struct rd_pdhg rd_pdhg;

/* Fill *o with the defaults listed in rd_opts. */
RD_API void rd_opts_default(rd_opts *o);

/* Create a solver for one grid / equation / time step.
 *   dt     physical time step h_t > 0
 *   tau    PDHG primal step tau_u > 0;  sigma  PDHG dual step tau_p > 0   (Section 2.1)
 *   precond may be NULL (= RD_PC_LINEAR); opts may be NULL (= rd_opts_default)
 *   cuda_stream: a cudaStream_t (NULL = legacy default stream); all work is issued on it.
 * Allocates every workspace (about 7 arrays of the grid size plus twiddle tables) and captures
 * the step graphs: the PDHG iteration loop runs on the device as a WHILE node of a CUDA graph
 * (graph_k iterations per trip) that the kernels end themselves, and the outer rounds of
 * defect correction as a WHILE node around it, so that a step of either precision is one graph
 * launch and one host read.  Needs a GPU and driver with CUDA-graph conditional nodes.  On
 * error *out is NULL. */
RD_API rd_status rd_pdhg_create(rd_pdhg **out, const rd_grid *grid, rd_bc bc, rd_operator op,
                         const rd_reaction *reaction, double dt, double tau, double sigma,
                         const rd_precond *precond, const rd_opts *opts, void *cuda_stream);

/* One implicit step: u_np1 <- root of F for U^k = u_n (both device, ncomp*ny*nx doubles; they
 * may alias).  Blocks until the step is finished (convergence needs a device->host read).
 * info (host, may be NULL) is filled in every case.  Returns RD_ERR_NOT_CONVERGED or
 * RD_ERR_DIVERGED with u_np1 holding the last iterate. */
RD_API rd_status rd_pdhg_step(rd_pdhg *h, const double *u_n, double *u_np1, rd_step_info *info);

/* Algorithm 1's time loop: nsteps implicit steps in place on u (device).  per_step (host) may be
 * NULL or an array of nsteps entries.  Stops at the first step that fails. */
RD_API rd_status rd_pdhg_solve(rd_pdhg *h, double *u, int nsteps, rd_step_info *per_step);

/* As rd_pdhg_solve, for a HOST array u: copies it to the device, solves, copies it back. */
RD_API rd_status rd_pdhg_solve_host(rd_pdhg *h, double *u_host, int nsteps, rd_step_info *per_step);

/* Change the physical time step h_t of a live handle (dt finite, > 0).  Every quantity that
 * depends on h_t (the residual and adjoint coefficients, the preconditioner symbol
 * (1 + c1 mu + c2 mu^2 + c3 mu^3)^2) is re-derived and the step graphs are captured again, so a change
 * costs about one graph capture; the tile plan and the workspaces are kept.  Synchronises the
 * handle's stream.  RD_ERR_INVALID_ARG leaves the handle unchanged. */
RD_API rd_status rd_pdhg_set_dt(rd_pdhg *h, double dt);

/* Adaptive time step size (Section 2.2, "Adaptive time stepsize").  After each accepted step
 * that took M PDHG iterations (DC: summed over inner solves) the next h_t is
 *     eta h_t  if M > n_hi;   h_t / eta  if M < n_lo and h_t / eta <= h_t^0;   else h_t,
 * with h_t^0 the handle's dt on entry (the upper bound).  A step whose solve fails
 * (RD_ERR_NOT_CONVERGED or RD_ERR_DIVERGED) is not accepted: it is taken again from the same
 * state with eta h_t.  The last step is shortened to end at t_end (the rule keeps acting on the
 * nominal h_t). */
typedef struct {
    double t_end;       /* integrate from t = 0 to t_end (finite, > 0)                          */
    int n_hi;           /* N^*: more iterations than this shrink h_t                             */
    int n_lo;           /* N_*: fewer iterations than this enlarge h_t; 0 <= n_lo <= n_hi         */
    double eta;         /* rescaling coefficient, 0 < eta < 1                                     */
    int max_attempts;   /* bound on accepted + rejected steps (> 0)                               */
} rd_adapt;

typedef struct {
    double t;           /* time at the start of the attempt                                       */
    double dt;          /* step size used                                                         */
    int iterations;     /* PDHG iterations of the attempt (DC: summed over inner solves)          */
    int outer_rounds;   /* DC outer rounds; 0 for plain FP64                                      */
    int status;         /* rd_status of the attempt's step                                        */
    int accepted;       /* 1 when the step converged and the state advanced                       */
} rd_adapt_step;

/* Run the adaptive loop in place on u (device, ncomp*ny*nx doubles: U at t = 0 in, U at the
 * reached time out).  log (host, may be NULL when log_cap = 0) receives the first log_cap
 * attempts in order; *n_attempts (may be NULL) the number of attempts and *t_reached (may be
 * NULL) the time reached.  Returns RD_OK when t_end - t <= 1e-12 t_end, RD_ERR_NOT_CONVERGED
 * when max_attempts ran out first (u holds the last accepted state), or the first error that is
 * not a failed solve (RD_ERR_CUDA, RD_ERR_TIMEOUT, ...).  The handle's dt is h_t^0 again on
 * return. */
RD_API rd_status rd_pdhg_solve_adaptive(rd_pdhg *h, double *u, const rd_adapt *a, rd_adapt_step *log,
                                        int log_cap, int *n_attempts, double *t_reached);

/* W <- F(U) for U^k = u_k (all device, FP64): the residual map of the handle's equation
 * (eq. F(U) rd equation / F(U) CH / Section 3.4.1). */
RD_API rd_status rd_pdhg_residual(rd_pdhg *h, const double *u, const double *u_k, double *w);

/* Y <- G^{-1} W (device, FP64): the preconditioner solve of eq. G-prox dynamic 1 with the
 * handle's G (rd_precond_kind: A_lin^2, A_s^2, or I), by FFT-type (periodic) or DCT-II (Neumann)
 * transforms along every axis.  y may alias w. */
RD_API rd_status rd_pdhg_apply_precond(rd_pdhg *h, const double *w, double *y);

/* Copy the handle's counters to *out (host). */
RD_API rd_status rd_pdhg_get_stats(const rd_pdhg *h, rd_stats *out);
RD_API rd_status rd_pdhg_reset_stats(rd_pdhg *h);

RD_API void rd_pdhg_destroy(rd_pdhg *h);

/* ---------------------------------------------------------------------------------------
 * Batched, continuously served solves (no counterpart in the paper: a serving layer over the
 * same method).  Every request is an independent run of nsteps implicit steps of one equation
 * (RD_RX_NONE, Allen-Cahn, Cahn-Hilliard, Gray-Scott or Schnakenberg; 2-D grids with sides powers
 * of two in [4, 1024], or -- scalar kinds -- 3-D grids with sides in [4, 512]; either boundary
 * condition) solved with FP32 PDHG sweeps (G = A_lin^2, RD_PC_LINEAR) inside FP64 defect
 * correction to the request's tolerance.  Small 2-D requests (up to 16 K points) run each
 * inner solve in one launch (rd_opts.small_solve).  The batch owns one device arena of
 * hbm_budget_bytes; a request is admitted when a slot is free and its workspace (about 48
 * bytes per grid point) fits the arena, its state then stays resident on the GPU across all its
 * steps, and all admitted requests advance together in shared launches (one per equation kind
 * and sweep kernel, over every admitted grid size) of a CUDA graph that a library thread
 * relaunches until the slot finishes.  Requests submitted while others run are admitted as slots and memory free up.
 * --------------------------------------------------------------------------------------- */
typedef struct rd_batch rd_batch;

typedef struct {
    rd_grid grid;
    int bc;                /* rd_bc                                                             */
    int op;                /* rd_operator (must match the kind, as for rd_pdhg_create)          */
    rd_reaction reaction;
    double dt;             /* h_t                                                               */
    double tau, sigma;     /* PDHG primal / dual steps                                          */
    double tol;            /* stopping threshold of every step (FP64 residual)                  */
    int tol_kind;          /* rd_tol_kind                                                       */
    int nsteps;            /* implicit steps to take (>= 1)                                     */
    const double *u0_host; /* host, ncomp*ny*nx doubles; copied by rd_batch_submit              */
    uint64_t tag;          /* caller's label, echoed in the result                              */
} rd_request;

typedef struct {
    uint64_t id, tag;
    int status;            /* rd_status of the run                                              */
    int steps;             /* steps completed                                                   */
    long long iterations;  /* FP32 PDHG updates over all steps                                  */
    int outer_rounds;      /* FP64 residual evaluations over all steps                          */
    double residual;       /* last stopping measure                                             */
    double t_submit, t_admit, t_done;  /* host steady-clock seconds                             */
} rd_result;

typedef struct {
    long long submitted, admitted, completed, graph_launches, queued, arena_free_bytes;
} rd_batch_stats;

/* Create a batch: arena of hbm_budget_bytes (allocated here, once), at most max_slots requests
 * resident at a time, solver options (graph_k, max_iter, dc_inner_rtol, dc_max_outer, omega,
 * small_solve, autotune; NULL = defaults), work issued on cuda_stream.  With autotune = 1 the
 * band rows and column width of the batched sweeps are measured here for every square grid size
 * the arena holds (16 .. 1024, a few milliseconds) and admitted requests take the fastest for
 * their size.  Starts the library's scheduling thread. */
RD_API rd_status rd_batch_create(rd_batch **out, size_t hbm_budget_bytes, int max_slots,
                                 const rd_opts *opts, void *cuda_stream);

/* Queue one request (u0 copied now).  When it finishes, its final state is copied to
 * u_out_host (host, ncomp*ny*nx doubles, must stay valid until then; may be NULL) and a result
 * becomes available to rd_batch_poll.  RD_ERR_BUSY: larger than the whole budget. */
RD_API rd_status rd_batch_submit(rd_batch *b, const rd_request *req, double *u_out_host,
                                 uint64_t *id);

/* Move up to cap finished results into done (host array); waits up to timeout_s seconds for
 * the first one when none is ready. */
RD_API rd_status rd_batch_poll(rd_batch *b, rd_result *done, int cap, int *n_done,
                               double timeout_s);

RD_API rd_status rd_batch_get_stats(rd_batch *b, rd_batch_stats *out);

/* Stop the scheduling thread (queued requests are dropped, running ones abandoned) and free
 * everything. */
RD_API void rd_batch_destroy(rd_batch *b);

/* Y <- G^{-1} W without any device allocation.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory when they need the operator -- code
 * running inside a fixed memory budget it does not own, latency-critical loops that must not
 * pay the device-wide synchronisation of cudaMalloc / cudaFree, or callers holding no solver
 * handle.  It computes the same G = A_lin^2 solve as rd_pdhg_apply_precond of an RD_PC_LINEAR
 * handle for the 2-D equation described by (grid, bc, op, reaction, dt), with its scratch
 * (transform buffer, twiddle and eigenvalue tables) in one static device array of 2.5 MiB that
 * every device loading the library holds until process exit.
 *   w, y: device arrays of ncomp*ny*nx doubles (caller-owned; y may alias w).
 *   cuda_stream: cudaStream_t to issue the work on (NULL = legacy default); returns after the
 *   stream is synchronised.
 *   Limits: ncomp*nx*ny <= 131072 points and sides <= 2048, else RD_ERR_UNSUPPORTED.
 *   The first call on a device does a one-time set-up for that device (looks up the scratch
 *   array's device address, raises the kernels' shared-memory limit); make it before any stream
 *   capture.  All calls share the scratch array and it keeps the last call's contents (every
 *   entry is rewritten before it is read); calls that overlap on the GPU race on it, so order
 *   them on one stream. */
RD_API rd_status rd_apply_precond_static(const rd_grid *grid, rd_bc bc, rd_operator op,
                                         const rd_reaction *reaction, double dt, const double *w,
                                         double *y, void *cuda_stream);

RD_API const char *rd_status_string(rd_status s);
RD_API const char *rd_last_error(void);   /* detail of the last failing call on this thread */

#ifdef __cplusplus
}
#endif

#endif /* RD_PDHG_H */
