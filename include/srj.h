/*
 * srj.h -- C ABI of the GB300 (sm_103a) Scheduled Relaxation Jacobi library.
 *
 * Method: Adsuara, Cordero-Carrion, Cerda-Duran, Aloy, "Scheduled Relaxation
 * Jacobi method: improvements and applications", arXiv:1511.04292.
 *
 * The library solves the Dirichlet Poisson problem -Laplace(u) = f on a uniform
 * 2-D (5-point stencil) or 3-D (7-point stencil) grid with spacing h by SRJ:
 * weighted-Jacobi steps (Sect. 3.1, Eq. 2nd-order_CD, with the Poisson source of
 * Sect. 5.1)
 *
 *     u'_p = u_p + (omega_k / 2d) * (h^2 f_p + sum_{neighbours q} u_q - 2d u_p),
 *
 * whose weights omega_k run through an M-cycle in which level i (weight omega_i)
 * appears q_i times (Sect. 2).  Convergence is tested at cycle ends on the
 * relative L2 norm of the residual r = b - A_h u, A_h = 2d I - neighbour sum,
 * b = h^2 f (+ Dirichlet ghost neighbours).
 *
 * GRID LAYOUT (all u / f / r arrays passed through this ABI)
 *   A dense row-major float64 array of the interior points plus one ghost layer
 *   on each side, x fastest:
 *     2-D: element (x, y)    at  y * (nx+2) + x,                 0 <= x <= nx+1, 0 <= y <= ny+1
 *     3-D: element (x, y, z) at  (z * (ny+2) + y) * (nx+2) + x
 *   Interior points have 1 <= x <= nx (etc.).  The ghost layer of u carries the
 *   Dirichlet boundary values and is never written.  The ghost layer of f is
 *   ignored.  h is the same on every axis.
 *
 * POINTERS, STREAMS AND OWNERSHIP
 *   Array arguments are DEVICE pointers on the CUDA device that was current when
 *   the plan was created, unless a function says otherwise.  The caller owns
 *   them; the library never frees or retains them past the call.  `stream` is a
 *   cudaStream_t passed as void* (NULL = legacy default stream).  Work is issued
 *   on that stream; functions that return numbers to the host (norms, stats)
 *   synchronise with the stream before returning.  A plan owns its device
 *   workspaces and its CUDA graphs; one plan must not be used by two host
 *   threads at once.
 *
 * ERRORS
 *   Every function returns SRJ_OK (0) or a negative status.  The text of the
 *   last error of the calling thread is returned by srj_last_error().  After
 *   SRJ_ERR_CUDA the CUDA context may be unusable (sticky errors).
 */
#ifndef SRJ_H
#define SRJ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SRJ_OK                 0
#define SRJ_ERR_INVALID_ARG   -1  /* bad dims, pointer, weight, precision ...           */
#define SRJ_ERR_BAD_SCHEDULE  -2  /* integer scheme does not contract on the grid     */
#define SRJ_ERR_NOT_CONVERGED -3  /* max_cycles reached before tol                   */
#define SRJ_ERR_DIVERGED      -4  /* residual not finite, or grew by more than 1e6x   */
#define SRJ_ERR_TIMEOUT       -5  /* a bounded device-side wait gave up (1 s limit)  */
#define SRJ_ERR_CUDA          -6  /* a CUDA runtime call failed                      */
#define SRJ_ERR_NO_MEMORY     -7  /* device or host allocation failed                */

/* Precision of the sweeps. */
#define SRJ_PREC_FP64   0  /* all arithmetic in FP64; operation order fixed and
                              without fused multiply-add, so that the iterates are
                              reproducible bit for bit                              */
#define SRJ_PREC_MIXED  1  /* FP64 defect correction: each M-cycle runs in FP32 on
                              A e = r (r = b - A u in FP64, e = 0 on the boundary),
                              then u += e in FP64                                   */
#define SRJ_PREC_FP64_FMA 2 /* all arithmetic in FP64, each step as
                              fma(c, fma(-2d, u, sum of neighbours + b), u): 6
                              operations per point instead of 8, iterates within
                              FP64 rounding of SRJ_PREC_FP64's (not bit for bit);
                              residuals as SRJ_PREC_FP64                           */

typedef struct srj_plan *srj_plan_t;

typedef struct srj_stats {
    int64_t cycles;          /* M-cycles applied                                   */
    int64_t sweeps;          /* weighted-Jacobi steps applied (= cycles * M)       */
    int64_t residual_checks; /* residual evaluations, including the initial one   */
    double  r0_l2;           /* ||b - A u0||_2                                     */
    double  res_l2;          /* ||b - A u||_2 at return                            */
    double  res_linf;        /* max_p |b - A u|_p at return                        */
    double  rel_res;         /* res_l2 / r0_l2 (0 if r0_l2 == 0)                   */
    double  sweep_ms;        /* device time of the M-cycle sweep graphs, summed over
                                cycles (CUDA events on `stream`)                   */
    int32_t stagnated;       /* 1 if the solve stopped at the floating-point floor
                                before tol: the residual did not halve in a cycle
                                while within 8 x res_floor, or had not halved its
                                best value for 4 cycles; status NOT_CONVERGED     */
    int32_t reserved;
    double  res_floor;       /* rounding floor of res_l2 at the last cycle end: the
                                unit roundoff 2^-53 times the 2-norm of the sums of
                                the absolute values of each residual entry's terms
                                (single-grid plans; 0 where not computed)         */
} srj_stats_t;

/*
 * srj_plan_create -- build an SRJ plan for one grid and one schedule.
 *   ndim       2 or 3.
 *   dims       interior points per axis, dims[0] = nx (fastest), dims[1] = ny
 *              [, dims[2] = nz]; each in 1..2^30, dims[1] <= 262140 (launch
 *              grid limit), at most 2^36 points in all.  Host pointer, copied.
 *   h          mesh spacing (> 0, finite).
 *   P          number of levels, 1 <= P <= 32.
 *   omega      P weights omega_1..omega_P (Sect. 2; any order, each finite and
 *              > 0).  Host pointer, copied.
 *   q          P repetitions q_i >= 1 per cycle; M = sum q_i <= 2^20.  Host.
 *   order      NULL, or M level indices (0-based, level i appearing exactly q_i
 *              times) giving the order of the steps inside one cycle.  With NULL
 *              the plan picks an order that keeps the running product of the
 *              amplification factors near its straight-line drift (Sect. 5.1
 *              asks only that large over-relaxations be spread out).  Host.
 *   precision  SRJ_PREC_FP64, SRJ_PREC_FP64_FMA or SRJ_PREC_MIXED.
 * The plan checks that the integer scheme contracts on the grid's spectrum,
 * max over kappa in [kappa_min, kappa_max] of |prod_i (1 - omega_i kappa)^q_i| < 1
 * (Sect. 4.3), with kappa_min = (2/d) sum_i sin^2(pi / 2(n_i+1)) and
 * kappa_max = (2/d) sum_i cos^2(pi / 2(n_i+1)) < 2 the extreme eigenvalues of
 * D^-1 A_h, and returns SRJ_ERR_BAD_SCHEDULE otherwise.  It allocates its workspaces on the
 * current device: FP64 plans 3 padded float64 grids, mixed plans 3 padded
 * float32 grids (+ a few KB).
 */
int srj_plan_create(srj_plan_t *plan, int ndim, const int64_t *dims, double h, int P,
                    const double *omega, const int32_t *q, const int32_t *order, int precision);

/* Free a plan and its workspaces (NULL is accepted). */
int srj_plan_destroy(srj_plan_t plan);

/*
 * srj_plan_info -- M, the grid's kappa_min (Sect. 5.1 / Eq. boundaries1D3D:
 * (2/d) sum_i sin^2(pi / 2(n_i+1))) and the largest log10 cycle factor found by
 * the contraction check.  Any output pointer may be NULL.  Host pointers.
 */
int srj_plan_info(srj_plan_t plan, int64_t *M, double *kappa_min, double *log10_cycle_factor_max);

/*
 * srj_plan_set_temporal_depth -- number T of consecutive FP32 steps that one
 * sweep launch applies per HBM round trip (temporal blocking; T = 1 is the
 * plain one-step sweep).  2-D mixed-precision plans: T = 1..8 on register-
 * resident tiles (default 8).  3-D mixed-precision plans: T = 1..3, tiles
 * streamed through z (default 2).  FP64 plans and plans with a mask or shift
 * accept only T = 1.  T blocked steps give the same bits as T single steps.
 * Re-captures the plan's cycle graph.
 */
int srj_plan_set_temporal_depth(srj_plan_t plan, int T);

/*
 * srj_plan_set_sweep_variant -- blocked FP32 sweep strategy of a 2-D mixed plan:
 * 0 = one thread block of 8 warps per 128 x 64 tile; 1 = persistent blocks of
 * 8 warps (2 per SM) that walk the 128 x 64 tiles and prefetch the next tile's
 * rows with bulk copies into shared memory while computing the current one;
 * 2 = one block of 16 warps per 128 x 128 tile (less halo recomputation);
 * 3 = persistent blocks of 16 warps (1 per SM) on 128 x 128 tiles with the same
 * prefetch.  All give the same bits.  Re-captures the cycle graph.  The
 * prefetching variants bound each wait for a prefetch to 1 s of wall time; a
 * wait that runs out ends its block, and the next call that reads the plan's
 * results (srj_solve at a cycle end, srj_steps, srj_plan_autotune) returns
 * SRJ_ERR_TIMEOUT.
 */
int srj_plan_set_sweep_variant(srj_plan_t plan, int variant);

/* srj_plan_sweep_variant -- current sweep variant (host output). */
int srj_plan_sweep_variant(srj_plan_t plan, int *variant);

/* srj_plan_temporal_depth -- current temporal depth (host output). */
int srj_plan_temporal_depth(srj_plan_t plan, int *T);

/*
 * srj_plan_autotune -- time the plan's sweep for every admissible temporal depth
 * and sweep variant (a library service; the paper has no counterpart) on its own workspaces (a few hundred steps each, CUDA
 * events on `stream`), keep the fastest and report it (best_T, microseconds per step; either output
 * may be NULL).  The workspaces' contents are overwritten; srj_solve resets
 * them.  Blocks until done.
 */
int srj_plan_autotune(srj_plan_t plan, void *stream, int *best_T, float *best_us_per_step);

/*
 * srj_plan_set_operator -- replace the plan's operator by
 *   (A u)_p = (2d + sigma) u_p - sum_{neighbours} u_q     on the active points p,
 * the setting of the paper's Grad-Shafranov test B (Sect. 5.3): the SRJ
 * iteration runs only inside a region given by `mask` (device, uint8, padded
 * layout; nonzero = active interior point, 0 = held at its value in u, which
 * then acts as Dirichlet data; NULL = every interior point active), and Eq.
 * GS_linear's linear term appears as a diagonal shift: sigma = -C^2 h^2 for
 * Laplace(u) + C^2 u = rhs (written -Laplace(u) - C^2 u = f), sigma = +k^2 h^2
 * for a screened Poisson operator.  sigma = 0 and mask = NULL restore the plain
 * operator (same bits as before).  The weights are renormalised by the diagonal
 * and the contraction check is redone on the shifted spectrum
 * [(2d kappa_min + sigma)/(2d + sigma), (2d kappa_max + sigma)/(2d + sigma)]
 * (SRJ_ERR_BAD_SCHEDULE if the operator is not positive definite or the scheme
 * does not contract).  The mask is copied.  Residual norms count active points
 * only.  Blocked sweeps implement the plain operator, so a mask or shift sets
 * the temporal depth to 1.  srj_gradient's boundary gradient covers the ghost
 * layer only (not the fixed points of a mask).
 */
int srj_plan_set_operator(srj_plan_t plan, double sigma, const unsigned char *mask, void *stream);

/* srj_plan_order -- copy the M level indices of the cycle order to order_out (host). */
int srj_plan_order(srj_plan_t plan, int32_t *order_out);

/*
 * srj_solve -- run SRJ cycles (Sect. 2: the M = sum q_i weighted-Jacobi steps of
 * Eq. 2nd-order_CD with the Poisson source of Sect. 5.1, in the plan's order)
 * until ||r||_2 / ||r_0||_2 <= tol (checked at cycle ends, the Sect. 4.1 monitor
 * taken on the residual) or max_cycles cycles have run.  Mixed plans run each
 * cycle in FP32 on the defect equation and correct u in FP64 (a library design;
 * the cycle is the same linear map, Sect. 2).
 *   f      device, padded layout, float64 (ghost layer ignored).
 *   u      device, padded layout, float64: on entry the initial guess u0 with
 *          the Dirichlet data in its ghost layer; on return the iterate.
 *   tol    relative tolerance (>= 0).   max_cycles >= 0.
 *   stats  host pointer or NULL.
 * Returns SRJ_OK when converged, SRJ_ERR_NOT_CONVERGED or SRJ_ERR_DIVERGED
 * otherwise (u then holds the last iterate and stats are filled).  The solve
 * also stops with SRJ_ERR_NOT_CONVERGED (stats->stagnated = 1) when 4
 * consecutive cycles fail to halve the smallest residual seen so far: the
 * residual has reached its floating-point floor above tol.  Blocks the host
 * until the solve ends; all device work is on `stream`.
 */
int srj_solve(srj_plan_t plan, const double *f, double *u, double tol, int64_t max_cycles,
              void *stream, srj_stats_t *stats);

/*
 * srj_solve_host -- srj_solve on HOST arrays: f and u (same padded float64
 * layout; pinned memory for full copy bandwidth) are copied to device staging
 * buffers that the plan allocates on the first call and keeps, the solve runs
 * there, and u is copied back (also after SRJ_ERR_NOT_CONVERGED or
 * SRJ_ERR_DIVERGED, as srj_solve leaves its iterate).  Copies and solve are on
 * `stream`; blocks the host until u is back.  SRJ_ERR_NO_MEMORY if the staging
 * buffers cannot be allocated.
 */
int srj_solve_host(srj_plan_t plan, const double *f, double *u, double tol, int64_t max_cycles,
                   void *stream, srj_stats_t *stats);

/*
 * srj_steps -- apply `count` consecutive steps of the cycle order (Sect. 2; each
 * step Eq. 2nd-order_CD with the Sect. 5.1 source), starting at position
 * `first` (mod M), to u in place, without residual checks.  FP64 plans
 * use the FP64 sweep; mixed plans round u and h^2 f to float32, apply the FP32
 * sweep and write the float32 iterate back to u as float64.  Used to compare
 * iterates at equal sweep counts.
 */
int srj_steps(srj_plan_t plan, const double *f, double *u, int64_t first, int64_t count, void *stream);

/*
 * srj_residual -- r = b - A_h u on the interior (FP64), its L2 and max norms
 * (the discrete Poisson operator of Sect. 5.1; the convergence monitor of
 * Sect. 4.1 taken on the residual).
 *   r_out  device padded float64 array or NULL (ghost layer set to 0).
 *   l2, linf  host pointers (may be NULL).
 */
int srj_residual(srj_plan_t plan, const double *f, const double *u, double *r_out,
                 double *l2, double *linf, void *stream);

/*
 * srj_boundary_adjoint -- adjoint of the map from Dirichlet data g to b (the
 * ghost terms of the Sect. 5.1 discretisation; the adjoint is a library feature):
 * for every ghost point q, grad_g[q] = sum of lambda_p over the interior
 * neighbours p of q (b_p = h^2 f_p + sum of ghost neighbours, so dL/dg = B^T
 * dL/db).  lambda and grad_g are device padded float64 arrays; the interior of
 * grad_g is set to 0 and the ghost layer of lambda is ignored.
 */
int srj_boundary_adjoint(srj_plan_t plan, const double *lambda, double *grad_g, void *stream);

/*
 * srj_schedule_check -- host-only contraction check of an integer scheme
 * (Sect. 4.3): *log10_max = max over kappa in [kappa_min, kappa_max] of
 * log10 |prod_i (1 - omega_i kappa)^q_i|; the scheme converges iff < 0.
 * 0 < kappa_min < kappa_max <= 2 (Eq. boundaries: kappa_M = 2 bounds every
 * grid).  Host pointers.  Needs no GPU.
 */
int srj_schedule_check(int P, const double *omega, const int32_t *q, double kappa_min, double kappa_max,
                       double *log10_max);

/*
 * srj_schedule_order -- host-only: the cycle order srj_plan_create uses when
 * its `order` argument is NULL (M = sum q_i level indices written to
 * order_out): the drift order (running log-products kept near their straight
 * line), ending with copies of the smallest weight, as many as minimise a model
 * of the FP32 rounding noise of one cycle.  Needs no GPU.
 */
int srj_schedule_order(int P, const double *omega, const int32_t *q, double kappa_min, int32_t *order_out);

/*
 * Batched solver: many independent 2-D problems, each with its own size and
 * SRJ schedule, solved together in mixed precision (FP32 M-cycles on the defect
 * equation inside FP64 correction, as SRJ_PREC_MIXED).  One phase advances every
 * unfinished problem by up to T steps of its own cycle order in one blocked
 * sweep launch over the tiles of the unfinished problems, then updates, checks
 * the residual of and restarts the problems whose cycle ended.  A CUDA graph of
 * several phases is replayed until every problem has converged, failed, or run
 * max_cycles cycles; between replays its launches are narrowed to the problems
 * still iterating.  Batches with at most 16 distinct grid sizes and at most 1024
 * problems use a faster sweep whose blocks locate their tiles from the launch
 * parameters; the results are the same bit for bit either way, and equal those
 * of single mixed-precision plans with the same temporal depth.  The paper's
 * method per problem is Sect. 2 / 3.1 / 5.1; the batching is this library's.
 */
typedef struct srj_batch *srj_batch_t;

typedef struct srj_batch_problem {
    int64_t nx, ny;        /* interior points (1..65536 each)                      */
    double h;              /* mesh spacing                                          */
    int32_t P;             /* levels                                                */
    const double *omega;   /* host, P weights                                       */
    const int32_t *q;      /* host, P repetitions                                   */
    const int32_t *order;  /* host, M level indices, or NULL for the drift order   */
} srj_batch_problem_t;

/* Build a batch (copies every schedule; allocates 3 pitched float32 grids per
 * problem).  temporal_depth: steps per sweep launch, 1..8, 0 = 8.  Each
 * problem's integer scheme must contract on its grid (SRJ_ERR_BAD_SCHEDULE). */
int srj_batch_create(srj_batch_t *batch, int nprob, const srj_batch_problem_t *problems, int temporal_depth);

int srj_batch_destroy(srj_batch_t batch);

/*
 * srj_batch_tune_depth -- temporal depth for a batch of these problems (a
 * library service; the paper has no counterpart): for T = tmax down to tmin it
 * builds the batch with depth T and times one cycle of every problem (each
 * solve started from copies of u, so f and u, device arrays as for
 * srj_batch_solve, are left unchanged; the copies are allocated and freed
 * here), keeping the depth with the shortest device time.  best_T: host
 * output; best_ms_per_cycle: host, may be NULL.  Blocks the host.
 */
int srj_batch_tune_depth(int nprob, const srj_batch_problem_t *problems, const double *const *f,
                         const double *const *u, int tmin, int tmax, void *stream, int *best_T,
                         double *best_ms_per_cycle);

/* Sizes of a batch (host outputs, each may be NULL). */
int srj_batch_info(srj_batch_t batch, int64_t *total_points, int64_t *tiles, int *temporal_depth, int64_t *sum_M);

/*
 * srj_batch_solve -- f, u: HOST arrays of nprob DEVICE pointers, each a padded
 * float64 grid of its problem (layout of srj_solve; u: initial guess with the
 * Dirichlet data in its ghost layer, overwritten by the iterate).  stats: host
 * array of nprob entries or NULL (sweep_ms = device time of the whole batch).
 * device_ms: host, may be NULL.  Returns SRJ_OK when every problem reached
 * ||r||_2 / ||r_0||_2 <= tol, else the first failing status.  Blocks the host.
 */
int srj_batch_solve(srj_batch_t batch, const double *const *f, double *const *u, double tol, int64_t max_cycles,
                    void *stream, srj_stats_t *stats, double *device_ms);

/* Text of the last batch error on the calling thread. */
const char *srj_batch_last_error(void);

/*
 * srj_gradient -- backward pass of u = S(f, g), the solution of A_h u = h^2 f + B g
 * (B: ghost neighbours; the discretisation of Sect. 5.1, whose A_h is
 * symmetric), for a scalar loss L(u).  The adjoint is a library feature.  Given grad_u = dL/du (device,
 * padded; its ghost layer is dL/dg through u's own ghost layer, which equals g):
 *   lambda solves A_h lambda = grad_u on the interior (A_h is symmetric, so the
 *   adjoint solve is the same SRJ solve) with lambda = 0 on the ghost layer;
 *   grad_f = h^2 lambda on the interior (0 on the ghosts);
 *   grad_g = B^T lambda + grad_u on the ghost layer (0 inside), B^T lambda being
 *   the sum of lambda over each ghost point's interior neighbours.
 * lambda is in/out: its interior is the initial guess (0 is fine), its ghost
 * layer is set to 0.  The solve uses the plan's schedule and precision, runs to
 * tol / max_cycles like srj_solve and fills stats.  Returns the solve's status
 * (outputs are written for SRJ_OK and SRJ_ERR_NOT_CONVERGED).
 */
int srj_gradient(srj_plan_t plan, const double *grad_u, double *lambda, double *grad_f, double *grad_g, double tol,
                 int64_t max_cycles, void *stream, srj_stats_t *stats);

/*
 * srj_schedule_optimal -- host-only optimal SRJ parameters (Sect. 3): for P levels
 * (1..32) and the spectral bound kappa_min in (0, 1), the weights omega[P]
 * (decreasing), fractions beta[P] (sum 1) and, if kappa_int is not NULL, the P-1
 * interior maxima of Gamma, minimising max over [kappa_min, 2] of
 * Gamma(kappa) = prod_i |1 - omega_i kappa|^beta_i (Eq. Gamma).  The reduced system
 * S(omega, kappa) of Sect. 3.5 (beta from Theorem 2, equal maxima, optimality in
 * Lagrange-multiplier form) is solved by Levenberg-Marquardt, level by level with the
 * initial guesses of Sect. 3.3.  Returns SRJ_ERR_BAD_SCHEDULE if no solution is
 * found (large P at small resolution, as the paper reports).  Needs no GPU.
 */
int srj_schedule_optimal(int P, double kappa_min, double *omega, double *beta, double *kappa_int);

/*
 * srj_schedule_for_grid -- host-only: optimal weights at the grid's kappa_min and
 * integer repetitions q_i = floor(beta_i / beta_1) (Sect. 4.3); checks that the
 * integer scheme contracts on the grid (SRJ_ERR_BAD_SCHEDULE otherwise).  Outputs
 * omega[P], q[P] and M = sum q (M_out may be NULL).  Needs no GPU.
 */
int srj_schedule_for_grid(int ndim, const int64_t *dims, int P, double *omega, int32_t *q, int64_t *M_out);

/* kappa_min of a Dirichlet grid with `ndim` axes of dims[i] interior points (host):
 * (2/d) sum_i sin^2(pi / 2(n_i + 1)), Sect. 5.1 with the normalisation of
 * Eq. boundaries1D3D. */
int srj_kappa_min(int ndim, const int64_t *dims, double *kappa_min);

/* Spectral range of the Jacobi-normalised Dirichlet operator D^-1 A of a grid
 * (host): kappa_min as above and kappa_max = (2/d) sum_i cos^2(pi / 2(n_i + 1)),
 * the exact extremes of its eigenvalues (2/d) sum_i sin^2(m_i pi / 2(n_i + 1)),
 * m_i = 1..n_i (Sect. 5.1 / Eq. boundaries1D3D; the schedules themselves are
 * optimised on [kappa_min, 2], Eq. boundaries).  Either output may be NULL. */
int srj_kappa_range(int ndim, const int64_t *dims, double *kappa_min, double *kappa_max);

/* Effective Neumann resolution of a Dirichlet grid (host), Eq.
 * effectiveNDirichlet: N_eff = pi / (2 asin(sqrt((2/d) sum_i sin^2(pi / 2N_i)))),
 * N_i = n_i + 1 zones for n_i interior points -- the N of the paper's tables
 * (computed for the Neumann model problem) whose schedule suits this grid. */
int srj_neff(int ndim, const int64_t *dims, double *n_eff);

/*
 * srj_steps_f32_noalloc -- the FP32 sweep of srj_steps without any device
 * allocation.  (The paper has no counterpart: this is a library service.)
 *
 * For callers that cannot allocate device memory when they need a few sweeps:
 * code whose device memory is all owned by its own fixed pool, and
 * latency-critical loops in which cudaMalloc / cudaFree would synchronise the
 * device.  Instead of a plan's workspaces the
 * work buffers live in one static device array of 12 MiB (3 x 2^20 floats) that
 * every GPU loading this library holds until the process exits; grids whose
 * pitched float32 layout needs more than 2^20 floats per buffer (about 1M padded
 * points, e.g. 1016 x 1016 or 96^3) are rejected with SRJ_ERR_INVALID_ARG.
 *
 * Applies `count` FP32 weighted-Jacobi steps with weights omega_seq[0..count-1]
 * (host array) to u in place, exactly as srj_steps does on a mixed-precision plan
 * whose cycle order gives the same weights: u and h^2 f are rounded to float32,
 * the sweeps run in float32, the interior of u is written back as float64 and its
 * ghost layer is left untouched.  f, u: device arrays in the padded layout.
 * Blocks until the work on `stream` is done.
 *
 * The first call in a device's CUDA context looks up the array's device address
 * (cudaGetSymbolAddress, which allocates nothing); a call after that context
 * was replaced (cudaDeviceReset, then a new context) looks it up again.  No call
 * allocates or frees device memory.  All calls share the array, which keeps the
 * last call's contents (each call clears what it reads); calls whose GPU work
 * overlaps race on it.  Errors are reported through srj_noalloc_last_error().
 */
int srj_steps_f32_noalloc(int ndim, const int64_t *dims, double h, int64_t count, const double *omega_seq,
                          const double *f, double *u, void *stream);

/* Text of the last error of srj_steps_f32_noalloc on the calling thread. */
const char *srj_noalloc_last_error(void);

/*
 * srj_selftest_wait_timeout -- self-test of the bounded device-side waits (a
 * library service; the paper has no counterpart).  Launches the prefetching
 * sweep (variant 1) on an internal 64 x 64 grid in a mode that issues no
 * prefetch copy, so every block's wait on its staging barrier runs out after
 * limit_us microseconds (1 .. 1e6) of wall time; each block then records the
 * timeout in a device status word and returns, leaving the CUDA context usable.
 * Allocates and frees its own small device buffers; blocks until done.
 * Returns SRJ_ERR_TIMEOUT when the waits ran out and were reported, as
 * designed; SRJ_OK would mean that no wait ran out (a failed self-test).
 */
int srj_selftest_wait_timeout(int64_t limit_us, void *stream);

/* Text of the last error on the calling thread ("" if none). */
const char *srj_last_error(void);

/* Library version string. */
const char *srj_version(void);

/* ---------------------------------------------------------------------------
 * Spherical-coordinate operators (Sect. 5.2), FP64
 *
 * Grid: dims[0] = n_r radial points (fastest), dims[1] = n_theta polar points
 * [, dims[2] = n_phi azimuthal points], cell centred on r in [0, 1], theta in
 * [0, pi], phi in [0, 2 pi]: r_i = (i - 1/2) / n_r etc.  Arrays are padded
 * float64 grids in the layout of srj_solve (one ghost layer per side).
 * Operator: the Poisson operator in spherical coordinates multiplied by r^2,
 * with separable coefficients (each array in padded index order):
 *   (L u)_p = cr_m[i] u(i-1) + cr_p[i] u(i+1) + ct_m[j] u(j-1) + ct_p[j] u(j+1)
 *             [+ cp[j] (u(k-1) + u(k+1))] - d_p u_p,
 *   d_p = cr_0[i] + ct_0[j] [+ 2 cp[j]];   radial = cr_m | cr_p | cr_0
 *   (3 (n_r + 2) doubles), polar = ct_m | ct_p | ct_0 (3 (n_theta + 2)),
 *   azim = cp (n_theta + 2; 3-D only).
 * System L u = b (b = r^2 s).  Boundary prescriptions, applied at every step:
 * the r = 1 ghost layer of u holds Dirichlet data; u_0 = u_1 = u_2 at r = 0 (the
 * row i = 1 copies row 2, which is iterated with u(i-1) = u(i)); Neumann mirrors
 * at theta = 0, pi; periodic in phi.  The active points are i = 2..n_r.
 * Step (Sect. 3.1 with diagonal -d): u' = u + omega ((L u - b) / d).
 * ------------------------------------------------------------------------- */
typedef struct srj_sph_plan *srj_sph_plan_t;

/* Host helper: the Sect. 5.2 coefficients for dims (central differences of
 * r^2 u_rr + 2 r u_r + u_tt + cot(t) u_t [+ u_pp / sin^2 t]):
 *   cr_m = r (r - dr) / dr^2, cr_p = r (r + dr) / dr^2, cr_0 = 2 r^2 / dr^2,
 *   ct_m = 1/dt^2 - cot(t) / (2 dt), ct_p = 1/dt^2 + cot(t) / (2 dt),
 *   ct_0 = 2 / dt^2, cp = 1 / (sin^2(t) dp^2) (polar / azimuthal ghosts 0).
 * Outputs are host arrays of the sizes above (azim may be NULL in 2-D). */
int srj_sph_coefficients(int ndim, const int64_t *dims, double *radial, double *polar, double *azim);

/* Build a plan: dims and coefficient arrays (host, copied; finite); the
 * schedule as in srj_plan_create (order NULL: drift order); precision
 * SRJ_PREC_FP64 (every step in FP64) or SRJ_PREC_MIXED (each cycle runs in FP32
 * on the defect equation L e = b - L u with e = 0 at the start and on the
 * boundary, FP64 residual and update: the same cycle map up to FP32 rounding
 * of the correction).  The integer scheme
 * must contract on [1 / max omega, 2) (SRJ_ERR_BAD_SCHEDULE); the Jacobi-scaled
 * operator's spectrum lies in (0, 2) for weakly diagonally dominant, irreducible
 * rows with strict dominance next to the Dirichlet boundary, which the Sect. 5.2
 * coefficients give. */
int srj_sph_plan_create(srj_sph_plan_t *plan, int ndim, const int64_t *dims, const double *radial,
                        const double *polar, const double *azim, int P, const double *omega, const int32_t *q,
                        const int32_t *order, int precision);
int srj_sph_plan_destroy(srj_sph_plan_t plan);

/* count FP64 steps of the cycle order from position first (either precision):
 * the weighted-Jacobi step of Sect. 3.1 on the Sect. 5.2 operator, with the
 * r = 0 and theta prescriptions applied at every step.  u (device, in place);
 * writes the active points and row i = 1, leaves the other ghosts as given. */
int srj_sph_steps(srj_sph_plan_t plan, const double *b, double *u, int64_t first, int64_t count, void *stream);

/* l2 / linf (host outputs) of res = L u - b (the Sect. 5.2 operator) over the
 * active points; r_out
 * (device, may be NULL) gets res there and 0 elsewhere.  Blocks the host. */
int srj_sph_residual(srj_sph_plan_t plan, const double *b, const double *u, double *r_out, double *l2,
                     double *linf, void *stream);

/* SRJ cycles (Sect. 2) on the Sect. 5.2 operator until ||res||_2 / ||res_0||_2
 * <= tol (or max_cycles, divergence, or a stalled residual: stats->stagnated),
 * then the ghost layer and row i = 1 are set from the prescriptions.  b, u:
 * device; u in place.  Blocks the host. */
int srj_sph_solve(srj_sph_plan_t plan, const double *b, double *u, double tol, int64_t max_cycles, void *stream,
                  srj_stats_t *stats);

/* Set the ghost layer and row i = 1 of u (device) from the prescriptions of
 * Sect. 5.2 (u_0 = u_1 = u_2 at r = 0, theta mirrors, periodic phi). */
int srj_sph_finalize(srj_sph_plan_t plan, double *u, void *stream);

/* FP32 steps per launch of a mixed 2-D spherical plan (1..8; default 8 when
 * n_r >= 2): T steps on register-resident tiles give the bits of T single
 * steps.  Other plans accept only T = 1.  Re-captures the cycle graph. */
int srj_sph_plan_set_temporal_depth(srj_sph_plan_t plan, int T);
int srj_sph_plan_temporal_depth(srj_sph_plan_t plan, int *T);

#ifdef __cplusplus
}
#endif

#endif /* SRJ_H */
