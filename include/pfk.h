/*
 * pfk.h -- C ABI of the GB300 pipelined flexible Krylov library.
 *
 * The library solves A x = b with the flexible Krylov methods of Sanan,
 * Schnepp and May, "Pipelined, Flexible Krylov Subspace Methods"
 * (arXiv 1511.07226): the problem statement is the one of Alg. 2 (FCG(A, B,
 * b, x0)) and Alg. 13 (FGMRES(A, B, b, x0, m)): an operator A, a possibly
 * nonlinear preconditioner B, a right-hand side b, an initial guess x0, a
 * relative tolerance and the truncation length nu_max (CG/CR types) or the
 * restart length m (GMRES types), Sec. 5 "Implementation".
 *
 * Every step of a solve runs in the library's CUDA kernels for sm_103a on one
 * GPU; there is no CPU fallback.  A call that needs the GPU and cannot get it
 * returns PFK_ERR_CUDA.
 *
 * Conventions (all entry points):
 *  - Every function returns a pfk_status; no C++ exception crosses the ABI.
 *  - Handles are opaque, created by pfk_create_* and owned by the library
 *    until the matching pfk_destroy_*; destroying NULL is a no-op.
 *  - Array arguments are borrowed for the duration of the call only; the
 *    library copies what it keeps.
 *  - "device pointer" means memory of the context's GPU (cudaMalloc, the
 *    PyTorch caching allocator, ...); "host pointer" means ordinary host
 *    memory.  Functions that take both say which via an explicit flag.
 *  - All device work is ordered on the context's CUDA stream.  Calls return
 *    after that work is complete unless stated otherwise.
 *  - A context is used by one host thread at a time.  pfk_last_error() holds
 *    the message of the last failing call on that context (or, for a NULL
 *    context, on the calling thread).
 *  - Vectors are FP64, length n, in the cell order index = i + nx (j + ny k).
 */
#ifndef PFK_H_
#define PFK_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PFK_ABI_VERSION 1
#define PFK_MAX_MMAX 32        /* largest nu_max / restart length m */
#define PFK_HISTORY_FIELDS 4   /* per iteration: rho, ||r||_2 (recurred), eta, alpha */
#define PFK_PERSISTENT_MAX_N 16384   /* largest system of the persistent single-launch path */

typedef enum {
  PFK_OK = 0,
  PFK_PENDING = 1,
  PFK_ERR_INVALID = -1,       /* bad argument; nothing was done */
  PFK_ERR_OOM = -2,           /* device allocation failed */
  PFK_ERR_CUDA = -3,          /* a CUDA call failed; the message has the CUDA error */
  PFK_ERR_BREAKDOWN = -4,     /* norm breakdown that restarting could not cure (Sec. 5) */
  PFK_ERR_NOT_CONVERGED = -5, /* maxit reached, or the true residual stayed above the goal after
                                 max_restarts residual replacements; x holds the last iterate */
  PFK_ERR_TIMEOUT = -6,       /* a bounded device or host wait gave up */
  PFK_ERR_CANCELLED = -7,
  PFK_ERR_BUSY = -8           /* server queue full */
} pfk_status;

typedef enum {
  PFK_STENCIL5_2D = 0,  /* -div(eta grad u) on nx x ny cells (nz = 1) */
  PFK_STENCIL7_3D = 1,  /* -div(eta grad u) on nx x ny x nz cells */
  PFK_CSR = 2           /* general sparse matrix in CSR form */
} pfk_op_kind;

typedef enum {
  PFK_STORAGE_MATRIX_FREE = 0, /* stencils: face coefficients + diagonal, applied on the fly */
  PFK_STORAGE_CSR = 1          /* stencils: assembled by the library into FP64 CSR */
} pfk_op_storage;

typedef enum {
  PFK_FCG = 0,          /* Alg. 2 */
  PFK_PIPEFCG = 1,      /* Alg. 8 */
  PFK_GCR = 2,          /* Alg. 9 */
  PFK_PIPEGCR = 3,      /* Alg. 11 */
  PFK_FGMRES = 4,       /* Alg. 13 */
  PFK_PIPEFGMRES = 5,   /* Alg. 15 */
  PFK_PIPEFCG_NAIVE = 6, /* Alg. 7 */
  PFK_PIPEGCR_W = 7,     /* Alg. 12: w recurred (w_i = w_{i-1} - alpha z_{i-1}), z history */
  PFK_PIPEFCG_THETA = 8  /* Alg. 8 with the projection repair of eq. (proj):
                            m_i = theta_i u_i + B(w_i - theta_i r_i), theta_i = <r_i, w_i>/<r_i, r_i> */
} pfk_method;

typedef enum {
  PFK_PC_NONE = 0,       /* B(v) = v */
  PFK_PC_JACOBI = 1,     /* B(v) = D^-1 v */
  PFK_PC_INNER_PCG = 2,  /* inner_iters iterations of Jacobi-PCG (Alg. 3, M^-1 = D^-1) from 0 */
  PFK_PC_CHEBYSHEV = 3,  /* inner_iters Chebyshev-Jacobi sweeps from 0 */
  PFK_PC_NOISY = 4,      /* B(r) = r + eta ||r|| xi_j / ||xi_j|| (pfk_create_noisy_preconditioner) */
  PFK_PC_BLOCK_UPPER = 5 /* nested block upper-triangular (pfk_create_block_preconditioner) */
} pfk_pc_kind;

typedef enum {
  PFK_FP64 = 0,          /* preconditioner arithmetic and storage in FP64 */
  PFK_FP32 = 1,          /* FP32 vectors and coefficient copies, FP64 dot combination */
  PFK_BF16_COEF_FP32 = 2 /* BF16-stored coefficients, FP32 vectors and accumulation */
} pfk_precision;

typedef enum { PFK_TRUNC_STANDARD = 0, PFK_TRUNC_RESTART = 1 } pfk_truncation;
typedef enum { PFK_NORM_NATURAL = 0, PFK_NORM_UNPRECONDITIONED = 1 } pfk_norm;

typedef struct pfk_context pfk_context;
typedef struct pfk_operator pfk_operator;
typedef struct pfk_pc pfk_pc;

/* ------------------------------------------------------------------------ */
/* Context                                                                   */
/* ------------------------------------------------------------------------ */

/* Creates a context on CUDA device `device` whose work is ordered on
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).  The
 * stream stays owned by the caller and must outlive the context.
 * Errors: PFK_ERR_INVALID (ctx NULL or bad device), PFK_ERR_CUDA. */
pfk_status pfk_create_context(int device, void* cuda_stream, pfk_context** ctx);
pfk_status pfk_destroy_context(pfk_context* ctx);

/* Message of the last failing call on ctx (ctx may be NULL: calling thread). */
const char* pfk_last_error(const pfk_context* ctx);

/* ABI version (PFK_ABI_VERSION) of the loaded library. */
int pfk_abi_version(void);

/* ------------------------------------------------------------------------ */
/* Operators                                                                 */
/* ------------------------------------------------------------------------ */

/* Stencil kinds: cell-centred finite volumes for -div(eta grad u) on the unit
 * square/cube with homogeneous Dirichlet boundaries, scaled so that
 *   (A u)_i = sum over faces f of cell i of K_f (u_i - u_nbr),
 *   K_f = 2 eta_i eta_j / (eta_i + eta_j) on interior faces, 2 eta_i with
 *   u_nbr = 0 on boundary faces,
 * plus, if vel != 0, first-order upwind advection h |v_d| (u_i - u_up) per
 * direction (h = 1/nx; upwind ghost outside the domain = 0).  This is the
 * n_z = 7 (3D) sparse operator of the paper's performance model (Sec. 8).
 * The right-hand side the caller passes is then h^2 f.
 *
 * CSR kind: n rows, nnz entries, int32 row pointers (n+1) and column indices,
 * FP64 values; columns need not be sorted.
 *
 * Ownership: eta / rowptr / colidx / vals are read during the call only; their
 * location is given by eta_on_device / csr_on_device (0 = host, 1 = device).
 * Errors: PFK_ERR_INVALID (sizes <= 0, nz != 1 for 2D, eta <= 0 is not checked
 * on device data), PFK_ERR_OOM, PFK_ERR_CUDA. */
typedef struct {
  int32_t kind;        /* pfk_op_kind */
  int32_t storage;     /* pfk_op_storage (stencils only) */
  int32_t nx, ny, nz;  /* stencils */
  const double* eta;   /* stencils: nx*ny*nz cell viscosities, > 0 */
  int32_t eta_on_device;
  double vel[3];       /* stencils: constant advection velocity (0 = none) */
  int64_t n, nnz;      /* CSR */
  const int32_t* rowptr;
  const int32_t* colidx;
  const double* vals;
  int32_t csr_on_device;
} pfk_operator_desc;

pfk_status pfk_create_operator(pfk_context* ctx, const pfk_operator_desc* desc, pfk_operator** op);
pfk_status pfk_destroy_operator(pfk_operator* op);
/* Number of rows n of the operator. */
pfk_status pfk_operator_size(const pfk_operator* op, int64_t* n);
/* y = A x; x and y are device pointers of length n, must not overlap. */
pfk_status pfk_operator_apply(pfk_context* ctx, const pfk_operator* op, const double* x, double* y);

/* ------------------------------------------------------------------------ */
/* Preconditioners                                                           */
/* ------------------------------------------------------------------------ */

/* The preconditioner B of the flexible methods (Sec. 2): any map v -> B(v);
 * the inner iterative ones are nonlinear in v.
 *  - JACOBI: B(v) = D^-1 v, D = diag(A).
 *  - INNER_PCG: `inner_iters` iterations of Alg. 3 with M^-1 = D^-1 on A y = v
 *    from y = 0, no tolerance test; the experiments of Sec. 6 use 5 such
 *    iterations per block.  If <D^-1 r, r> or <s, p> becomes exactly 0 the
 *    current iterate is returned.
 *  - CHEBYSHEV: `inner_iters` Chebyshev sweeps on D^-1 A over [cheb_lo,
 *    cheb_hi] from 0 (Saad, Iterative Methods for Sparse Linear Systems, 2nd
 *    ed., Alg. 12.1).  cheb_lo = cheb_hi = 0 selects [0.1 L, 1.1 L] with L the
 *    Gershgorin bound max_i sum_j |a_ij| / a_ii.
 *  - precision: PFK_FP64, PFK_FP32 (INNER_PCG, CHEBYSHEV) or
 *    PFK_BF16_COEF_FP32 (CHEBYSHEV): the preconditioner's copy of A stores the
 *    diagonal, the face coefficients and D^-1 rounded FP64 -> FP32 (-> BF16,
 *    nearest-even); its vectors are FP32; the outer method stays FP64.
 * Stencil operators support every kind; CSR operators support NONE and JACOBI.
 * The preconditioner keeps a reference to `op`, which must outlive it. */
typedef struct {
  int32_t kind;        /* pfk_pc_kind */
  int32_t inner_iters;
  int32_t precision;   /* pfk_precision */
  double cheb_lo, cheb_hi;
} pfk_pc_desc;

pfk_status pfk_create_preconditioner(pfk_context* ctx, const pfk_operator* op, const pfk_pc_desc* desc,
                                     pfk_pc** pc);
/* The preconditioner of the paper's toy experiment (Sec. 3.2, Fig. FCGtoy):
 * B(r) = r + eta ||r||_2 xi_j / ||xi_j||_2, where xi_j is row (j mod count) of
 * `bank` (count x n doubles, row-major; host or device per bank_on_device; copied
 * at creation) and j counts this preconditioner's applications since its
 * creation (j = 0 first).  The noise is an input, so a CPU reference drawing the
 * same rows reproduces the sequence.  Works with any operator.  Errors:
 * PFK_ERR_INVALID (eta < 0, count < 1, a zero bank row), PFK_ERR_OOM, PFK_ERR_CUDA. */
pfk_status pfk_create_noisy_preconditioner(pfk_context* ctx, const pfk_operator* op, double eta, const double* bank,
                                           int count, int bank_on_device, pfk_pc** pc);
/* Inner solve of a nested preconditioner: a CG- or CR-type method (PFK_FCG,
 * PFK_PIPEFCG, PFK_PIPEFCG_THETA, PFK_GCR, PFK_PIPEGCR, PFK_PIPEGCR_W) with a
 * Jacobi preconditioner, from a zero guess, stopping when its natural norm
 * falls below rtol times the initial one, at maxit iterations, or at a norm
 * breakdown (no restarts, no true-residual check). */
typedef struct {
  int32_t method;
  int32_t mmax;     /* 1..PFK_MAX_MMAX, standard truncation */
  double rtol;
  int32_t maxit;    /* >= 1; each application records this many iterations */
  int32_t pad;
} pfk_inner_solve;

/* The block upper-triangular preconditioner of the paper's Stokes experiment
 * (Sec. 6, ex43): for v = (v_u, v_p) with nu = K's size and N = Bt's size,
 *   y_p = S_hat^-1 v_p,   y_u = K_hat^-1 (v_u - B^T y_p),
 * S_hat = diag(schur_diag) (host, N - nu entries, finite and non-zero; copied),
 * K_hat^-1 one inner solve (`inner`) of K y_u = t.  Bt is an N x N operator
 * holding B^T in its first nu rows (zero rows for the pressure block).  K and
 * Bt must outlive the preconditioner.  Nonlinear through the inner solve: use
 * it with a flexible outer method (e.g. PFK_FGMRES, PFK_PIPEFGMRES).  An
 * application is a fixed sequence of device launches, so outer solves record it
 * in their CUDA graphs.  Errors: PFK_ERR_INVALID, PFK_ERR_OOM, PFK_ERR_CUDA. */
pfk_status pfk_create_block_preconditioner(pfk_context* ctx, const pfk_operator* K, const pfk_operator* Bt,
                                           const double* schur_diag, const pfk_inner_solve* inner, pfk_pc** pc);
pfk_status pfk_destroy_preconditioner(pfk_pc* pc);
/* y = B(v); device pointers of length n, must not overlap. */
pfk_status pfk_pc_apply(pfk_context* ctx, const pfk_pc* pc, const double* v, double* y);

/* ------------------------------------------------------------------------ */
/* Solve                                                                     */
/* ------------------------------------------------------------------------ */

/* Solve parameters.
 *  method      pfk_method.
 *  mmax        nu_max (FCG/PIPEFCG/GCR/PIPEGCR) or restart length m
 *              (FGMRES/PIPEFGMRES); 1 <= mmax <= PFK_MAX_MMAX.
 *  truncation  STANDARD: nu_i = min(i, nu_max); RESTART: nu_i =
 *              ((i-1) mod nu_max) + 1, i counted since the last (re)start
 *              ("Truncation strategies", Sec. 5).
 *  norm        NATURAL: sqrt|gamma_i| (CG/CR types; the only norm free of
 *              extra reductions, Sec. 5); UNPRECONDITIONED: recurred ||r_i||_2.
 *              GMRES types always use the least-squares residual estimate.
 *  rtol, atol  converged when rho_i <= max(rtol rho_0, atol), rho_0 from the
 *              first pipeline fill.
 *  maxit       iteration limit (all restarts together).
 *  max_restarts  bound on breakdown restarts plus residual replacements.
 *  sigma       constant shift of PIPEFGMRES (Sec. 5.3); NaN = estimate it by
 *              10 power iterations on v -> A B(v).
 *  true_residual_check  1: at convergence require ||b - A x||_2 <= rtol ||b||_2
 *              (else restart from x with the target tightened by
 *              0.5 rtol ||b|| / ||b - A x||); 0: accept the recurred norm.
 *  graph_iters iterations per captured CUDA graph launch (0 = default 8).
 *  history     optional HOST buffer of history_capacity * PFK_HISTORY_FIELDS
 *              doubles; entry e = (rho, ||r||_2 recurred or NaN, eta, alpha)
 *              for each pipeline fill and each iteration, in order.
 *  profile     1: record CUDA events around the method's fused recurrence
 *              pass in every iteration (the graphs then carry event nodes and
 *              one graph launch is in flight instead of two) and report the
 *              pass's total device time in pfk_solve_info.pass_ms.
 *  persistent  small systems (n <= PFK_PERSISTENT_MAX_N, assembled CSR
 *              operator, Jacobi or no preconditioner, PIPEFCG or FCG): run
 *              many iterations per cooperative launch, the blocks meeting at
 *              bounded grid barriers (one per PIPEFCG iteration, three per FCG
 *              iteration) instead of kernel boundaries.  0 (default): when
 *              eligible; 1: never; 2: required (PFK_ERR_INVALID when not
 *              eligible).  A barrier wait that gives up (barrier_timeout_us)
 *              ends the solve with PFK_ERR_TIMEOUT.
 *  barrier_timeout_us  bound of each grid-barrier wait of the persistent
 *              path: 0 = 2 s; > 0 = that many microseconds; < 0 = no wait
 *              allowed (a barrier that has to wait fails at once: the solve
 *              ends with PFK_ERR_TIMEOUT and the context stays usable -- for
 *              testing the time-out path). */
typedef struct {
  int32_t method;
  int32_t mmax;
  int32_t truncation;
  int32_t norm;
  double rtol;
  double atol;
  int32_t maxit;
  int32_t max_restarts;
  double sigma;
  int32_t true_residual_check;
  int32_t graph_iters;
  double* history;
  int32_t history_capacity;
  int32_t profile;
  int32_t persistent;
  int32_t barrier_timeout_us;
} pfk_solve_params;

typedef struct {
  int32_t status;       /* pfk_status of the solve */
  int32_t iterations;
  int32_t restarts;     /* breakdown restarts + residual replacements */
  int32_t breakdowns;
  int32_t replacements;
  int32_t history_len;  /* entries written (may exceed capacity: then truncated) */
  double rho0, rho_final;
  double rnorm_true;    /* ||b - A x||_2 at exit */
  double bnorm;         /* ||b||_2 */
  double time_ms;       /* device time of the solve, CUDA events on the stream */
  /* Accounting of the fused recurrence pass (the dominant kernel), over the
   * passes that did work: launches, algorithmic HBM bytes (each vector read or
   * written once per pass) and FP64 flops (FMA = 2), and, with profile = 1,
   * the summed device time of those passes. */
  int32_t pass_launches;
  int32_t kernel_launches;  /* all library kernels launched by the solve */
  double pass_bytes;
  double pass_flops;
  double pass_ms;
} pfk_solve_info;

/* Fills `params` with the defaults: PIPEFCG, mmax 30, standard truncation,
 * natural norm, rtol 1e-8, atol 0, maxit 10000, max_restarts 20, sigma NaN,
 * true_residual_check 1, graph_iters 8, no history. */
pfk_status pfk_default_params(pfk_solve_params* params);

/* Solves A x = b.  b and x are host pointers (ptr_on_device = 0) or device
 * pointers (1), length n; x holds x0 on entry and the solution on exit (also
 * on PFK_ERR_NOT_CONVERGED and PFK_ERR_BREAKDOWN, where it is the last
 * iterate).  `pc` may be NULL (= PFK_PC_NONE).  info may be NULL.
 * Returns PFK_OK on convergence, PFK_ERR_NOT_CONVERGED at maxit,
 * PFK_ERR_BREAKDOWN (Sec. 5: breakdown in a fill or right after a breakdown
 * restart, or restarts exhausted), PFK_ERR_INVALID, PFK_ERR_OOM, PFK_ERR_CUDA. */
pfk_status pfk_solve(pfk_context* ctx, const pfk_operator* op, const pfk_pc* pc, const pfk_solve_params* params,
                     const double* b, double* x, int ptr_on_device, pfk_solve_info* info);

/* Number of length-n vectors the paper counts for a method's storage:
 * PIPEFCG 4 nu+11, FCG nu+6 (Sec. 3.2.3); GCR 2 nu+7, PIPEGCR 3 nu+9 (Sec. 4);
 * FGMRES 2m+2, PIPEFGMRES 4m+2 (Sec. 5.3).  Returns -1 for a bad method. */
int pfk_method_storage_vectors(int method, int mmax);

/* Device bytes pfk_solve allocates for one solve of size n (vectors, rings,
 * partial sums, control block; excludes the preconditioner's own scratch,
 * reported by pfk_pc_workspace_bytes). */
pfk_status pfk_solve_workspace_bytes(int method, int mmax, int64_t n, int64_t* bytes);
pfk_status pfk_pc_workspace_bytes(const pfk_pc* pc, int64_t* bytes);

/* ------------------------------------------------------------------------ */
/* Batched solve: many independent systems in one persistent launch          */
/* ------------------------------------------------------------------------ */

/* Solves nsys independent systems A_j x_j = b_j with PIPEFCG (Alg. 8) in one
 * persistent kernel launch: each thread block takes the next system from a
 * work counter (largest first) and runs that system's whole solve - fill,
 * iterations, restarts, true-residual check - with block-level reductions, so
 * no block ever waits for another.  A system's result does not depend on the
 * other systems of the batch (bit for bit).
 *  - ops[j]: stencil operators (matrix-free storage), at most 2^31 - 1 cells.
 *  - pc: kind NONE, JACOBI or INNER_PCG with precision FP64 or FP32; applied
 *    per system (the same description for all).
 *  - params: method must be PFK_PIPEFCG; mmax <= PFK_MAX_MMAX; graph_iters and
 *    profile are ignored; history (if set) holds nsys consecutive blocks of
 *    history_capacity entries, one block per system.
 *  - b[j], x[j]: host (ptrs_on_device = 0) or device (1) pointers of length
 *    n_j; x[j] holds x0 on entry and the solution on exit.
 *  - infos: nsys entries (may be NULL); time_ms is the kernel time of the
 *    whole batch; block_threads used is reported in pass_launches.
 *  - block_threads: threads per block (multiple of 32, 64..512), or 0 to pick
 *    it by timing a short trial of each candidate on this batch (cached for
 *    batches of the same size profile in this context).
 * Returns PFK_OK if every system converged, else the first non-OK status of a
 * system (each system's own status is in infos[j].status). */
pfk_status pfk_solve_batched(pfk_context* ctx, int nsys, const pfk_operator* const* ops, const pfk_pc_desc* pc,
                             const pfk_solve_params* params, const double* const* b, double* const* x,
                             int ptrs_on_device, int block_threads, pfk_solve_info* infos);

/* Solves nsys independent stencil systems with PIPEFCG (Alg. 8), PIPEGCR
 * (Alg. 11) or PIPEFGMRES (Alg. 15, constant shift sigma: params.sigma, or
 * NaN for 10 power iterations on v -> A B(v)) on the grouped persistent
 * kernel: each system is advanced by its own group of CTAs
 * (a contiguous range of x-rows per CTA) and the active systems share
 * cooperative launches of a few iterations each, between which finished
 * systems leave and queued ones (in the given order) join.  Within a group
 * the reductions meet at the system's own barrier (bounded waits; a wait that
 * gives up ends that system with PFK_ERR_TIMEOUT) and every CTA combines the
 * partial sums in rank order, so a system's result depends only on its data
 * and its CTA count, not on the rest of the batch (bit for bit).  Fill,
 * iterations, breakdown restarts and the true-residual check run as in
 * pfk_solve.
 *  - ops[j]: matrix-free stencil operators; pc: NONE, JACOBI or INNER_PCG in
 *    FP64 or FP32 (1..64 inner iterations; FP32: vectors and coefficient
 *    copies in FP32, inner products accumulated in FP64), the same
 *    description for all systems.
 *  - params: method PFK_PIPEFCG, PFK_PIPEGCR or PFK_PIPEFGMRES; graph_iters, profile and persistent are
 *    ignored; barrier_timeout_us as for pfk_solve; history (if set) holds
 *    nsys consecutive blocks of history_capacity entries.
 *  - b[j], x[j]: host (ptrs_on_device = 0) or device (1) vectors of length
 *    n_j; x[j] holds x0 on entry and the solution on exit.
 *  - ctas_per_system: 1..64; 0 for about one CTA per 4,096 cells; -1 for a
 *    size chosen by timing: on the first call for a (device, size bucket =
 *    ceil log2 of the largest n, method, preconditioner) key, the systems
 *    that fit one launch run their fill and two timed steps at 2,048, 4,096,
 *    8,192 and 16,384 cells per CTA (x restored afterwards) and the fastest
 *    per cell is kept for the process.  Always at most 64 and at most one
 *    per x-row.  infos[j].pass_launches reports the CTA count used, time_ms
 *    the device time of all launches, kernel_launches their number.
 * Returns PFK_OK if every system converged, else the first non-OK status of
 * a system; PFK_ERR_INVALID for an ineligible system or a system needing more
 * CTAs than the GPU holds at once. */
pfk_status pfk_solve_grouped(pfk_context* ctx, int nsys, const pfk_operator* const* ops, const pfk_pc_desc* pc,
                             const pfk_solve_params* params, const double* const* b, double* const* x,
                             int ptrs_on_device, int ctas_per_system, pfk_solve_info* infos);

/* ------------------------------------------------------------------------ */
/* Serving: continuous batching of independent solves                        */
/* ------------------------------------------------------------------------ */

/* A server accepts solve requests at any time, queues them in arrival order
 * (one queue per path below) and admits a path's next one (by
 * pfk_server_params.order: the head of its queue, or its smallest queued
 * request) as soon as the path has room and the device
 * memory the active solves hold (operator, preconditioner scratch, Krylov
 * workspace) plus the new request's estimate fits the budget; a request larger
 * than the budget still runs when nothing else is active.  Small requests that
 * the grouped kernel can run (group_max_n) are advanced together by one
 * scheduler thread: each gets its own group of CTAs in cooperative launches of
 * a few iterations, between which finished requests leave and queued ones
 * join (room = free CTAs of the launch).  The others go to worker threads that
 * each own a CUDA stream and run whole solves (graph-replayed iterations,
 * Krylov basis resident on the device); the kernels of both kinds overlap on
 * the GPU.  A request's arithmetic does not depend on the other requests: its
 * result is bit for bit the one a solve of the same request alone gives
 * (pfk_solve_grouped with the same CTA count, or pfk_solve).  The server is
 * internally synchronised (any thread may submit and poll). */
typedef struct pfk_server pfk_server;

/* Admission order of queued requests (a scheduling choice; the paper has no
 * counterpart).  FIFO: arrival order.  SMALLEST_FIRST: the queued request with
 * the fewest unknowns (earliest arrival among equals) -- a lower median
 * latency for an oversubscribed stream, large requests wait longer. */
typedef enum { PFK_SERVE_FIFO = 0, PFK_SERVE_SMALLEST_FIRST = 1 } pfk_serve_order;

typedef struct {
  int32_t workers;         /* concurrent whole-GPU solves; 0 = 4 */
  int32_t queue_capacity;  /* queued + active requests; 0 = 4096 */
  int64_t memory_budget;   /* device bytes for active solves; 0 = 80 % of free memory */
  int32_t order;           /* pfk_serve_order; 0 = FIFO */
  int32_t group_max_n;     /* requests of at most this many unknowns that the grouped
                              kernel can run (pfk_solve_grouped: stencil, PIPEFCG,
                              PIPEGCR or PIPEFGMRES, NONE / JACOBI / INNER_PCG) are
                              advanced together on
                              it; 0 = 110,592 (48^3), < 0 = never */
  int32_t group_ctas;      /* CTAs per grouped request, as pfk_solve_grouped's
                              ctas_per_system; 0 = automatic */
  int32_t reserved;        /* 0 */
} pfk_server_params;

typedef struct {
  pfk_operator_desc op;     /* host arrays only; copied by pfk_submit */
  pfk_pc_desc pc;           /* kind PFK_PC_NONE for no preconditioner */
  pfk_solve_params params;  /* history and profile are ignored */
  const double* b;          /* host, length n, copied */
  const double* x0;         /* host or NULL (zero), copied */
} pfk_request;

/* ctx supplies the device; the server creates its own streams and contexts. */
pfk_status pfk_server_create(pfk_context* ctx, const pfk_server_params* params, pfk_server** srv);
/* Queues a request; *ticket identifies it.  PFK_ERR_BUSY when the queue is
 * full, PFK_ERR_INVALID for a bad description (message: pfk_last_error(NULL)). */
pfk_status pfk_submit(pfk_server* srv, const pfk_request* req, uint64_t* ticket);
/* Waits up to wait_ms (< 0: without limit) for the request.  PFK_PENDING if it
 * is not done yet; otherwise the solve's status, with x_out (host, length n;
 * may be NULL), info (may be NULL) and latency_ms = submission to completion
 * (may be NULL) filled in, and the ticket released.  For a request served on
 * the grouped kernel info->time_ms is the host time from its admission to its
 * completion (its launches are shared with other requests) and
 * info->pass_launches its CTA count.  PFK_ERR_INVALID for an unknown or
 * already collected ticket. */
pfk_status pfk_poll(pfk_server* srv, uint64_t ticket, double* x_out, pfk_solve_info* info, double* latency_ms,
                    int wait_ms);
/* Stops admitting, finishes the active solves, drops queued requests. */
pfk_status pfk_server_destroy(pfk_server* srv);

/* ------------------------------------------------------------------------ */
/* Measurement                                                               */
/* ------------------------------------------------------------------------ */

/* FP64 FMA throughput of the device, the denominator of the "alu" roofline of
 * the FP64 Krylov kernels (none of them is a dense contraction; on GB300 their
 * FP64 arithmetic, not HBM, bounds them).  The paper has no counterpart: it is
 * a measurement of the machine.  Runs a kernel of eight independent FMA chains
 * per thread, 8 blocks of 256 threads per SM, `iters` steps per chain (1 <=
 * iters <= 2^24), once to warm up and once timed with CUDA events on ctx's
 * stream.  *tflops = 16 iters threads / time (an FMA counts 2 flops), *ms =
 * the timed launch.  Returns after the work completes.
 * Errors: PFK_ERR_INVALID, PFK_ERR_CUDA. */
pfk_status pfk_probe_fp64_fma(pfk_context* ctx, int iters, double* tflops, double* ms);

/* ------------------------------------------------------------------------ */
/* Allocation-free preconditioner application                                */
/* ------------------------------------------------------------------------ */

/* Largest operator size accepted by pfk_pc_apply_inner_pcg_noalloc. */
#define PFK_NOALLOC_MAX_N 262144

/* y = B(v) for the FP64 inner Jacobi-PCG preconditioner (the same result as
 * pfk_pc_apply with a PFK_PC_INNER_PCG / PFK_FP64 preconditioner of
 * `inner_iters` iterations on `op`), without allocating any device memory.
 * The paper has no counterpart: this is a library service for callers that
 * cannot allocate device memory at the point where they apply the
 * preconditioner -- for instance a framework that has handed all device memory
 * to its own pool allocator, or code that cannot tolerate the device-wide
 * synchronisation cudaMalloc/cudaFree may imply.
 *  - op: a stencil operator (created beforehand) of at most PFK_NOALLOC_MAX_N
 *    unknowns; larger sizes return PFK_ERR_INVALID.  1 <= inner_iters <= 64.
 *  - v, y: device pointers of length n; must not overlap.
 *  - Scratch: one static device array of about 10.5 MB, present on every GPU
 *    that loads the library until the process exits.  The first call on a
 *    device looks up the array's device address (cudaGetSymbolAddress); make
 *    that first call before any stream capture.
 *  - Every call shares the array: calls that overlap on the GPU (other
 *    streams, other host threads, other contexts on the same device) race and
 *    give wrong results.  Each call clears the parts that must start at zero.
 *  - Ordered on ctx's stream; returns after the work completes.
 * Errors: PFK_ERR_INVALID (also when the reduction grid, up to 8 blocks per
 * SM, would need more than the scratch's 2048 partial sums: a GPU with more
 * than 256 SMs), PFK_ERR_CUDA. */
pfk_status pfk_pc_apply_inner_pcg_noalloc(pfk_context* ctx, const pfk_operator* op, int inner_iters,
                                          const double* v, double* y);

#ifdef __cplusplus
}
#endif

#endif /* PFK_H_ */
