/*
 * tlqr.h -- C ABI of the B300 (sm_103a) rake-compress solver for branched,
 * dual-regularized LQR problems ("Rake-Compress Riccati Recursions for Parallel
 * Scenario-Tree Model Predictive Control", arXiv 2608.01332).
 *
 * Problem (Sec. III-A, eq. (1)-(2)).  A rooted tree with N nodes, parent[root]
 * = -1.  Every edge e = (i, j) is identified with its child j.  Node data:
 * Q_i (n x n, symmetric), q_i (n), c_i (n), Delta_i (n x n, symmetric PSD).  Edge
 * data: M_e (n x m), R_e (m x m, SPD), r_e (m), A_e (n x n), B_e (n x m).  The
 * solver returns the unique solution (Prop. 1) of the KKT system eq. (kkt):
 *   Q_i x_i + q_i - y_i + sum_{e=(i,j)} (M_e u_e + A_e^T y_j) = 0
 *   M_e^T x_i + R_e u_e + r_e + B_e^T y_j = 0
 *   c_rho - x_rho - Delta_rho y_rho = 0
 *   A_e x_i + B_e u_e + c_j - x_j = Delta_j y_j
 * together with the Riccati matrices P_i (Thm. 1) and the gains K_e
 * (eq. (factor-local)).  Assumptions of Def. 1 are the caller's responsibility;
 * violations are reported as TLQR_ERR_NOT_PD / TLQR_ERR_SINGULAR where a
 * factorisation detects them.
 *
 * Layout.  All numerical arrays are FP64, C-contiguous, row-major dense
 * blocks.  Node arrays are [N][..] in the caller's node order.  Edge arrays
 * are indexed by the child node, [N][..]; the root slot is ignored on input and
 * written as zero on output.  Shapes: Q, P, Delta [N][n][n]; q, c, x, y [N][n];
 * M, B [N][n][m]; R [N][m][m]; r, u [N][m]; A [N][n][n]; K [N][m][n].
 *
 * Memory.  Each call that takes data says whether its pointers are device
 * pointers (TLQR_MEM_DEVICE) or host pointers (TLQR_MEM_HOST); with host
 * pointers the library stages the copies itself on the given stream and the
 * call returns after the results have reached the host.  The caller owns all
 * data buffers; the library owns plans, factor objects and their device
 * workspace.
 *
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream).  Device-pointer calls are asynchronous with respect to the host,
 * except that a call which must report a numerical status (factor, solve)
 * synchronises the stream before returning it.
 *
 * Errors.  Every int-returning entry point returns TLQR_OK (0) or one of the
 * TLQR_ERR_* codes below; no exception crosses the ABI.  Outputs are undefined
 * when an error is returned.  tlqr_status_string() names a code.
 */
#ifndef TLQR_H
#define TLQR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ codes */
enum {
  TLQR_OK = 0,
  TLQR_ERR_ARG = 1,            /* invalid argument (null pointer, bad size, bad flag)      */
  TLQR_ERR_TOPOLOGY = 2,       /* parent[] is not a rooted tree (roots != 1, cycle, range) */
  TLQR_ERR_NOT_PD = 3,         /* Cholesky of R_e or G_e failed (Def. 1 violated)           */
  TLQR_ERR_SINGULAR = 4,       /* zero or nonfinite pivot in S = I + C P~ or F = I + Delta P */
  TLQR_ERR_NONFINITE = 5,      /* NaN/Inf met in the data or the result                    */
  TLQR_ERR_OOM = 6,            /* device or host allocation failed                         */
  TLQR_ERR_TIMEOUT = 7,        /* a bounded device wait gave up                            */
  TLQR_ERR_NO_CONVERGENCE = 8, /* iterative refinement did not reach the requested tol   */
  TLQR_ERR_CUDA = 9,           /* a CUDA runtime call failed                               */
  TLQR_ERR_STATE = 10          /* call out of order (e.g. solve before factor)             */
};

enum { TLQR_MEM_DEVICE = 0, TLQR_MEM_HOST = 1 };

/* Arithmetic of the contraction.  FP64: every kernel in double precision.
 * MIXED: condensation, contraction, expansion, local factors and the
 * right-hand-side passes in FP32; the KKT residual of eq. (kkt) and the
 * accumulated solution in FP64; iterative refinement re-solves the residual
 * through the stored FP32 factors until eta <= refine_tol. */
enum { TLQR_PREC_FP64 = 0, TLQR_PREC_MIXED = 1 };

/* Node operation kinds reported by tlqr_plan_schedule(). */
enum { TLQR_OP_ROOT = 0, TLQR_OP_RAKE = 1, TLQR_OP_COMPRESS = 2 };

typedef struct tlqr_plan_t tlqr_plan_t;     /* opaque, immutable after creation */
typedef struct tlqr_factor_t tlqr_factor_t; /* opaque, device-resident workspace + factors */

typedef struct {
  int32_t n, m;          /* state and control dimension, 1 <= n, m <= TLQR_MAX_DIM */
  int32_t precision;     /* TLQR_PREC_*                                           */
  int32_t has_M;         /* 1: problems carry M_e; 0: M_e = 0                     */
  int32_t has_delta;     /* 1: problems carry Delta_i; 0: Delta_i = 0             */
  int32_t max_refine;    /* MIXED: maximum refinement steps (default 10)          */
  double refine_tol;     /* MIXED: target eta (default 1e-8)                      */
  int32_t use_graphs;    /* 1: replay per-round launch sequences from CUDA graphs */
  int32_t generic_kernels; /* 1: use the run-time-n kernels even where compile-time-n
                              kernels exist (n = 4, 6, 8, 12, 16); for testing        */
  int32_t async_ops;     /* level-asynchronous factorisation tail (compile-time-n
                            kernels): every structural round from the first one after
                            which each round holds at most this many rakes plus
                            compressions runs, with its expansions, in one persistent
                            launch ordered by the dependency levels of
                            eq. (earliest-level) instead of round by round.
                            0 = the library's default (1024), < 0 = off            */
  int32_t spin_limit;    /* polls of one dependency wait of that launch, and of one
                            mbarrier wait of the node-organised residual, before it
                            gives up with TLQR_ERR_TIMEOUT (0 = default, about a
                            second or more)                                        */
  int32_t test_withhold; /* testing failure detection only (bits): 1 = the first
                            operation of the level-asynchronous launch never signals
                            completion, so the waits that depend on it run out; 2 = the
                            node-organised residual announces its first node's bulk
                            copies and issues none, so that mbarrier wait runs out.
                            Either way the call returns TLQR_ERR_TIMEOUT              */
  int32_t tail_ops;      /* right-hand-side passes: the rounds from the first one after
                            which every phase holds at most this many operations run in
                            one single-block launch per pass (0 = default 128, < 0 =
                            none; compile-time-n kernels only)                      */
  int32_t async_solve;   /* right-hand-side passes (compile-time-n kernels): 1 = every
                            round of the affine pass in one level-asynchronous launch
                            and every round of the state pass in another (the
                            dependency DAG of eq. (earliest-level) applied to the
                            passes of Sec. VI-VII); 0 (default) or < 0 = round by
                            round with the single-block tail of tail_ops            */
  int32_t residual;      /* MIXED refinement residual kernels: 1 = one KKT row per
                            thread; 2 = one node per lane group, the node's FP64
                            blocks staged by bulk copies (TMA), compile-time (n, m)
                            and 16-byte aligned matrix arrays only (else 1);
                            0 = the library's choice for n                       */
  int32_t fp64_resolve;  /* MIXED, compile-time-n kernels: 0 (default) = a linear
                            solve of the contraction (S = I + C U, I + C P~ of eq.
                            (compress-intermediates), F = I + Delta P of eq. (FW))
                            whose FP32 pivots span more than 1e4 is solved again in
                            FP64 and rounded to FP32 (up to 4096 per factorisation;
                            tlqr_info.fp64_resolves counts them); < 0 = never       */
  int32_t pdl;           /* 0 (default) = the kernels of the factorisation and of the
                            right-hand-side passes are launched with programmatic
                            dependent launch (each may be scheduled while its
                            predecessor drains, and waits for its results on the
                            device); < 0 = plain stream-ordered launches            */
} tlqr_options;

#define TLQR_MAX_DIM 64

typedef struct {
  int32_t mem;           /* TLQR_MEM_DEVICE or TLQR_MEM_HOST for every pointer   */
  const double *Q, *q;   /* node: [N][n][n], [N][n]                              */
  const double *M;       /* edge: [N][n][m], NULL iff options.has_M == 0         */
  const double *R, *r;   /* edge: [N][m][m], [N][m]                              */
  const double *A, *B;   /* edge: [N][n][n], [N][n][m]                           */
  const double *c;       /* node: [N][n] (c[root] = c_rho)                       */
  const double *Delta;   /* node: [N][n][n], NULL iff options.has_delta == 0     */
} tlqr_problem;

typedef struct {
  int32_t mem;           /* TLQR_MEM_DEVICE or TLQR_MEM_HOST                     */
  double *x, *u, *y;     /* [N][n], [N][m], [N][n]; required                      */
  double *P, *K;         /* [N][n][n], [N][m][n]; may be NULL                     */
} tlqr_solution;

typedef struct {
  int32_t N;
  int32_t root;
  int32_t rounds;        /* structural rounds (Sec. X-A)                            */
  int32_t n_rake, n_compress;
  int32_t n_combine;     /* binary sibling combinations of the reductions (Lemma 3) */
  int32_t n_absorb;
  int32_t levels;        /* nonempty dependency levels, eq. (earliest-level); -1 if
                            a reduction's readiness weights exceeded 120 bits      */
  int32_t height;        /* longest root-to-leaf path, in edges                     */
  int32_t max_degree;
  int32_t n_trees;       /* trees of a forest plan (1 for tlqr_plan_create)          */
} tlqr_plan_stats_t;

typedef struct {
  int32_t refine_steps;  /* MIXED: refinement steps taken by the last solve      */
  double eta;            /* backward error of the last solve, if it computed one   */
  double abs_residual;   /* ||K z - b||_inf of the last solve, if computed         */
  int32_t fp64_resolves; /* MIXED: eliminations of the last factorisation solved
                            again in FP64 (see tlqr_options.fp64_resolve)        */
} tlqr_info;

/* ------------------------------------------------------------------ plan */

/* Build the topology-only contraction plan (Alg. 1 step 1; schedule of
 * Sec. X-A: each structural round rakes every nonroot leaf, then compresses a
 * maximal set of pairwise nonadjacent unary nonroot nodes chosen greedily in
 * increasing node index).  parent: host int32[N], exactly one -1.  Host only;
 * touches no GPU.  On success *out owns the plan (free with
 * tlqr_plan_destroy).  Errors: TLQR_ERR_ARG (N < 1, null), TLQR_ERR_TOPOLOGY,
 * TLQR_ERR_OOM. */
int tlqr_plan_create(const int32_t *parent, int32_t N, tlqr_plan_t **out);

/* Batch of independent problems: a forest.  Same as tlqr_plan_create but
 * parent[] may hold several -1 entries, one per tree.  The KKT system is then
 * block diagonal, one block per tree, each the system of eq. (kkt) of its own
 * tree; every tree is contracted by the same structural rule in the same
 * rounds, so each tree's schedule -- and, in FP64, each tree's result -- is
 * exactly the one it has alone, while the whole batch runs in one launch
 * sequence.  Node and edge arrays of all trees are concatenated in parent[]
 * order.  Errors as tlqr_plan_create (TLQR_ERR_TOPOLOGY: no root, a cycle, an
 * index out of range). */
int tlqr_plan_create_forest(const int32_t *parent, int32_t N, tlqr_plan_t **out);

/* Free a plan (NULL is ignored).  A plan must outlive the factors made from it. */
void tlqr_plan_destroy(tlqr_plan_t *plan);

/* Counts of the plan: rounds, rakes, compressions (Sec. IX-B: rakes +
 * compressions = N - 1 per tree), dependency levels of eq. (earliest-level) with the
 * readiness-weighted sibling reduction of eq. (readiness-code-data) (Lemma 3,
 * Lemma 4), height and maximum out-degree.  Host only. */
int tlqr_plan_stats(const tlqr_plan_t *plan, tlqr_plan_stats_t *out);

/* Per node: the structural round (1-based; 0 for the root) in which it is
 * removed and how (TLQR_OP_*), as drawn in Fig. 2.  Host arrays int32[N]. */
int tlqr_plan_schedule(const tlqr_plan_t *plan, int32_t *round_of_node, int32_t *op_of_node);

/* ---------------------------------------------------------------- factor */

/* Allocate the device workspace of a factorisation for this plan and
 * dimensions on the current CUDA device: one device allocation holding the
 * plan's arrays and the workspace, plus a few pinned host words.  The options
 * are copied; the plan must outlive the factor.  Errors: TLQR_ERR_ARG
 * (dimensions out of range, bad precision), TLQR_ERR_OOM, TLQR_ERR_CUDA. */
int tlqr_factor_create(const tlqr_plan_t *plan, const tlqr_options *opts, tlqr_factor_t **out);

/* Device bytes tlqr_factor_create would allocate for this plan and options
 * (host only, nothing is allocated) -- for admission control by device
 * memory.  Calls with host-memory problems add a lazily allocated FP64
 * staging area of the problem's size. */
int tlqr_factor_workspace_bytes(const tlqr_plan_t *plan, const tlqr_options *opts, size_t *bytes);

/* An operation list of the level-asynchronous launches that a factor object
 * with state dimension n would run for this plan (host only, for inspection
 * and testing): which = 0 the factorisation tail for tlqr_options.async_ops =
 * async_ops, 1 the affine pass of a right-hand side, 2 its state pass.
 * counts[4] receives the first asynchronous round (0-based; = rounds when there
 * is none), the padded operation count P, the flag count and the number of
 * dependency levels.  When `kind` is non-NULL the host arrays receive, per
 * position p < P: kind[p] (0 rake, 1 absorption, 2 compression, 3 expansion
 * -- their affine-pass counterparts for which = 1 -- and for which = 2: 4 offset
 * composition, 5 state expansion of a compressed centre, 6 of a raked leaf),
 * node[p] (raked leaf, absorbing parent or compressed centre; -1 for a padding
 * slot), round[p] (1-based structural round), dep_flag[3p..3p+2] (flag
 * indices, -1 = none), dep_target[3p..3p+2] (the value each flag must reach;
 * flag q < P is the completion flag of position q, flags >= P count the
 * finished rakes of one sibling segment) and signal[p] (the counter a rake
 * increments, else -1).  Errors: TLQR_ERR_ARG, TLQR_ERR_OOM. */
int tlqr_async_schedule(const tlqr_plan_t *plan, int32_t n, int32_t which, int32_t async_ops, int32_t *counts,
                        int32_t *kind, int32_t *node, int32_t *round, int32_t *dep_flag, int32_t *dep_target,
                        int32_t *signal);

/* The options a factor object was created with (defaults filled in). */
int tlqr_factor_options(const tlqr_factor_t *f, tlqr_options *out);

/* dims[3] = {N, n, m} of a factor object (host array). */
int tlqr_factor_dims(const tlqr_factor_t *f, int32_t *dims);

/* Device bytes a factor object holds now (workspace + staging, if any). */
int tlqr_factor_bytes(const tlqr_factor_t *f, size_t *bytes);

/* Free a factor object and its device memory (NULL is ignored). */
void tlqr_factor_destroy(tlqr_factor_t *f);

/* Factor the KKT matrix of eq. (kkt) (Alg. 1 steps 2-3): condensation
 * eq. (edge-components); per structural round the rakes eq. (terminal-fold)
 * with in-order sibling sums absorbed into the parent, then the compressions
 * eq. (compress-intermediates)-(composition) with their tape
 * eq. (quadratic-compress); the reverse reconstruction eq. (value-reconstruction)
 * giving every P_i; the local factors eq. (FW), (factor-local); and the
 * composed transition matrices of eq. (transition-compose) reused by every
 * right-hand side.  Only Q, M, R, A, B, Delta of the problem are read (q, r, c
 * may be NULL).  Synchronises `stream` to report TLQR_ERR_NOT_PD /
 * TLQR_ERR_SINGULAR / TLQR_ERR_NONFINITE. */
int tlqr_factor(tlqr_factor_t *f, const tlqr_problem *prob, void *stream);

/* Solve one right-hand side (q, r, c) with the stored factorisation
 * (Alg. 1 steps 4-6, Sec. VI): affine maps eq. (affine-edge), their
 * contraction and expansion eq. (affine-rake), (affine-compose); the local
 * affine solve eq. (local-affine-solve) and root state eq. (xroot); the state
 * maps eq. (state-map) contracted and expanded from x_rho; recovery
 * eq. (recover).  Pointers follow `mem`; x, u, y are written.  In MIXED
 * precision this is one pass through the FP32 factors without refinement
 * (refinement needs the problem's matrices: use tlqr_solve). */
int tlqr_solve_rhs(tlqr_factor_t *f, int32_t mem, const double *q, const double *r, const double *c,
                   double *x, double *u, double *y, void *stream);

/* Several right-hand sides with the stored factorisation (factor reuse across
 * Newton right-hand sides, Sec. VI): q [nrhs][N][n], r [nrhs][N][m], c
 * [nrhs][N][n] in, x, u, y of the same shapes out, all device pointers.  With
 * the compile-time-(n, m) kernels the right-hand sides run as panels of up to
 * 8: every local operation loads its factor block once and applies it to the
 * whole panel (an n x n block times an n x k panel instead of k matrix-vector
 * products), in the launches of one right-hand side.  Otherwise they are solved
 * one by one.  Each result equals tlqr_solve_rhs of that right-hand side alone (one
 * pass through the factors, no refinement); the first panel call allocates the
 * panel vectors once.  Synchronises `stream` to report a status. */
int tlqr_solve_rhs_panel(tlqr_factor_t *f, int32_t nrhs, const double *q, const double *r, const double *c,
                         double *x, double *u, double *y, void *stream);

/* One-shot solve = tlqr_factor + tlqr_solve_rhs, and in MIXED precision the
 * iterative refinement: the FP64 KKT residual of eq. (kkt) is re-solved through
 * the FP32 factors and added to the FP64 solution until eta <= refine_tol
 * (TLQR_ERR_NO_CONVERGENCE after max_refine steps).  Writes x, u, y and, when
 * non-NULL, P and K.  prob->mem and sol->mem may differ. */
int tlqr_solve(tlqr_factor_t *f, const tlqr_problem *prob, tlqr_solution *sol, void *stream);

/* Adjoint (reverse-mode) solve through the right-hand side, for
 * differentiating a loss L(x, u, y) of the solution with respect to the data
 * (q, r, c) (Sec. IX-A mentions differentiation through a right-hand side).
 * The solution is z = -K^{-1} b with K the matrix of eq. (kkt) and b = (q, r, c)
 * in its row blocks; K is symmetric, so dL/db = -K^{-1} dL/dz, which is the
 * solution of the same factored system with (q, r, c) := (xbar, ubar, ybar).
 * Inputs xbar [N][n], ubar [N][m] (root slot ignored), ybar [N][n] = dL/dx,
 * dL/du, dL/dy; outputs qbar [N][n], rbar [N][m] (root slot 0), cbar [N][n] =
 * dL/dq, dL/dr, dL/dc.  Uses the factor of the last tlqr_factor / tlqr_solve;
 * in MIXED precision the result is refined like tlqr_solve (to refine_tol),
 * which needs that call's problem matrices to still be valid.  Pointers follow
 * `mem`.  Errors: TLQR_ERR_STATE before a factorisation, and those of
 * tlqr_solve. */
int tlqr_solve_adjoint(tlqr_factor_t *f, int32_t mem, const double *xbar, const double *ubar, const double *ybar,
                       double *qbar, double *rbar, double *cbar, void *stream);

/* Copy the Riccati matrices P_i (Thm. 1) and gains K_e (eq. (factor-local)) of
 * the last factorisation into P [N][n][n] and K [N][m][n] (either may be
 * NULL).  In MIXED precision these are the FP32 factors widened to FP64. */
int tlqr_get_PK(tlqr_factor_t *f, int32_t mem, double *P, double *K, void *stream);

/* Resident-problem update and re-solve, for interior-point and
 * receding-horizon loops in which only diagonals and the right-hand side
 * change between solves.  The problem the factor last factorised (its own
 * staged copy when that problem came from host memory, else the caller's
 * device arrays, which this call then modifies) is updated in place --
 *   Q_i += diag(dq_i) (dq: N x n),  R_i += diag(dr_i) (dr: N x m)  (NULL: none)
 *   q, r, c replaced by the arrays given (NULL: unchanged)
 * -- then factorised and solved exactly as by tlqr_solve (refinement in
 * MIXED), writing sol.  With mem = TLQR_MEM_HOST only dq, dr, q, r, c cross
 * the bus: N (3n + 2m) doubles instead of the whole problem.  The matrices
 * A, B, M, Delta and the off-diagonal entries of Q and R stay as they were.
 * Errors: TLQR_ERR_ARG; TLQR_ERR_STATE when no problem has been factorised on
 * f yet; otherwise as tlqr_solve. */
int tlqr_update_solve(tlqr_factor_t *f, int32_t mem, const double *dq, const double *dr, const double *q,
                      const double *r, const double *c, tlqr_solution *sol, void *stream);

/* FP64 KKT residual of eq. (kkt) for a given (x, u, y) on the GPU.
 * stats[0] = ||K z - b||_inf, stats[1] = eta = ||K z - b||_inf /
 * (||K||_inf ||z||_inf + ||b||_inf) (normwise backward error), written to the
 * host array stats[2].  For a forest plan the norms are taken tree by tree:
 * stats[0] is the largest residual and stats[1] the largest eta over the trees
 * (a batch meets a tolerance when each of its trees does; the refinement of
 * tlqr_solve stops on the same per-tree eta).  Synchronises `stream`. */
int tlqr_kkt_residual(tlqr_factor_t *f, const tlqr_problem *prob, int32_t mem, const double *x,
                      const double *u, const double *y, double *stats, void *stream);

/* Allocation-free FP64 KKT residual.  The paper has no counterpart: this entry
 * point exists for callers that must not allocate device memory while they
 * run -- for example a receding-horizon controller with a hard deadline
 * (cudaMalloc / cudaFree can synchronise the device and take unbounded time) or
 * a process whose device memory belongs to another framework's allocator.  It
 * computes the same stats as tlqr_kkt_residual() from a plan alone, without a
 * factor object: stats[0] = ||K z - b||_inf and stats[1] = eta, and for a
 * forest plan the largest residual and the largest eta over the trees, each
 * tree's norms taken on its own (the per-tree rule of tlqr_kkt_residual).
 *   - prob->mem must be TLQR_MEM_DEVICE, and every data pointer as well as x
 *     [N][n], u [N][m], y [N][n] must be device (or managed) memory: the call
 *     asks CUDA what each pointer is and returns TLQR_ERR_ARG for a host
 *     pointer before any work is issued.  stats is a host array of 2 doubles.
 *   - Scratch (the tree's parent/child lists, the tree ordinals of a forest,
 *     the residual vectors and the running maxima) lives in one fixed device
 *     array of TLQR_NOALLOC_SCRATCH_BYTES that every GPU loading the library
 *     keeps until the process exits; nothing is allocated per call.  A plan
 *     that needs more scratch (about N (2n + m) 8 + 12 N bytes, plus 4 N + 32 T
 *     for a forest of T trees) is rejected with TLQR_ERR_ARG before any work is
 *     issued.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current.
 *   - Each call copies the plan's index arrays from host memory and waits for
 *     `stream`.
 *   - All calls share the one array and it keeps the previous call's contents:
 *     calls whose GPU work can overlap (different streams, different host
 *     threads) race on it and must be serialised by the caller. */
#define TLQR_NOALLOC_SCRATCH_BYTES (16u << 20)
int tlqr_kkt_residual_noalloc(const tlqr_plan_t *plan, int32_t n, int32_t m, const tlqr_problem *prob,
                              const double *x, const double *u, const double *y, double *stats,
                              void *stream);

/* Per-tree ||K z - b||_inf and eta of the last residual evaluation (the last
 * refinement check of a MIXED tlqr_solve, or tlqr_kkt_residual; an FP64
 * tlqr_solve evaluates none), for the first
 * min(max_trees, number of trees) trees in increasing root label.  Host
 * arrays; either may be NULL.  A single tree has one entry. */
int tlqr_tree_residuals(const tlqr_factor_t *f, double *abs_res, double *eta, int32_t max_trees);

/* Refinement steps and backward error of the last tlqr_solve. */
int tlqr_last_info(const tlqr_factor_t *f, tlqr_info *out);

/* ------------------------------------------------------------- profiling */
/* Kernel kinds launched by the library (one per step of Alg. 1 above).
 * TLQR_K_AFF_TAIL / TLQR_K_STATE_TAIL: the launches that run several rounds
 * of the affine and state passes at once (the single-block kernels of the late
 * rounds, or with async_solve = 1 one level-asynchronous launch per pass);
 * TLQR_K_FACTOR_TAIL: the
 * persistent level-asynchronous launch of the late factorisation rounds (see
 * tlqr_options.async_ops; its units are the operations of its list). */
enum {
  TLQR_K_CONDENSE = 0, TLQR_K_RAKE, TLQR_K_ABSORB, TLQR_K_COMPRESS, TLQR_K_EXPAND,
  TLQR_K_LOCAL_FACTOR, TLQR_K_COMPOSE_T, TLQR_K_AFF_INIT, TLQR_K_AFF_RAKE, TLQR_K_AFF_ABSORB,
  TLQR_K_AFF_COMPRESS, TLQR_K_AFF_EXPAND, TLQR_K_LOCAL_SOLVE, TLQR_K_STATE_COMPRESS,
  TLQR_K_STATE_EXPAND, TLQR_K_RECOVER, TLQR_K_RESIDUAL, TLQR_K_EXPORT, TLQR_K_AFF_TAIL,
  TLQR_K_STATE_TAIL, TLQR_K_FACTOR_TAIL, TLQR_K_COUNT
};

typedef struct {
  int64_t launches;      /* kernel launches of this kind since the last read          */
  int64_t units;         /* local operations (warps) those launches processed         */
  int64_t timed;         /* launches bracketed by CUDA events (kinds in the mask)     */
  double ms;             /* summed event time of the timed launches                    */
} tlqr_kernel_profile;

/* Select the kernel kinds (bit k = kind k) whose launches are bracketed by
 * CUDA events on the launching stream from now on; 0 turns timing off.
 * Launch and unit counters are kept for every kind regardless of the mask. */
int tlqr_profile_mask(tlqr_factor_t *f, uint32_t mask);

/* Synchronise the recorded events, write TLQR_K_COUNT entries to out[] and
 * reset all counters.  Host array. */
int tlqr_profile_read(tlqr_factor_t *f, tlqr_kernel_profile *out);

/* The individual timed launches since the last tlqr_profile_read, in launch
 * order: kind, operations (warps or groups) and milliseconds.  Writes at most
 * `max` entries to the host arrays and the total count to *count; call before
 * tlqr_profile_read, which clears them. */
int tlqr_profile_launches(tlqr_factor_t *f, int32_t *kind, int64_t *units, double *ms, int32_t max,
                          int32_t *count);

/* Measured FMA throughput of the current device's FP32 (precision =
 * TLQR_PREC_MIXED) or FP64 (TLQR_PREC_FP64) pipe in TFLOP/s: independent FMA
 * chains on every resident warp, best of five ~10 ms launches timed with CUDA
 * events on `stream` (a diagnostic for roofline denominators, not part of the
 * solver).  Changes no clock or device setting. */
int tlqr_pipe_peak(int32_t precision, double *tflops, void *stream);

/* Static name of a status code. */
const char *tlqr_status_string(int code);

/* ---------------------------------------------------- batched primitives */
/* Device-pointer batches of the local algebra, for testing each kernel on its
 * own.  count independent problems, contiguous [count][..] device arrays, FP64
 * in and out (converted to and from the working precision by device kernels on
 * `stream`); `precision` selects the arithmetic (TLQR_PREC_FP64 or
 * TLQR_PREC_MIXED = FP32).  Each call runs the kernel the solver itself
 * launches for this n and precision: the compile-time-(n, m) group kernels for
 * n in {4, 6, 8, 12, 16, 32} (at n = 32 in FP32 with the 3xTF32 tensor-core
 * block products), else the run-time-n warp kernels; OR-ing
 * TLQR_BATCHED_GENERIC into `precision` forces the run-time-n kernels.  The
 * library allocates its own device workspace per call.  Return
 * TLQR_ERR_SINGULAR / TLQR_ERR_NOT_PD if any factorisation in the batch failed,
 * TLQR_ERR_ARG on a null pointer or a size out of range (synchronises
 * `stream`). */
#define TLQR_BATCHED_GENERIC 0x100

/* Rake fold eq. (terminal-fold): out = P + A^T U (I + C U)^{-1} A.  All n x n. */
int tlqr_batched_tau(int32_t count, int32_t n, const double *A, const double *C, const double *P,
                     const double *U, double *out, int32_t precision, void *stream);

/* Compress composition eq. (compress-intermediates)-(composition) of
 * alpha_l = (Al, Cl, Pl) (edge into the centre), alpha_r = (Ar, Cr, Pr) (edge out
 * of it) and centre data U: writes (An, Cn, Pn) and the tape's P~ = Pr + U
 * into Pt.  All n x n. */
int tlqr_batched_compose(int32_t count, int32_t n, const double *Al, const double *Cl,
                         const double *Pl, const double *Ar, const double *Cr, const double *Pr,
                         const double *U, double *An, double *Cn, double *Pn, double *Pt,
                         int32_t precision, void *stream);

/* Condensation eq. (edge-components): (Abar, Cbar, Pbar) from A [n x n], B [n x m],
 * R [m x m], M [n x m] (NULL = 0) and Delta [n x n] (NULL = 0). */
int tlqr_batched_condense(int32_t count, int32_t n, int32_t m, const double *A, const double *B,
                          const double *R, const double *M, const double *Delta, double *Abar,
                          double *Cbar, double *Pbar, int32_t precision, void *stream);

/* Reconstruction at a compressed node, eq. (value-reconstruction): from the
 * tape (Ar, Cr, Pt) of eq. (quadratic-compress) and the child's P_k,
 * Pj = Pt + Ar^T Pk (I + Cr Pk)^{-1} Ar.  All n x n. */
int tlqr_batched_expand(int32_t count, int32_t n, const double *Ar, const double *Cr, const double *Pt,
                        const double *Pk, double *Pj, int32_t precision, void *stream);

/* Local factors eq. (FW), (factor-local) of an edge given the child's Riccati
 * matrix P [n x n]: F = I + Delta P, W = P F^{-1}, G = R + B^T W B (Cholesky),
 * K = -G^{-1} (B^T W A + M^T) [m x n], T = F^{-1} (A + B K) [n x n].  A [n x n],
 * B [n x m], R [m x m], M [n x m] (NULL = 0), Delta [n x n] (NULL = 0). */
int tlqr_batched_local_factor(int32_t count, int32_t n, int32_t m, const double *P, const double *A,
                              const double *B, const double *R, const double *M, const double *Delta,
                              double *K, double *T, int32_t precision, void *stream);

/* Composite transition of eq. (transition-compose): out = Tk Tj.  All n x n. */
int tlqr_batched_compose_T(int32_t count, int32_t n, const double *Tk, const double *Tj, double *out,
                           int32_t precision, void *stream);

/* ------------------------------------------------ node-control lifting */

/* Prop. 2 (Sec. III-B): map a node-control problem eq. (node-lagrangian) on a
 * tree with N nodes (state n, one control v_i of size m per nonterminal node)
 * to an edge-control problem with state n + m.  Host arrays.  Inputs, indexed
 * by node: Q [N][n][n], q [N][n], Mv [N][n][m], Rv [N][m][m], rv [N][m] (used at
 * nonterminal nodes), c [N][n], Delta [N][n][n] (NULL = 0); indexed by the child
 * j of each uncertainty edge (i, j): Av [N][n][n], Bv [N][n][m].
 * Output sizes: *Nl = N + (number of nonterminal nodes) <= 2N - 1 lifted nodes.
 * Call first with lifted_parent = NULL to get *Nl; then pass host buffers with
 * Nl entries: lifted_parent [Nl], lQ [Nl][n+m][n+m], lq [Nl][n+m], lM
 * [Nl][n+m][m], lR [Nl][m][m], lr [Nl][m], lA [Nl][n+m][n+m], lB [Nl][n+m][m],
 * lc [Nl][n+m], lDelta [Nl][n+m][n+m], and map [2][N] (map[0][i] = lifted
 * predecision node i-, map[1][i] = decision node i+ or -1).  Dummy controls of
 * uncertainty edges get R = I and zero input. */
int tlqr_lift_node_controls(const int32_t *parent, int32_t N, int32_t n, int32_t m,
                            const double *Q, const double *q, const double *Mv, const double *Rv,
                            const double *rv, const double *Av, const double *Bv, const double *c,
                            const double *Delta, int32_t *Nl, int32_t *lifted_parent, double *lQ,
                            double *lq, double *lM, double *lR, double *lr, double *lA, double *lB,
                            double *lc, double *lDelta, int32_t *map);

/* Projection of Prop. 2: from the lifted solution (lx [Nl][n+m], lu [Nl][m],
 * ly [Nl][n+m]) recover x [N][n], v [N][m] (zero at terminal nodes) and
 * y [N][n].  Host arrays. */
int tlqr_project_lifted(int32_t N, int32_t n, int32_t m, const int32_t *map, const double *lx,
                        const double *lu, const double *ly, double *x, double *v, double *y);

/* Device-side versions of the two calls above, for node-form data that already
 * live on the GPU.  The topology arguments (parent, Nl, lifted_parent, map)
 * are host arrays, computed on the host as by tlqr_lift_node_controls (plans
 * are built on the host from them); every numerical array (Q ... Delta in,
 * lQ ... lDelta out; lx, lu, ly in and x, v, y out for the projection) must be
 * device memory (checked: TLQR_ERR_ARG otherwise), and every lifted block is
 * written by a kernel on `stream`.  Same layouts and size query (call with
 * lifted_parent = NULL for *Nl).  The calls allocate a small index array with
 * cudaMallocAsync on `stream` and return after the stream has finished.
 * Errors: TLQR_ERR_ARG, TLQR_ERR_TOPOLOGY, TLQR_ERR_OOM, TLQR_ERR_CUDA. */
int tlqr_lift_node_controls_device(const int32_t *parent, int32_t N, int32_t n, int32_t m, const double *Q,
                                   const double *q, const double *Mv, const double *Rv, const double *rv,
                                   const double *Av, const double *Bv, const double *c, const double *Delta,
                                   int32_t *Nl, int32_t *lifted_parent, double *lQ, double *lq, double *lM,
                                   double *lR, double *lr, double *lA, double *lB, double *lc, double *lDelta,
                                   int32_t *map, void *stream);
int tlqr_project_lifted_device(int32_t N, int32_t n, int32_t m, const int32_t *map, const double *lx,
                               const double *lu, const double *ly, double *x, double *v, double *y, void *stream);

/* ------------------------------------------- interior-point driver (synthetic) */
/* Box-constrained tree LQR solved by a primal-dual interior-point method whose
 * Newton systems are tree KKT solves -- the call pattern of the nonlinear
 * solver the paper plugs its method into (Sec. IX-B, XI-B): the problem of
 * eq. (1)-(2) with u_lo <= u_e <= u_hi componentwise (+-Inf = no bound; the
 * root slots are ignored).  With slacks s_lo = u - u_lo, s_hi = u_hi - u and
 * multipliers l_lo, l_hi > 0, each iteration solves the tree system with
 * R~ = R + diag(S), r~ = r - S u - mu / s_lo + mu / s_hi, S = l_lo / s_lo +
 * l_hi / s_hi (tlqr_solve on `f`, in its precision), steps to the fraction tau
 * of the boundary and sets mu = sigma * mean(l s); it stops after a full Newton
 * step once mean(l s) <= tol.  With a MIXED factor object the Newton systems
 * are solved in FP32 + refinement until the barrier terms l / s exceed 1e6
 * (they grow like 1 / mu; past that the FP32 factors stop resolving the step on
 * the active bounds, although each solve still meets its normwise tolerance)
 * or a solve fails, and from then on with an FP64 factor object of the same
 * plan, created on first need and freed on return.  Device arrays: prob (mem
 * must be
 * TLQR_MEM_DEVICE), u_lo, u_hi [N][m]; outputs x, u, y [N][n|m|n] and the
 * multipliers lam_lo, lam_hi [N][m] (zero where a bound is absent).  f must be
 * a factor object of `plan`.  The call allocates one device workspace for its
 * duration and synchronises `stream` once per iteration.  Errors:
 * TLQR_ERR_ARG (bad pointer, host memory, empty box), TLQR_ERR_NO_CONVERGENCE
 * (max_iter reached), and those of tlqr_solve. */
typedef struct {
  int32_t max_iter;      /* default 100 */
  double mu0;            /* initial barrier parameter, default 1 */
  double sigma;          /* centring factor in (0, 1), default 0.1 */
  double tau;            /* fraction to the boundary in (0, 1), default 0.995 */
  double tol;            /* target mean complementarity, default 1e-9 */
  int32_t no_fp64_fallback; /* 1: never allocate the FP64 factor object; a MIXED Newton
                               solve whose refinement stalls is used as it stands
                               (an inexact Newton step), and a Newton system the FP32
                               factors cannot take (not positive definite, singular or
                               nonfinite once the barrier terms outgrow FP32) ends the
                               iteration at the current iterate with
                               TLQR_ERR_NO_CONVERGENCE -- for callers that budget
                               device memory per request */
} tlqr_ipm_options;

typedef struct {
  int32_t iterations;
  double mu, mean_gap;   /* last barrier parameter and mean l s */
  double last_alpha;     /* step length of the last iteration */
  double last_eta;       /* backward error of the last Newton solve (MIXED) */
  int32_t fp64_solves;   /* Newton systems re-solved in FP64 (MIXED factor objects) */
} tlqr_ipm_info;

int tlqr_ipm_box(const tlqr_plan_t *plan, tlqr_factor_t *f, const tlqr_problem *prob, const double *u_lo,
                 const double *u_hi, const tlqr_ipm_options *opts, double *x, double *u, double *y,
                 double *lam_lo, double *lam_hi, tlqr_ipm_info *info, void *stream);

/* ------------------------------------------------------------- autotuner */
/* Pick the execution shape for one plan and problem by timing it on the
 * current device: every combination of async_ops in {-1 (off), 256, 1024,
 * 4096} with the right-hand-side passes level-asynchronous (async_solve = 1)
 * or round by round with a single-block tail of tail_ops in {-1 (none), 64,
 * 128, 512}; then, in mixed precision with base->residual = 0, the fastest
 * of those with residual = 1 and residual = 2.  Each
 * candidate gets a factor object of its own (created and freed in turn, so
 * only one workspace is held at a time), one warm-up tlqr_solve and `trials`
 * timed ones (CUDA events on `stream`, median).  *best receives `base` with the
 * fastest candidate's four fields; table (may be NULL) up to max_entries
 * rows, *n_entries the number written.  prob: device data (mem must be
 * TLQR_MEM_DEVICE).  The call allocates x, u, y for the trials.  Errors:
 * TLQR_ERR_ARG, TLQR_ERR_OOM, TLQR_ERR_NO_CONVERGENCE (no candidate finished),
 * and the first hard error of a candidate. */
typedef struct {
  int32_t async_ops, async_solve, tail_ops, residual;
  int32_t status;        /* TLQR_OK or the candidate's error */
  double ms;             /* median time of one tlqr_solve, -1 when it failed */
} tlqr_autotune_entry;

int tlqr_autotune(const tlqr_plan_t *plan, const tlqr_options *base, const tlqr_problem *prob, int32_t trials,
                  tlqr_options *best, tlqr_autotune_entry *table, int32_t max_entries, int32_t *n_entries,
                  void *stream);

#ifdef __cplusplus
}
#endif
#endif /* TLQR_H */
