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
  int32_t reserved[6];
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

/* One-shot solve = tlqr_factor + tlqr_solve_rhs, and in MIXED precision the
 * iterative refinement: the FP64 KKT residual of eq. (kkt) is re-solved through
 * the FP32 factors and added to the FP64 solution until eta <= refine_tol
 * (TLQR_ERR_NO_CONVERGENCE after max_refine steps).  Writes x, u, y and, when
 * non-NULL, P and K.  prob->mem and sol->mem may differ. */
int tlqr_solve(tlqr_factor_t *f, const tlqr_problem *prob, tlqr_solution *sol, void *stream);

/* Copy the Riccati matrices P_i (Thm. 1) and gains K_e (eq. (factor-local)) of
 * the last factorisation into P [N][n][n] and K [N][m][n] (either may be
 * NULL).  In MIXED precision these are the FP32 factors widened to FP64. */
int tlqr_get_PK(tlqr_factor_t *f, int32_t mem, double *P, double *K, void *stream);

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
 * computes the same stats as tlqr_kkt_residual() (stats[0] = ||K z - b||_inf,
 * stats[1] = eta) from a plan alone, without a factor object.
 *   - prob->mem must be TLQR_MEM_DEVICE; x [N][n], u [N][m], y [N][n] are device
 *     pointers; stats is a host array of 2 doubles.
 *   - Scratch (the tree's parent/child lists, the residual vectors and the
 *     running maxima) lives in one fixed device array of
 *     TLQR_NOALLOC_SCRATCH_BYTES that every GPU loading the library keeps until
 *     the process exits; nothing is allocated per call.  A tree that needs
 *     more scratch (about N (2n + m) 8 + 12 N bytes) is rejected with
 *     TLQR_ERR_ARG before any work is issued.
 *   - The first call on a device looks up the array's device address with that
 *     device current; make that first call before any stream capture.
 *   - All calls share the one array and it keeps the previous call's contents:
 *     calls whose GPU work can overlap (different streams, different host
 *     threads) race on it and must be serialised by the caller.
 *   - Synchronises `stream`. */
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
 * TLQR_K_AFF_TAIL / TLQR_K_STATE_TAIL: the single-block kernels that run the
 * late rounds of the affine and state passes; TLQR_K_FACTOR_TAIL is reserved
 * (no factorisation tail kernel is launched: in the late rounds one
 * operation's latency, not the launch, sets the time). */
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

/* Static name of a status code. */
const char *tlqr_status_string(int code);

/* ---------------------------------------------------- batched primitives */
/* Device-pointer batches of the local algebra, for testing each kernel on its
 * own.  count independent problems, contiguous [count][..] arrays, FP64 in and
 * out; `precision` selects the arithmetic (TLQR_PREC_FP64 or TLQR_PREC_MIXED =
 * FP32).  Return TLQR_ERR_SINGULAR / TLQR_ERR_NOT_PD if any factorisation in the
 * batch failed (synchronises `stream`). */

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

#ifdef __cplusplus
}
#endif
#endif /* TLQR_H */
