/*
 * tree_ot.h -- C ABI of the GB300 solver for tree-structured optimal transport
 * with local entropic regularisation ("A parallel framework for graphical
 * optimal transport", Sec. 3).
 *
 * Problem (Sec. 3, eq. ot_graph_pairwise_mass): a tree G = (V, E); node j has a
 * support of n_j points; edge (j,k) has a cost C_(j,k) (n_j x n_k) with
 * C_(k,j) = C_(j,k)^T.  Nodes in Gamma ("fixed") carry a given probability
 * vector mu_j; they must be leaves and no edge may join two fixed nodes
 * (Sec. 3.1).  The solver minimises
 *     sum_e <C_e, B_e> + eps H(B_e | M_e),  M_(j,k) = gamma_j x gamma_k,
 * gamma_j = mu_j on Gamma and 1 elsewhere (eq. jointdist), subject to
 * B_(j,k) 1 = mu_j, B_(j,k)^T 1 = mu_k, 1^T mu_j = 1 for free j.
 *
 * Method: the closed-form block updates of theorem thm:tree_dual_var in
 * log form, scheduled as in the Bipartite Iterative Scaling algorithm: the tree
 * is two-coloured; a half-step updates every node of one colour from its
 * neighbours' current potentials.  The colour of node 0 goes first.  One
 * half-step = one "edge apply" launch (every edge's Gibbs kernel applied once,
 * in log-sum-exp form, toward the active side) + one node-update launch.
 *
 * Potentials: one vector per DIRECTED edge.  Within problem p, directed edge
 * 2e runs from edges[e][0] to edges[e][1] and holds
 *     f_(a,b) = eps * log u_(a,b)  (length n_a, a = edges[e][0]);
 * directed edge 2e+1 holds f_(b,a) (length n_b).  The plan of edge e is
 *     B_e(x,y) = gamma_a(x) gamma_b(y) exp((f_(a,b)(x) + f_(b,a)(y) - C_e(x,y)) / eps).
 *
 * Conventions for every entry point:
 *   - return 0 on success, a negative TREE_OT_ERR_* code on failure, or
 *     TREE_OT_NOT_CONVERGED (+1, a warning: results are valid);
 *   - tree_ot_last_error() returns a thread-local message for the last failure;
 *   - host pointers are only read during the call unless stated otherwise;
 *   - a handle is not thread-safe; distinct handles are independent;
 *   - cuda_stream is a cudaStream_t (NULL = legacy default stream); all device
 *     work of a call is queued on it; calls that return host data synchronise it.
 */
#ifndef TREE_OT_H
#define TREE_OT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------ */
#define TREE_OT_OK                 0
#define TREE_OT_NOT_CONVERGED      1   /* warning: iteration cap reached, results valid */
#define TREE_OT_ERR_ARG          (-1)  /* NULL pointer, bad size or option */
#define TREE_OT_ERR_NOT_TREE     (-2)  /* not J-1 edges, self loop, cycle or disconnected */
#define TREE_OT_ERR_FIXED_NOT_LEAF (-3) /* a fixed node has degree != 1 (Sec. 3.1) */
#define TREE_OT_ERR_FIXED_ADJACENT (-4) /* an edge joins two fixed nodes (Sec. 3.1) */
#define TREE_OT_ERR_MARGINAL     (-5)  /* mu_j negative, non-finite, or |sum - 1| > 1e-9 */
#define TREE_OT_ERR_NONFINITE    (-6)  /* NaN / -inf cost or non-finite coordinates */
#define TREE_OT_ERR_EPS          (-7)  /* eps <= 0 or not finite */
#define TREE_OT_ERR_CUDA         (-8)  /* a CUDA runtime call failed (see tree_ot_last_error) */
#define TREE_OT_ERR_OOM          (-9)  /* device allocation failed */
#define TREE_OT_ERR_TIMEOUT      (-10) /* a bounded device wait ran out */
#define TREE_OT_ERR_STATE        (-11) /* call not valid in the handle's current state */

/* ---- problem description ------------------------------------------------ */
#define TREE_OT_COST_DENSE_F32   0  /* stored FP32 matrix per edge                       */
#define TREE_OT_COST_SQEUCLID    1  /* C(x,y) = cost_scale * ||x - y||^2 from coordinates */

#define TREE_OT_INPUT_DEVICE     1u /* coords / dense_cost pointers are device pointers   */

typedef struct tree_ot_problem {
    int32_t num_nodes;               /* J >= 2                                            */
    const int32_t *edges;            /* host, [J-1][2] node ids (0-based)                  */
    const int32_t *support_size;     /* host, [J] n_j >= 1                                 */
    const uint8_t *is_fixed;         /* host, [J] 1 = node in Gamma                        */
    const double *const *marginal;   /* host, [J] pointers; mu_j (n_j doubles) for fixed
                                        nodes, ignored (may be NULL) for free nodes        */
    double eps;                      /* regularisation, > 0                                */
    int32_t cost_kind;               /* TREE_OT_COST_*                                     */
    int32_t dim;                     /* D in 1..3 for SQEUCLID (also used by DENSE when
                                        coords are given; may be 0 then)                   */
    const float *const *coords;      /* [J] pointers to n_j x D row-major FP32 points;
                                        required for SQEUCLID, optional for DENSE          */
    double cost_scale;               /* SQEUCLID scale (> 0)                               */
    const float *const *dense_cost;  /* DENSE: [J-1] pointers; edge e is an n_a x n_b
                                        row-major FP32 matrix, a = edges[e][0]; +inf
                                        entries are allowed (K = 0), NaN / -inf are not    */
    uint32_t flags;                  /* TREE_OT_INPUT_DEVICE: the coords / dense_cost
                                        pointers are device pointers.  A device dense_cost
                                        whose row length is a multiple of 4 floats and
                                        whose base is 16-byte aligned is BORROWED (must
                                        stay valid until tree_ot_destroy); other inputs
                                        are copied at create.                              */
} tree_ot_problem;

/* ---- options ------------------------------------------------------------ */
#define TREE_OT_PREC_FP32        0  /* FP32 per-element arithmetic, FP64 vectors (default) */
#define TREE_OT_PREC_FP64        1  /* FP64 everywhere (small problems; e.g. 1e-9 stops)   */

#define TREE_OT_APPLY_AUTO       0
#define TREE_OT_APPLY_LSE        1  /* log-sum-exp on C (stored or recomputed)             */

#define TREE_OT_TOL_SUM          0  /* the paper's stopping sum (Bipartite Iterative Scaling) */
#define TREE_OT_TOL_MAX          1  /* the largest single term of that sum                 */

typedef struct tree_ot_options {
    int32_t precision;        /* TREE_OT_PREC_*                                          */
    int32_t apply_mode;       /* TREE_OT_APPLY_*                                         */
    double tol;               /* stop when the stopping quantity < tol (delta')           */
    int32_t tol_kind;         /* TREE_OT_TOL_*                                           */
    int64_t max_half_steps;   /* iteration cap (half-steps)                               */
    int32_t check_every;      /* half-steps between convergence read-backs (even, >= 2)  */
    int32_t use_graph;        /* 1: replay each chunk of half-steps as a CUDA graph      */
    uint32_t flags;           /* reserved, 0                                             */
} tree_ot_options;

/* ---- per-problem result ------------------------------------------------- */
typedef struct tree_ot_result {
    int32_t status;             /* TREE_OT_OK or TREE_OT_NOT_CONVERGED                    */
    int64_t half_steps;         /* half-steps applied to this problem                     */
    double residual_sum_l1;     /* stopping sum of the returned potentials (FP64 check)  */
    double max_marginal_l1;     /* largest single term of that sum (FP64 check)          */
    double primal;              /* sum_e <C_e,B_e> + eps H(B_e|M_e)                       */
    double dual;                /* -eps f(u,rho) of eq. tree_dual_mass_consv              */
    double transport_cost;      /* sum_e <C_e,B_e>                                       */
    double wall_ms;             /* host wall time of the solve call                      */
} tree_ot_result;

typedef struct tree_ot_handle tree_ot_handle;

/* Fill *opt with defaults: FP32, AUTO, tol 1e-6 (SUM), cap 100000, check 32, graph on. */
void tree_ot_default_options(tree_ot_options *opt);

/* Human-readable name of a return code (static string). */
const char *tree_ot_error_string(int code);

/* Thread-local detail of the last failure of this thread ("" if none). */
const char *tree_ot_last_error(void);

/* Host-only check of the assumptions of Sec. 3 on one problem (no CUDA call).
 * Returns 0 or the TREE_OT_ERR_* code of the first violation found. */
int tree_ot_validate(const tree_ot_problem *prob);

/* Host-only two-colouring of a tree (Sec. 3.1): colour_out[j] in {0,1}, node 0
 * gets colour 0 (updated first).  edges: [num_nodes-1][2].  No CUDA call. */
int tree_ot_bipartition(int32_t num_nodes, const int32_t *edges, uint8_t *colour_out);

/* Validate all problems, build the device plan and upload the data.  Several
 * problems form one batch ("forest"); each converges and retires on its own.
 * Potentials start at zero (u = 1).  opt may be NULL (defaults). */
int tree_ot_create(const tree_ot_problem *probs, int32_t num_probs, const tree_ot_options *opt,
                   void *cuda_stream, tree_ot_handle **out);

/* Release every device buffer the handle owns (borrowed inputs are not freed).
 * NULL-safe. */
int tree_ot_destroy(tree_ot_handle *h);

/* Reset every problem to u = 1 and clear iteration counters. */
int tree_ot_reset(tree_ot_handle *h, void *cuda_stream);

/* Iterate from the current state until every problem meets opt->tol or the
 * cap, then run the FP64 check.  results: host array [num_probs] (may be NULL).
 * Returns TREE_OT_NOT_CONVERGED if some problem hit the cap. */
int tree_ot_solve(tree_ot_handle *h, void *cuda_stream, tree_ot_result *results);

/* Queue exactly T half-steps (no convergence test, no retirement, no sync).
 * Continues the schedule: half-step number t uses colour (t+1) % 2 ... i.e. the
 * first half-step after create/reset updates colour 0. */
int tree_ot_half_steps(tree_ot_handle *h, void *cuda_stream, int64_t T);

/* The two launches of one half-step on colour c, exposed separately so callers
 * can time the edge-apply kernel on its own stream.  tree_ot_apply writes the
 * partial log-sum-exp buffers for every directed edge owned by a colour-c node;
 * tree_ot_node_update merges them, updates the colour-c potentials and records
 * the stopping terms of the other colour.  Calling apply(c) then
 * node_update(c) equals one half-step on colour c. */
int tree_ot_apply(tree_ot_handle *h, void *cuda_stream, int32_t colour);
int tree_ot_node_update(tree_ot_handle *h, void *cuda_stream, int32_t colour);

/* FP64 check of the current potentials (marginals, stopping sum, objectives).
 * results: host [num_probs]; half_steps/status/wall_ms reflect the last solve. */
int tree_ot_check(tree_ot_handle *h, void *cuda_stream, tree_ot_result *results);

/* Marginal of node j of problem p from the last tree_ot_check / tree_ot_solve
 * (FP64): B_(j,k_j) 1 for fixed j, the mean of {B_(j,k) 1}_k for free j.
 * out: host, n_j doubles. */
int tree_ot_marginals(tree_ot_handle *h, int32_t prob, int32_t node, double *out);

/* Copy the potential vector of directed edge `dedge` (0 <= dedge < 2(J-1), see
 * the numbering above) of problem p to / from host memory (FP64, n_owner values).
 * set_potentials is how warm starts and checkpoint resumes enter; the free-node
 * dual constraint (sum_k f_(j,k) constant) need not hold for the supplied values. */
int tree_ot_get_potentials(tree_ot_handle *h, void *cuda_stream, int32_t prob, int32_t dedge, double *out);
int tree_ot_set_potentials(tree_ot_handle *h, void *cuda_stream, int32_t prob, int32_t dedge, const double *in);

/* Plan statistics of the handle (host values), first nstats of:
 * [0] directed edges, [1] edges, [2] plan elements per half-step
 * (sum_e n_a n_b: every half-step applies every edge once), [3] stored cost
 * bytes read per half-step (4 sum_e n_a n_b for dense costs, 0 when costs are
 * recomputed), [4] apply tasks of colour 0, [5] of colour 1, [6] device bytes
 * owned by the handle, [7] node-update CTAs of colour 0, [8] of colour 1. */
int tree_ot_plan_stats(tree_ot_handle *h, int64_t *stats, int32_t nstats);

/* Allocation-free apply of one stored cost matrix (the paper has no
 * counterpart: this is a packaging of the edge-apply kernel for callers that
 * cannot allocate device memory -- code running while a CUDA graph is being
 * captured, serving runtimes that own every byte of device memory through a
 * pre-sized pool, or real-time loops that forbid the device-wide
 * synchronisation cudaMalloc/cudaFree can cause).
 *
 *   m_out[x] = log sum_{y < n_cols} exp( g[y] - cost[x * ld + y] / eps ),  x < n_rows
 *
 * cost: device, n_rows x ld FP32 row-major (ld >= n_cols, ld % 4 == 0, base
 *       16-byte aligned); entries past n_cols in a row are ignored; +inf entries
 *       contribute nothing; NaN / -inf are not allowed (not checked).
 * g:    device, n_cols FP64 (e.g. f_(k,j)/eps + log gamma_k of the neighbour).
 * m_out: device, n_rows FP64 (natural log; -inf where every term is zero).
 * All three are caller-owned; the call allocates nothing (no cudaMalloc,
 * cudaFree or allocating library routine).  Its scratch -- the two-float
 * operand and the per-1024-column partial sums -- lives in a file-scope device
 * array of 4 MiB that every GPU that loads the library holds until exit;
 * requests needing more than that (2 * roundup64(n_cols) + 2 * n_rows *
 * ceil(n_cols / 1024) floats > 2^20) are rejected with TREE_OT_ERR_ARG.
 * The first call on a device looks up the array's device address (one
 * cudaGetSymbolAddress, with that device current); make that first call before
 * any stream capture.  Every call reuses the same array and overwrites the
 * part it reads before reading it, so nothing needs clearing, but calls whose
 * work overlaps on the GPU (different streams, or different host threads) race
 * on it: serialise them.  Work is queued on cuda_stream; the call does not
 * synchronise it. */
int tree_ot_edge_apply_noalloc(const float *cost, int64_t ld, int32_t n_rows, int32_t n_cols, const double *g,
                               double eps, double *m_out, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* TREE_OT_H */
