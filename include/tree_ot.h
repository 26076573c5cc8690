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
#define TREE_OT_APPLY_BF16       2  /* BF16 phase, then FP32 LSE refinement (see refine_tol,
                                       absorb_tau, lowp_start): stored costs use an absorbed
                                       BF16 kernel per edge; squared-Euclidean problems whose
                                       directed edges share supports, scale and eps (at least
                                       8 per kernel) use one shared kernel on the tensor cores;
                                       other problems run FP32 throughout                    */

/* options.flags: which kernel streams stored costs (FP32 path).  With neither
 * bit the autotuner (autotune = 1) times both and keeps the faster; with
 * autotune = 0 the plain-load kernel runs. */
#define TREE_OT_OPT_DENSE_TMA    1u /* bulk-copy staged kernel (one producer warp, ring)   */
#define TREE_OT_OPT_DENSE_LDG    2u /* plain 16-byte streaming loads                       */
/* Recomputed (squared-Euclidean) costs are formed in FP32; the rounding of
 * |x - y|^2 alone perturbs C/eps enough to hold some iterates ~1e-7..1e-6 (max
 * marginal L1) away from the solution at small eps.  Problems the certification
 * (see tree_ot_solve) finds stuck above tol continue with exactly formed squared
 * distances (coordinates split hi + lo, ~1.8x the FP32 work per element); this
 * bit uses the exact form from the first half-step for every such problem. */
#define TREE_OT_OPT_EXACT_DIST   4u
/* Stored costs: when the device has room (free memory above twice the matrices'
 * size plus 1 GiB) every edge also keeps its cost transposed, so the column
 * node's apply streams contiguous rows like the row node's (the same bytes per
 * apply; twice the memory).  This bit keeps only the given layout. */
#define TREE_OT_OPT_NO_TRANSPOSE 8u
/* Test hook for the staged kernel's failure path: its producer issues no
 * copies, so every consumer's bounded wait runs out (about a second); the
 * kernel returns normally and tree_ot_solve reports TREE_OT_ERR_TIMEOUT.
 * Implies TREE_OT_OPT_DENSE_TMA.  No GPU fault is involved. */
#define TREE_OT_OPT_TEST_STALL   16u
/* Batches whose costs are all recomputed from points of one dimension (FP32,
 * no BF16 phase): run chunks of half-steps as ONE persistent launch each
 * (inside tree_ot_solve's captured CUDA graph, one graph node per chunk), the
 * CTAs taking apply tasks and node-update chunks in schedule order from an
 * atomic ticket and each waiting only for its own problem's previous phase
 * (per-problem phase counters): trees advance on their own, a tree's node
 * update overlaps other trees' applies, and retired trees cost nothing.  At
 * create the per-half-step launches and the persistent kernel at 2 and 3 CTAs
 * per SM are timed over 8 half-steps and the fastest is kept (plan_stats[13]:
 * 0 = per-half-step launches, else the persistent kernel's CTAs per SM); with
 * autotune = 0 the persistent kernel runs at 2 CTAs per SM.
 * Every wait is bounded (1 s); one that runs out ends the launch and the
 * solve reports TREE_OT_ERR_TIMEOUT.  With TREE_OT_OPT_TEST_STALL as well, the
 * node-update items never report completion, so the next waits run out (tests
 * the failure path without a GPU fault).  tree_ot_apply / tree_ot_node_update
 * always launch their own kernels. */
#define TREE_OT_OPT_PERSISTENT  64u
/* Node update bookkeeping.  Each CTA updates a chunk of one node's points;
 * the node's normaliser Z_j, its stopping terms and the problem's stopping
 * quantity (with phase control and retirement) are finished either by the
 * last-arriving chunk (arrival counters: fences and serial atomics on a
 * chunk's way out) or by one extra launch after the chunks (one warp per
 * problem), chosen per colour: the extra launch when the colour has more than
 * four chunks per SM, where the chunks' exit latency outweighs it
 * (plan_stats[14], bit c for colour c).  Same arithmetic either way; these
 * bits force one form for every colour (DEFER wins if both are set). */
#define TREE_OT_OPT_NODE_DEFER  128u
#define TREE_OT_OPT_NODE_ARRIVE 256u
#define TREE_OT_OPT_SK_MMA_SYNC 32u /* shared-kernel BF16 phase: multiply with the legacy
                                       mma.sync kernel instead of tcgen05 (tensor memory
                                       accumulators); for comparison and for devices
                                       without tcgen05                                     */
#define TREE_OT_OPT_SK_ONE_CTA 512u /* the tcgen05 product with one CTA per 128-row tile
                                       instead of CTA pairs of one cluster (256-row MMAs,
                                       each CTA holding half of a tile's V' operand); the
                                       same sums, for comparison                           */

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
    uint32_t flags;           /* TREE_OT_OPT_* bits, 0 by default                        */
    /* APPLY_BF16 only.  The first lowp_start half-steps use the FP32 kernels.
     * Stored costs: the potentials are then absorbed into a BF16 copy of the
     * Gibbs kernel,
     *     Kt(x,y) = 2^(A(x) + B(y) - C(x,y) log2(e)/eps - rho(x))   (row max 1),
     * A, B the apply operands at absorption time, and each apply multiplies Kt
     * by 2^(h - base) on the reduction side (FP32 accumulation).  An edge whose
     * operand drifts more than absorb_tau (log2 units) from its base is
     * re-absorbed on the device.
     * Shared squared-Euclidean kernels: each half-step, one colour's messages of
     * a group are S = K' V' with K'(x,y) = 2^(b(y) - R(x) - s C(x,y)) and
     * V'(y,j) = 2^(h_j(y) - b(y)), b the envelope of the columns' operands and
     * R its row frame, both factors split into two BF16 parts and multiplied on
     * the tensor cores with FP32 accumulation (three products); outputs whose
     * sum falls below 2^-96 are recomputed exactly.
     * A problem leaves the phase for the FP32 kernels for good when its stopping
     * quantity falls below refine_tol, or when it has not fallen by 10 % for 128
     * half-steps; refine_tol = 0 keeps it in the phase (the phase alone). */
    double refine_tol;        /* default 1e-5                                            */
    double absorb_tau;        /* default 48                                              */
    int32_t lowp_start;       /* default 16                                              */
    int32_t autotune;         /* 1 (default): at create, time the recomputed-cost apply for
                                 each tile shape (output block 256/512/1024, CTAs per SM)
                                 and keep the fastest, cached per problem shape; and time
                                 the two stored-cost kernels (see TREE_OT_OPT_DENSE_*)  */
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
    int64_t lowp_half_steps;    /* APPLY_BF16: half-steps spent in the BF16 phase            */
    int64_t absorptions;        /* APPLY_BF16: edge absorptions performed (whole handle)  */
} tree_ot_result;

typedef struct tree_ot_handle tree_ot_handle;

/* Fill *opt with defaults: FP32, AUTO, tol 1e-6 (SUM), cap 100000, check 32, graph on,
 * refine_tol 1e-5, absorb_tau 48, lowp_start 16, autotune on. */
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

/* Validate all problems, build the device plan and upload the data.  Each
 * problem is the coupled bi-marginal problem of Sec. 3 (eq.
 * ot_graph_pairwise_mass: tree, costs C_(j,k), fixed marginals mu_j on leaves,
 * eps) with the inputs of the Bipartite Iterative Scaling algorithm; the
 * stopping threshold delta' and the other controls come in *opt.  Several
 * problems form one batch ("forest"); each converges and retires on its own.
 * Potentials start at zero (u = 1, the algorithm's initialisation); warm starts
 * and checkpoint resumes enter afterwards through tree_ot_set_potentials*.
 * opt may be NULL (defaults).  On failure *out is NULL and nothing is leaked. */
int tree_ot_create(const tree_ot_problem *probs, int32_t num_probs, const tree_ot_options *opt,
                   void *cuda_stream, tree_ot_handle **out);

/* Release every device buffer the handle owns (borrowed inputs are not freed).
 * NULL-safe. */
int tree_ot_destroy(tree_ot_handle *h);

/* Reset every problem to u = 1 and clear iteration counters. */
int tree_ot_reset(tree_ot_handle *h, void *cuda_stream);

/* Iterate from the current state until every problem meets opt->tol or the
 * cap, then run the FP64 check.  A problem retires on the FP32 stopping
 * quantity the half-step kernels accumulate (Algorithm "Bipartite Iterative
 * Scaling"'s while-condition, or its largest term); the FP64-grade check of the
 * returned potentials then certifies it: if the check exceeds tol, the problem
 * resumes with a retirement threshold below the FP32 quantity it retired on,
 * scaled by how far the check missed (8 times at most,
 * and only while each round still lowers the check: FP32 iterates have an
 * accuracy floor, typically 1e-7 to 1e-6 in max marginal L1, that grows as eps
 * shrinks).
 * results: host array [num_probs] (may be NULL).  Returns TREE_OT_NOT_CONVERGED
 * if some problem hit the cap or was not certified. */
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
 * (FP64): B_(j,k_j) 1 for fixed j, the mean of {B_(j,k) 1}_k for free j (the
 * arithmetic mean qbar_j of lemma lem:f_upper_bound_tree; for a star this is
 * the barycenter).  out: host, n_j doubles.  The potentials of the same
 * iterate come from tree_ot_get_potentials. */
int tree_ot_marginals(tree_ot_handle *h, int32_t prob, int32_t node, double *out);

/* History of the stopping quantity (the while-condition of the Bipartite
 * Iterative Scaling algorithm, Sec. 3.1, and its largest term) as the half-step
 * kernels accumulate it in FP32 -- the value problems retire on.  The terms of
 * iterate t (the potentials after t half-steps) are non-zero only on the side
 * the next half-step updates, and that half-step (number t + 1) forms them from
 * the messages it computes anyway; the other side's terms vanish up to
 * rounding (lemma cor:tree_mass and the block updates of thm:tree_dual_var),
 * except at t = 0 (u = 1), where that side is not measured.
 * sum_out[i] / max_out[i] (host, count doubles each; either may be NULL) get
 * the values of iterate first + i.  The last 256 iterates are kept; iterates
 * must satisfy 0 <= first, first + count <= half-steps done, and
 * first >= half-steps done - 256 (else TREE_OT_ERR_ARG).  A problem retired by
 * tree_ot_solve skips later half-steps; its later entries read 0, and a
 * problem resumed by the certification restarts its history.  Synchronises
 * cuda_stream. */
int tree_ot_residual_history(tree_ot_handle *h, void *cuda_stream, int32_t prob, int64_t first, int64_t count,
                             double *sum_out, double *max_out);

/* ---- rounding to feasible plans -------------------------------------------
 * The rounding algorithm of Sec. 3.1 ("Rounding for transport plan on a
 * bipartite graph") with the error bounds of lemmas lem:round and
 * lem:round_applied (Sec. 3.2).  After a half-step the colour class it did not
 * update (S) misses its marginals; every plan B_(j,k) with j in S is rounded by
 * Algorithm 2 of Altschuler, Weed and Rigollet (2017) to row sums t_j and column
 * sums c_k:
 *     x = min(t / B 1, 1),  B' = diag(x) B,  y = min(c / B'^T 1, 1),  B'' = B' diag(y),
 *     B^ = B'' + err_r err_c^T / ||err_r||_1,  err_r = t - B'' 1,  err_c = c - B''^T 1,
 * with t_j = mu_j (j fixed) or qbar_j = mean_k B_(j,k) 1 (j free).  The paper
 * keeps c = B_(j,k)^T 1, which the last half-step made equal to k's marginal;
 * an FP32 iterate matches that only to its own accuracy, so c_k is k's
 * marginal itself (mu_k, or the mean of k's plan marginals), and t and c are
 * taken at unit mass (exactly 1 by lemma cor:tree_mass).  In exact arithmetic
 * y = 1 and this is the paper's rounding; in floating point the rounded plans
 * meet every constraint of the unregularised problem (eq. ot_graph_pairwise:
 * fixed marginals mu_j / sum mu_j, one marginal per free node) to FP64 rounding.
 * Plan entries are the FP64-grade check's (double-float exponent, ~1e-7
 * relative each; FP64 handles: FP64); every sum over them is FP64. */
typedef struct tree_ot_round_result {
    int32_t side;                   /* colour class S that was rounded                    */
    int64_t half_steps;             /* iterate rounded (half-steps applied to the problem) */
    double residual_sum_l1;         /* stopping sum r of the input plans (their FP64 sums) */
    double transport_cost;          /* sum_e <C_e, B_e> of the input plans                 */
    double rounded_transport_cost;  /* sum_e <C_e, B^_e> (+inf if a correction lands on a
                                       +inf cost entry)                                   */
    double c_inf;                   /* max_e max |C_e| over finite entries                 */
    double bound;                   /* 2 eps |E| log(d) + 4 C_inf r, d = max_j n_j: the
                                       bound of lem:round_applied on rounded_transport_cost
                                       minus the unregularised optimum                     */
} tree_ot_round_result;

/* Round the plans of the current potentials of every problem.  side = -1: per
 * problem, the colour its last half-step did not update (a retired problem's
 * last half-step is the one it retired at; a problem with no half-step yet
 * returns TREE_OT_ERR_STATE); side = 0 or 1: that colour class for every
 * problem.  results: host [num_probs] (may be NULL).  The rounded plans are kept
 * implicitly (row scales and rank-one factors, a few vectors per edge) until the
 * potentials next change; buffers are allocated on the first call.
 * Synchronises cuda_stream. */
int tree_ot_round(tree_ot_handle *h, void *cuda_stream, int32_t side, tree_ot_round_result *results);

/* Write the rounded plan of edge `edge` (0 <= edge < J-1) of problem `prob` from
 * the last tree_ot_round into plan_out: DEVICE memory, caller-owned, n_a x ld
 * FP64 row-major with rows on node a = edges[edge][0] (ld >= n_b; entries past
 * n_b are left alone).  TREE_OT_ERR_STATE if the potentials changed since the
 * last tree_ot_round.  Enqueued on cuda_stream; does not synchronise. */
int tree_ot_round_plan(tree_ot_handle *h, void *cuda_stream, int32_t prob, int32_t edge, double *plan_out,
                       int64_t ld);

/* Copy the potential vector of directed edge `dedge` (0 <= dedge < 2(J-1), see
 * the numbering above) of problem p to / from host memory (FP64, n_owner values).
 * set_potentials is how warm starts and checkpoint resumes enter; the free-node
 * dual constraint (sum_k f_(j,k) constant) need not hold for the supplied values. */
int tree_ot_get_potentials(tree_ot_handle *h, void *cuda_stream, int32_t prob, int32_t dedge, double *out);
int tree_ot_set_potentials(tree_ot_handle *h, void *cuda_stream, int32_t prob, int32_t dedge, const double *in);

/* Set many directed-edge potentials at once from DEVICE memory (a predicted
 * warm start lands here without a host round trip).  Item i sets the potential
 * of directed edge dedges[i] of problem probs[i] (host arrays of `count`) to
 * values[i * ld + x], x < n_owner (device FP32, cost units, row stride ld >= the
 * largest n_owner).  All items are checked first: a non-finite value returns
 * TREE_OT_ERR_NONFINITE and changes nothing.  One stream synchronisation per
 * call; the values buffer may be reused once the call returns. */
int tree_ot_set_potentials_batch(tree_ot_handle *h, void *cuda_stream, int32_t count, const int32_t *probs,
                                 const int32_t *dedges, const float *values, int64_t ld);

/* The reverse: values[i * ld + x] = f(x) of directed edge dedges[i] of problem
 * probs[i], x < n_owner, as FP32 cost units into DEVICE memory (ld >= the
 * largest n_owner; entries past n_owner are left alone).  flags & 1: subtract
 * the mean over x (the gauge mean_x f = 0; plans do not depend on the gauge).
 * Enqueued on the stream; returns without synchronising. */
#define TREE_OT_GET_CENTRED 1u
int tree_ot_get_potentials_batch(tree_ot_handle *h, void *cuda_stream, int32_t count, const int32_t *probs,
                                 const int32_t *dedges, float *values, int64_t ld, uint32_t flags);

/* Plan statistics of the handle (host values), first nstats of:
 * [0] directed edges, [1] edges, [2] plan elements per half-step
 * (sum_e n_a n_b: every half-step applies every edge once), [3] stored cost
 * bytes read per half-step (4 sum_e n_a n_b for dense costs, 0 when costs are
 * recomputed), [4] apply tasks of colour 0, [5] of colour 1, [6] device bytes
 * owned by the handle, [7] node-update CTAs of colour 0, [8] of colour 1,
 * [9] output block of recomputed-cost tasks, [10] their CTAs per SM (0 = by
 * occupancy), [11] their kernel register budget (0: 2 CTAs per SM, 1: 3), all
 * as chosen by the autotuner, [12] 1 when stored costs stream through the
 * bulk-copy staged kernel (TREE_OT_OPT_DENSE_TMA or the autotuner's choice),
 * [13] 0 when half-steps run as per-half-step launches, else the persistent
 * forest kernel's CTAs per SM (TREE_OT_OPT_PERSISTENT), [14] bit c set when
 * colour c's node update finishes its bookkeeping in an extra launch
 * (TREE_OT_OPT_NODE_DEFER), [15] the shared-kernel BF16 phase's product: 0
 * no shared-kernel group, 1 mma.sync, 2 tcgen05 with one CTA per 128-row tile,
 * 3 tcgen05 over CTA pairs (TREE_OT_OPT_SK_ONE_CTA, TREE_OT_OPT_SK_MMA_SYNC). */
int tree_ot_plan_stats(tree_ot_handle *h, int64_t *stats, int32_t nstats);

/* Launch timing (no paper counterpart: measurement support).  While enabled,
 * every launch group the handle queues outside CUDA-graph capture (so not the
 * graph chunks of tree_ot_solve) is bracketed by CUDA events on its stream,
 * by category; tree_ot_profile_read waits for the last event, returns per
 * category the summed milliseconds and the number of launch groups, and starts
 * a new record.  Enabling or disabling also clears the record.  Events are
 * created on demand and released by tree_ot_destroy. */
#define TREE_OT_PROF_APPLY_STORED    0  /* stored-cost edge apply (plain-load or staged kernel)   */
#define TREE_OT_PROF_APPLY_RECOMPUTE 1  /* recomputed-cost edge apply (one launch per dimension)  */
#define TREE_OT_PROF_APPLY_BF16      2  /* absorbed BF16 apply                                    */
#define TREE_OT_PROF_SK_BUILD        3  /* shared-kernel phase: envelope, K' and V' builds        */
#define TREE_OT_PROF_SK_PRODUCT      4  /* shared-kernel phase: the tensor-core product           */
#define TREE_OT_PROF_SK_FIXUP        5  /* shared-kernel phase: exact recomputation of underflows */
#define TREE_OT_PROF_NODE_UPDATE     6  /* node update (block updates + stopping terms)          */
#define TREE_OT_PROF_ABSORB          7  /* absorption step                                        */
#define TREE_OT_PROF_CHECK           8  /* FP64-grade check                                       */
#define TREE_OT_PROF_ROUND           9  /* rounding passes                                        */
#define TREE_OT_PROF_APPLY_FP64     10  /* FP64 edge apply                                        */
#define TREE_OT_PROF_FOREST         11  /* persistent forest launch (applies + node updates)      */
#define TREE_OT_PROF_CATEGORIES     12
int tree_ot_profile(tree_ot_handle *h, int32_t enable);
/* ms, launches: host arrays of ncat entries (either may be NULL); synchronises
 * with the recorded work. */
int tree_ot_profile_read(tree_ot_handle *h, double *ms, int64_t *launches, int32_t ncat);

/* Allocation-free apply of one stored cost matrix (the paper has no
 * counterpart: this is a packaging of the edge-apply kernel for callers that
 * cannot allocate device memory -- serving runtimes that own every byte of
 * device memory through a pre-sized pool, plug-ins hosted by such a runtime,
 * or real-time loops that forbid the device-wide synchronisation
 * cudaMalloc/cudaFree can cause).
 *
 *   m_out[x] = log sum_{y < n_cols} exp( g[y] - cost[x * ld + y] / eps ),  x < n_rows
 *
 * Accuracy: every term is formed and summed in FP32 (the argument exact up to
 * its final rounding, as in the solver's apply); the pieces of a row are merged
 * and the logarithm taken in FP64, so m_out carries the FP32 sums' relative
 * error (about 1e-7 of the row's sum, i.e. ~1e-7 absolute in m) and no more.
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

/* ---- warm-start predictor ------------------------------------------------
 * The paper has no counterpart: this is a learned initialisation for the
 * potentials of the leaves of a star (a project extension; the solver itself
 * never depends on it).  A 3-layer MLP,
 *     y = W3 g(W2 g(W1 x + b1) + b2) + b3,   g = GELU (erf form),
 * with FP32 master parameters laid out as [W1 (hidden x in), b1, W2 (hidden x
 * hidden), b2, W3 (out x hidden), b3] (each tensor starting at a multiple of
 * 8 floats; tree_ot_mlp_num_params returns the six offsets), BF16 copies of
 * the weights and BF16 activations feeding tensor-core MMAs with FP32
 * accumulation.  Loss: mean squared error over the batch and outputs.
 * x, y, target, grads are device pointers (row-major batch x dim FP32); get /
 * set_params use host memory (set_params also clears Adam's moments).
 * Not thread-safe per handle.  Errors: tree_ot_mlp_last_error(). */
typedef struct tree_ot_mlp tree_ot_mlp;
int tree_ot_mlp_create(int32_t in_dim, int32_t hidden, int32_t out_dim, int32_t max_batch, uint64_t seed,
                       tree_ot_mlp **out);
int tree_ot_mlp_destroy(tree_ot_mlp *m);
int tree_ot_mlp_num_params(tree_ot_mlp *m, int64_t *n, int64_t *offsets /* [6] or NULL */);
int tree_ot_mlp_get_params(tree_ot_mlp *m, float *host_out);
int tree_ot_mlp_set_params(tree_ot_mlp *m, const float *host_in);
/* Input transform applied inside the first kernel: features 0..count-1 of every
 * row become log(max(x, floor_value)) * scale (default count 0: none). */
int tree_ot_mlp_set_input_log(tree_ot_mlp *m, int32_t count, double floor_value, double scale);
/* y = MLP(x) for batch rows (batch <= max_batch). */
int tree_ot_mlp_forward(tree_ot_mlp *m, void *cuda_stream, const float *x, int32_t batch, float *y);
/* Forward + backward of the MSE loss; grads (device, num_params floats, the
 * parameter layout) and loss (host) may be NULL.  Parameters are unchanged. */
int tree_ot_mlp_backward(tree_ot_mlp *m, void *cuda_stream, const float *x, const float *target, int32_t batch,
                         float *grads, double *loss);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8, bias-corrected) at learning rate lr. */
int tree_ot_mlp_train_step(tree_ot_mlp *m, void *cuda_stream, const float *x, const float *target, int32_t batch,
                           double lr, double *loss);
const char *tree_ot_mlp_last_error(void);

/* ---- General graphs: coupled MOT on a modified junction tree ------------
 * Sec. 4 (def:jt_general, problem eq:ot_graph_local_reg, Assumption
 * ass:inclusion, prop:local_reg_dual and the separator update of
 * prop:general_algo).  Variables 0 .. num_vars-1 with support sizes
 * var_size[v].  Cost clique c has the variables
 * clique_vars[clique_var_begin[c] .. clique_var_begin[c+1]) (the axis order of
 * its cost tensor) and a dense FP32 cost tensor clique_cost[c] (host memory,
 * row-major, the last variable fastest; copied at create; +inf allowed, NaN
 * and -inf rejected).  Separator s has the variables
 * sep_vars[sep_var_begin[s] .. ), its neighbour cliques
 * sep_cliques[sep_clique_begin[s] .. ) in the order of its inclusion sequence
 * (the intersections with the first two cliques equal, the rest nested), and
 * optionally a constraint: the variables sep_gamma[sep_gamma_begin[s] .. )
 * (inside the smallest intersection; none: unconstrained) with the marginal
 * sep_mu[s] (host FP64, row-major over the constraint's variables; NULL when
 * unconstrained).  Every clique must join exactly two separators, and the
 * separators must two-colour through the cliques (TREE_OT_ERR_NOT_TREE
 * otherwise).  A clique holds at most 8 variables.
 * The dual variable u^s_i lives on s n c_i (variables in the separator's
 * order); a half-step updates every separator of one colour (separator 0's
 * colour first), all on the device in FP64 log domain.  The stopping quantity
 * (the paper defines none for Sec. 4; this reading): per separator, the L1
 * distances between the marginals on s n c_i of clique c_i's plan and of clique
 * c_1's, i >= 2, plus the distance of c_1's marginal on the constraint from
 * mu (or |mass - 1| unconstrained); its sum and largest term. */
typedef struct tree_ot_jt_problem {
    int32_t num_vars;
    const int32_t *var_size;          /* [num_vars]                                  */
    int32_t num_cliques;
    const int32_t *clique_var_begin;  /* [num_cliques + 1]                           */
    const int32_t *clique_vars;
    const float *const *clique_cost;  /* [num_cliques] host pointers                 */
    int32_t num_seps;
    const int32_t *sep_var_begin;     /* [num_seps + 1]                              */
    const int32_t *sep_vars;
    const int32_t *sep_clique_begin;  /* [num_seps + 1]                              */
    const int32_t *sep_cliques;
    const int32_t *sep_gamma_begin;   /* [num_seps + 1]                              */
    const int32_t *sep_gamma;
    const double *const *sep_mu;      /* [num_seps] host pointers or NULL            */
    double eps;
} tree_ot_jt_problem;

typedef struct tree_ot_jt_handle tree_ot_jt_handle;

/* Validates, plans the half-steps and uploads costs and marginals; u = 1. */
int tree_ot_jt_create(const tree_ot_jt_problem *prob, void *cuda_stream, tree_ot_jt_handle **out);
int tree_ot_jt_destroy(tree_ot_jt_handle *h);
/* u = 1 again */
int tree_ot_jt_reset(tree_ot_jt_handle *h, void *cuda_stream);
/* T half-steps, colours alternating (prop:general_algo per separator) */
int tree_ot_jt_half_steps(tree_ot_jt_handle *h, void *cuda_stream, int64_t T);
/* the stopping quantity of the current iterate: its sum and largest term */
int tree_ot_jt_residual(tree_ot_jt_handle *h, void *cuda_stream, double *sum, double *max);
/* half-steps in groups of check_every until the stopping quantity (tol_kind
 * TREE_OT_TOL_SUM or _MAX) is below tol or max_half_steps are done; returns
 * TREE_OT_OK or TREE_OT_NOT_CONVERGED, the half-steps done and the quantity */
int tree_ot_jt_solve(tree_ot_jt_handle *h, void *cuda_stream, double tol, int32_t tol_kind, int64_t max_half_steps,
                     int32_t check_every, int64_t *half_steps, double *residual);
/* clique c's plan B_c (prop:local_reg_dual) into host memory, in the axis
 * order of its cost tensor */
int tree_ot_jt_plan(tree_ot_jt_handle *h, void *cuda_stream, int32_t clique, double *plan);
/* sum_c <C_c, B_c> */
int tree_ot_jt_transport_cost(tree_ot_jt_handle *h, void *cuda_stream, double *cost);
/* log u^s_i (s = sep, i = pos in its clique list) into host memory, over
 * s n c_i in the separator's variable order */
int tree_ot_jt_get_dual(tree_ot_jt_handle *h, void *cuda_stream, int32_t sep, int32_t pos, double *log_u);
/* the two-colouring: colour[s] for every separator (host) */
int tree_ot_jt_colour(tree_ot_jt_handle *h, int32_t *colour);

#ifdef __cplusplus
}
#endif
#endif /* TREE_OT_H */
