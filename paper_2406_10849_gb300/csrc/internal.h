// Internal plan structures shared by the host planner (api.cpp) and the CUDA
// kernels.  Plain structs of POD fields and device pointers; no torch types.
//
// Vocabulary (Sec. 3 of the paper): a directed edge (j -> k) is owned by node
// j and carries the potential f_(j,k) = eps log u_(j,k) (length n_j).  The
// "message" of that directed edge is
//     m_(j,k)(x) = LSE_y [ (f_(k,j)(y) - C_(j,k)(x,y)) / eps + log gamma_k(y) ],
// the log of K_(j,k)(u_(k,j) gamma_k) that the block updates (thm:tree_dual_var) divide by.  A
// half-step on colour c computes the messages of every directed edge whose
// owner has colour c (edge apply), then applies those updates at the owners
// (node update).
#pragma once
#include <string>
#include <cstdint>
#include <cuda_runtime.h>

namespace treeot {

constexpr double kLog2e = 1.4426950408889634074;
constexpr double kLn2 = 0.69314718055994530942;
constexpr int kResidRing = 256;        // residual history slots (half-steps) kept on device
constexpr int kApplyThreads = 256;     // 8 warps per apply CTA
constexpr int kRowCols = 1024;         // ROW task: columns per task (32 lanes x 4 x 8)
constexpr int kRowRowsPerWarp = 8;     // ROW task: rows per warp (task = 64 rows)
constexpr int kColCols = 128;          // COL task: columns per task (32 lanes x 4)
constexpr int kColRows = 512;          // COL task: rows per task (8 warps x 64)
constexpr int kRecOut = 1024;          // RECOMP task: outputs per task (256 threads x 4)
constexpr int kRecRed = 512;           // RECOMP task: reduction points per task
constexpr int kNodeThreads = 256;
// node update: (owned edge, point) pairs per CTA.  Larger chunks amortise a
// CTA's dependent metadata loads over more pairs: on 2000 stars the node update
// took 0.347 / 0.297 / 0.274 ms per half-step at 1024 / 2048 / 4096 pairs, on
// the 512 batched trees 0.363 / 0.325 / 0.329 ms; but a colour with few pairs
// (the 64-node tree: 32 leaves of 4096 points) needs the smaller chunks to
// fill the GPU at all (its node update took 0.106 against 0.045 ms).
constexpr int kNodePairs = 4096;
constexpr int kNodePairsSmall = 1024;
constexpr int kBfCols = 256;           // BF16 COL task: columns per task (32 lanes x 8)
constexpr int kBfRowTask = 256;        // BF16 ROW task: rows per task
constexpr double kGrid = 1024.0;       // apply operands and frames live on a 2^-10 grid
constexpr int64_t kLowpStall = 128;    // a BF16 phase whose stopping quantity has not fallen by 10 %
                                       // for this many half-steps hands the problem to FP32

enum TaskKind : int32_t {
  TASK_ROW = 0,     // stored matrix, owner is the row node: reduce along a row
  TASK_COL = 1,     // stored matrix, owner is the column node: reduce down columns
  TASK_RECOMP = 2,  // squared-Euclidean cost recomputed from coordinates
};

struct DEdgeD {
  int64_t off;       // owner-side vector offset in the f / m / h arenas (length n_owner)
  int64_t rev_off;   // offset of the reverse directed edge's vectors (length n_nbr)
  int64_t part_off;  // partial (split s, output x) lives at part_off + s * n_owner + x
  int32_t owner, nbr;  // global node ids
  int32_t edge;        // global undirected edge id
  int32_t dir;         // 0: owner is the row node of the stored matrix, 1: column node
  int32_t nsplit;      // number of partial log-sum-exp pieces per output
  int32_t prob;        // problem id
};

struct EdgeD {
  const float* C;   // dense cost, rows = node a, row stride ld (multiple of 4); pad columns +inf
  int64_t ld;
  const float* CT;  // its transpose (rows = node b, stride ldt, +inf pads) or null
  int64_t ldt;
  uint16_t* K;      // absorbed BF16 Gibbs kernel (low-precision mode), row stride ldk (multiple of 8)
  int64_t ldk;
  int32_t a, b;     // global node ids (rows a, columns b)
  int32_t na, nb;
};

struct NodeD {
  int64_t node_off;   // node-level vectors (log gamma, mu), length n
  int64_t coord_off;  // coordinates, n x dim floats (or -1)
  int32_t n, deg, prob, fixed;
  int32_t dedge_begin;  // owned directed edges: node_dedges[dedge_begin .. dedge_begin+deg)
  int32_t colour;
  int32_t chunk_base;   // node-update chunks of this node: zpart[chunk_base .. +nchunks)
  int32_t nchunks;
};

struct NodeChunk {
  int32_t node, chunk, x0, cnt;
};

// Node update: points per CTA for a node of n points and degree deg, so that a
// CTA holds at most `pairs` (edge, point) pairs (a multiple of 32 points when
// that is at least 32, and at least one point).
inline int32_t node_chunk_points(int32_t n, int32_t deg, int32_t pairs) {
  int32_t c = pairs / (deg > 0 ? deg : 1);
  if (c >= 32) c &= ~31;
  if (c < 1) c = 1;
  return c < n ? c : n;
}

// A directed edge of a shared-kernel group (BF16 phase): where the product of
// its colour leaves the message's sum S(x) (one float per output; negative
// where the output was listed for the exact fix-up, which writes (frame, sum)
// to the partials instead), the group's row frames R(x) and the column's
// maximum M_j; the message is R(x) + M_j + log2 S(x) (log2 units).
struct SkRefD {
  const float* s;
  const float* rf;
  const float* cm;
};
// A fixed leaf's node-update chunk with its node and its one owned directed edge
// resolved on the host (the fixed-leaf kernel's fast path: the chunk's loads
// depend on one load of this record).
struct FixedChunkD {
  int64_t d_off, part_off, node_off;  // the directed edge's vectors, its partials, the node's vectors
  int32_t node, x0, cnt, n;           // node, first point, points, support size
  int32_t prob, di, nbr, edge;        // problem, directed edge, neighbour node, edge
  int32_t nsplit, cost_kind;
  double eps_ln2;
  SkRefD sk;                          // shared-kernel references (null pointers outside a group)
};

// the same, as a node-update CTA keeps it (the column maximum read once)
struct SkEdgeS {
  const float* s;
  const float* rf;
  float cm, pad;
};

// Node update: dynamic shared memory of one CTA (deg edges, cnt points), in
// this order: edge records, neighbour normalisers, edge ids, drift flags,
// per-edge stopping sums, shared-kernel references, per-pair messages and q,
// per-point s and mean q.  q and the sums are double for FP64 handles, float
// otherwise.
struct NodeSmem {
  uint32_t de, zn, di, dr, r, sk, mi, q, s, qb, bytes;
};
__host__ __device__ inline uint32_t node_align16(uint32_t b) { return (b + 15u) & ~15u; }
__host__ __device__ inline NodeSmem node_smem_layout(int32_t deg, int32_t cnt, bool f64) {
  const uint32_t qs = f64 ? 8u : 4u, np = (uint32_t)deg * (uint32_t)cnt;
  NodeSmem L;
  L.de = 0;
  L.zn = L.de + node_align16((uint32_t)deg * (uint32_t)sizeof(DEdgeD));
  L.di = L.zn + node_align16((uint32_t)deg * 8u);
  L.dr = L.di + node_align16((uint32_t)deg * 4u);
  L.r = L.dr + node_align16((uint32_t)deg * 4u);
  L.sk = L.r + node_align16((uint32_t)deg * qs);
  L.mi = L.sk + node_align16((uint32_t)deg * (uint32_t)sizeof(SkEdgeS));
  L.q = L.mi + node_align16(np * 8u);
  L.s = L.q + node_align16(np * qs);
  L.qb = L.s + node_align16((uint32_t)cnt * 8u);
  L.bytes = L.qb + node_align16((uint32_t)cnt * qs);
  return L;
}
// FP32 free nodes of degree at most kNodePmDeg take the point-major update in
// the shared-kernel phase (one thread per point, all of its edges in
// registers): of the layout above it uses the per-edge tables and s, placed
// where the per-pair arrays start, node_smem_pm_bytes in all (the launch
// reserves the full layout: outside the phase the same chunk is pair-major)
constexpr int kNodePmDeg = 8;
__host__ __device__ inline uint32_t node_smem_pm_bytes(int32_t deg, int32_t cnt) {
  return node_smem_layout(deg, cnt, false).mi + node_align16((uint32_t)cnt * 8u);
}

struct ProbD {
  double eps, inv_eps;
  double cost_scale;
  float s2, s2_lo;                 // log2(e) / eps as a two-float (hi + lo)
  float s2_scaled, s2_scaled_lo;   // cost_scale * log2(e) / eps (recompute), two-float
  int32_t dim;
  int32_t cost_kind;
  int32_t nodes_in_colour[2];
  int32_t edge_begin, edge_count;  // global ids of this problem's edges
};

struct Task {
  int32_t dedge, kind;
  int32_t o0, ocount;   // output range (owner support)
  int32_t r0, rcount;   // reduction range (neighbour support)
  int32_t split;
  int32_t pad;          // RECOMP: warp groups sharing the task (1, 2, 4, 8); ROW: 1 = rows of CT
};

// A stored-cost (ROW / COL) task with every address resolved on the host, for
// the bulk-copy staged kernel.  The tile's stage rows are C + r * ld: output
// rows for ROW tasks, reduction rows for COL tasks.
struct StreamTask {
  const float* C;      // first element of the tile
  int64_t ld;          // row stride of the cost (floats, multiple of 4)
  int64_t m_off;       // frame sources m[m_off + i], i < ocount
  int64_t h_off;       // reduction-side operand hh / hl[h_off + j], j < rcount
  int64_t out_off;     // partials part32[out_off + i], i < ocount
  int32_t kind, prob;
  int32_t ocount, rcount;
  float s2, s2_lo;     // log2(e) / eps as a two-float
};

struct ApplyArgs {
  const Task* tasks;
  int32_t ntasks;
  const DEdgeD* dedges;
  const EdgeD* edges;
  const NodeD* nodes;
  const ProbD* probs;
  const int32_t* done;       // per problem: 1 = retired
  const float* fr;           // frames of the latest messages: log2 on the 2^-10 grid (0 if not finite)
  const float* hh;           // operand (f/eps + log gamma) * log2(e), high part
  const float* hl;           // low part
  const double* f;           // potentials (FP64 path)
  const double* logg;        // node log gamma (FP64 path)
  const float* coords;
  const float* coords_hi;    // coordinates split hi + lo (hi on the problem's 2^-10 sigma grid)
  const float* coords_lo;
  const int32_t* exact;      // per problem: 1 = recompute costs with exact squared distances
  int32_t any_exact;         // host: some problem has exact set (selects the kernel instantiation)
  float2* part32;            // FP32 path partials: (frame R, sum) in base 2
  double2* part64;           // FP64 path partials: (max M, sum S) in base e
  int32_t* queue;            // work-queue counters of this launch (next task, CTAs finished)
  // low-precision (absorbed) phase
  const int32_t* lowp;       // per problem: 1 = BF16 phase (the FP32 kernels skip it), else FP32
  const float* bh;           // absorbed bases (operand at absorption), high / low parts
  const float* bl;
  const float* arho;         // row normalisers of the absorbed kernels (row side of each edge)
  int32_t* err;              // error word: bit 1 = a bounded wait of a staged kernel ran out
  const StreamTask* stasks;  // staged kernel: resolved stored-cost tasks (ntasks of them)
  int32_t test_stall;        // staged kernel: the producer issues nothing (tests the timeout path)
  const int32_t* fp32_live;  // problems the FP32 kernels still process (not retired, not in a BF16
                             // phase); 0 = the launch has nothing to do (null: always run)
};

struct AbsorbArgs {
  const Task* tasks;         // (dedge 2e, rows o0..o0+ocount) blocks of every stored-cost edge
  int32_t ntasks;
  const DEdgeD* dedges;
  const EdgeD* edges;
  const ProbD* probs;
  const float* hh;
  const float* hl;
  float* bh;
  float* bl;
  float* arho;
  const int32_t* lowp;
  int32_t* drift;            // per edge: 1 = re-absorb
  int32_t nedges;
  unsigned long long* count; // edge absorptions performed
};

// Potentials are stored in a normalised form: f[d] holds f'_(j,k) with the
// free-node constant split off, f_(j,k) = f'_(j,k) - eps * Z[j] (Z = 0 for
// fixed nodes), where Z_j = LSE_x s_j(x) and rho_j = -|N(j)| Z_j (thm:tree_dual_var).
// h[d] = (f'/eps + log gamma_owner) * log2(e); the apply therefore returns the
// message plus Z of the neighbour, which the node update subtracts.
struct NodeArgs {
  const NodeChunk* chunks;   // CTAs of this launch: (node, chunk) pairs of the colour
  int32_t nchunks;
  uint32_t smem;             // dynamic shared memory per CTA (the largest chunk of the colour)
  int32_t colour;
  const NodeD* nodes;
  const DEdgeD* dedges;
  const int32_t* node_dedges;
  const ProbD* probs;
  int32_t nprob;
  int32_t* done;
  int64_t* done_at;
  double* f;
  float* fr;                 // frame of the merged message for the next apply (log2, 2^-10 grid)
  float* hh;
  float* hl;
  double* Z;                 // per node
  double* rho;               // per node
  const float2* part32;
  const double2* part64;
  const double* logg;
  const double* mu;
  const float4* lgf;         // FP32 path, per node point: log2 mu as (hi on the grid, lo), mu, 0
  double2* zpart;            // per node chunk: (max, sum) of the chunk's s values
  double* resid_acc;         // per directed edge: stopping term being accumulated
  double* resid_dedge;       // per directed edge: latest complete stopping term
  double* res_sum;           // [kResidRing][nprob]
  unsigned long long* res_max;  // [kResidRing][nprob], bit pattern of a non-negative double
  int32_t* node_arrive;      // per node: chunks finished in this launch
  int32_t* node_count;       // per problem: nodes finished in this launch
  int32_t* launch_count;     // CTAs finished in this launch
  int64_t* hs;               // half-steps completed (device counter)
  int32_t* err;              // device error flags (bit 0: non-finite potential)
  double tol;
  const double* ptol;        // per problem: the retirement threshold (tol, tightened by certification)
  const int64_t* deadline;   // per problem: retire at this half-step at the latest (resumed problems)
  int32_t tol_kind;
  int32_t retire;            // 1: retire problems whose stopping quantity < tol
  // low-precision phase control (absorbed != 0 only for handles built for it)
  int32_t absorbed;
  int32_t* lowp;             // per problem: 2 = waiting for lowp_start, 1 = BF16 phase, 0 = FP32
  const float* bh;
  const float* bl;
  int32_t* drift;            // per edge
  double refine_tol;
  float tau;                 // drift limit (log2 units)
  int32_t lowp_start;
  int64_t* lowp_span;        // per problem: half-steps at which the BF16 phase began / ended (-1: not yet)
  double* lowp_best;         // per problem: smallest stopping quantity seen in the BF16 phase
  int64_t* lowp_best_t;      // per problem: the half-step of that last improvement
  int32_t* fp32_live;        // count of problems the FP32 applies process (kept by the last node
                             // of a problem as it retires or enters / leaves a BF16 phase; may be null)
  int32_t count_launch;      // 1: the last CTA of the launch advances the half-step counter
  int32_t defer;             // 1: chunks leave the arrival bookkeeping to node_finish_kernel
  const SkRefD* sk_ref;      // per directed edge, for problems in the shared-kernel phase (or null)
  const FixedChunkD* fixed;  // per chunk of a fixed-leaf launch with deferred bookkeeping (or null)
};

// Per problem, what node_finish_kernel reads for one colour: the directed
// edges owned by the colour's nodes (dedges[dbeg[p] .. dbeg[p+1])) and its
// free nodes (nodes[nbeg[p] .. nbeg[p+1])).
struct FinishList {
  const int32_t* dbeg;
  const int32_t* dedges;
  const int32_t* nbeg;
  const int32_t* nodes;
};

// FP64-grade check of the current potentials.  Per element the exponent
// a(x) + b(y) - C(x,y)/eps is formed in double-float (pairs of FP32 values with
// error-free transformations) and exponentiated with an accurate FP32 expf,
// so every plan entry carries ~1e-7 relative error, uncorrelated across
// entries (FP64 proper runs at a small fraction of the FP32 rate here).
struct CheckArgs {
  const Task* tasks;   // kind ROW: rows of edge e, owner a; kind COL: columns, owner b
  int32_t ntasks;
  const DEdgeD* dedges;
  const EdgeD* edges;
  const NodeD* nodes;
  const ProbD* probs;
  const float* ah;     // per directed edge: a = f/eps + log gamma_owner, high FP32 part
  const float* al;     // low part
  const double* f;     // FP64 check: potentials f' (with Z and log gamma read directly)
  const double* Z;
  const double* logg;
  const float* coords;
  double* marg;        // per directed edge: B 1 on the owner's side (layout of f)
  double* edge_tc;     // per edge sum C B
  double* edge_mass;   // per edge sum B
  const int32_t* mask; // per problem: 0 = skip its tasks (null: check every problem)
};

// ---- launchers (defined in the .cu files) --------------------------------
// slot 0: stored-cost tasks (ROW/COL); slot D (1..3): recomputed squared-Euclidean tasks
// variant (recomputed costs): 0 = 2 CTAs per SM register budget, 1 = 3 CTAs per SM
cudaError_t launch_apply_f32(const ApplyArgs& a, int slot, int variant, int grid, cudaStream_t s);
// stored-cost (slot 0) tasks with bulk-copy staged rows; one CTA per SM, grid = SM count
bool apply_tma_available();
cudaError_t launch_apply_tma(const ApplyArgs& a, int grid, cudaStream_t s);
cudaError_t launch_apply_f64(const ApplyArgs& a, int grid, cudaStream_t s);
// fixed_only: every chunk of the launch belongs to a fixed node (a kernel without
// the free-node path, so more CTAs fit on an SM)
// the message tree_ot_last_error returns (thread-local; api.cpp)
void set_last_error(const std::string& msg);

cudaError_t launch_node_update(const NodeArgs& a, bool fp64, bool fixed_only, cudaStream_t s);
// the deferred bookkeeping of a node update of one colour (one warp per problem)
cudaError_t launch_node_finish(const NodeArgs& a, const FinishList& l, cudaStream_t s);
// *out = number of problems with done == 0 and lowp != 1 (lowp may be null: all count)
cudaError_t launch_count_live(const int32_t* done, const int32_t* lowp, int32_t nprob, int32_t* out, cudaStream_t s);
// FP32 handles: the stored potentials f from the operand (hh, hl) and log2 mu
cudaError_t launch_materialise_f(const DEdgeD* dedges, int32_t ndedges, const NodeD* nodes, const ProbD* probs,
                                 const float4* lgf, const float* hh, const float* hl, double* f, cudaStream_t s);
// v = (f'/eps - Z_owner + log gamma) * scale as FP32 (hi, lo); Z may be null.
// quantize: hi on the 2^-10 grid (the apply operand), else hi = nearest float.
cudaError_t launch_set_potentials(const float* values, int64_t ld, const int32_t* dlist, int32_t count,
                                  const DEdgeD* dedges, const NodeD* nodes, const ProbD* probs, const double* Z,
                                  double* f, DEdgeD* picked, int32_t* bad, bool write, cudaStream_t s);
cudaError_t launch_get_potentials(const int32_t* dlist, int32_t count, const DEdgeD* dedges, const NodeD* nodes,
                                  const ProbD* probs, const double* Z, const double* f, float* values, int64_t ld,
                                  bool centred, cudaStream_t s);
cudaError_t launch_operand(const double* f, const double* Z, const double* logg, const DEdgeD* dedges,
                           const NodeD* nodes, const ProbD* probs, int32_t ndedges, double scale, bool quantize,
                           float* vh, float* vl, cudaStream_t s);
cudaError_t launch_check64(const CheckArgs& a, cudaStream_t s);
cudaError_t launch_scan_cost(const float* C, int64_t ld, int32_t rows, int32_t cols, int32_t* bad, cudaStream_t s);
// dst (cols x dst_ld) = transpose of src (rows x src_ld, first cols columns), +inf pads
cudaError_t launch_transpose_pad(const float* src, int64_t src_ld, int32_t rows, int32_t cols, float* dst,
                                 int64_t dst_ld, cudaStream_t s);
// coordinates split hi + lo for the exact-distance recomputation (cmax: nprob scratch words)
cudaError_t launch_split_coords(const float* coords, const NodeD* nodes, int32_t nnodes, const ProbD* probs,
                                uint32_t* cmax, int32_t nprob, float* hi, float* lo, cudaStream_t s);
cudaError_t launch_check(const CheckArgs& a, cudaStream_t s);
cudaError_t launch_fill_f32(float* p, int64_t n, float v, cudaStream_t s);
cudaError_t launch_pad_copy(const float* src, int64_t src_ld, float* dst, int64_t dst_ld, int32_t rows,
                            int32_t cols, cudaStream_t s);
int apply_ctas_per_sm(int slot, int variant);
int apply_bf16_ctas_per_sm();
cudaError_t launch_apply_bf16(const ApplyArgs& a, int grid, cudaStream_t s);
cudaError_t launch_absorb(const AbsorbArgs& a, int grid, cudaStream_t s);
// allocation-free single-matrix row apply (scratch in a file-scope device array)
cudaError_t noalloc_scratch(float** out, int64_t* capacity_floats);
int64_t noalloc_scratch_floats_needed(int32_t n_rows, int32_t n_cols);
cudaError_t launch_edge_apply_noalloc(const float* C, int64_t ld, int32_t n_rows, int32_t n_cols, const double* g,
                                      float shi, float slo, double* m_out, float* scratch, cudaStream_t s);
constexpr int kApplySlots = 4;

}  // namespace treeot

namespace treeot {
// ---- warm-start MLP kernels (mlp.cu) ---------------------------------------
cudaError_t mlp_gemm(const void* A, int lda, int ta, const void* B, int ldb, int tb, float* C, int ldc, int M, int N,
                     int K, const float* bias, int accumulate, cudaStream_t s);
cudaError_t mlp_gelu_fwd(const float* z, void* a16, int64_t n, cudaStream_t s);
cudaError_t mlp_gelu_bwd(const float* da, const float* z, void* dz16, float* dz32, int64_t n, cudaStream_t s);
cudaError_t mlp_to_bf16(const float* x, void* y, int64_t n, cudaStream_t s);
cudaError_t mlp_input(const float* x, void* y, int64_t rows, int cols, int nlog, float floor_, float scale,
                      cudaStream_t s);
cudaError_t mlp_mse(const float* y, const float* t, float* dy32, void* dy16, int64_t n, double* loss, cudaStream_t s);
cudaError_t mlp_colsum(const float* dz, int M, int N, float* db, cudaStream_t s);
cudaError_t mlp_adam(float* w, const float* g, float* m1, float* m2, void* w16, int64_t n, float lr, float b1, float b2,
                     float eps, float c1, float c2, cudaStream_t s);
}  // namespace treeot
