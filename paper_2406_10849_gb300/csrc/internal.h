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
constexpr int kNodeChunk = 512;        // node update: support points per CTA
constexpr double kGrid = 1024.0;       // apply operands and frames live on a 2^-10 grid

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

struct ProbD {
  double eps, inv_eps;
  double cost_scale;
  float s2, s2_lo;                 // log2(e) / eps as a two-float (hi + lo)
  float s2_scaled, s2_scaled_lo;   // cost_scale * log2(e) / eps (recompute), two-float
  int32_t dim;
  int32_t cost_kind;
  int32_t nodes_in_colour[2];
};

struct Task {
  int32_t dedge, kind;
  int32_t o0, ocount;   // output range (owner support)
  int32_t r0, rcount;   // reduction range (neighbour support)
  int32_t split, pad;
};

struct ApplyArgs {
  const Task* tasks;
  int32_t ntasks;
  const DEdgeD* dedges;
  const EdgeD* edges;
  const NodeD* nodes;
  const ProbD* probs;
  const int32_t* done;       // per problem: 1 = retired
  const double* m;           // latest messages (frames for the next apply)
  const float* hh;           // operand (f/eps + log gamma) * log2(e), high part
  const float* hl;           // low part
  const double* f;           // potentials (FP64 path)
  const double* logg;        // node log gamma (FP64 path)
  const float* coords;
  float2* part32;            // FP32 path partials: (frame R, sum) in base 2
  double2* part64;           // FP64 path partials: (max M, sum S) in base e
};

// Potentials are stored in a normalised form: f[d] holds f'_(j,k) with the
// free-node constant split off, f_(j,k) = f'_(j,k) - eps * Z[j] (Z = 0 for
// fixed nodes), where Z_j = LSE_x s_j(x) and rho_j = -|N(j)| Z_j (thm:tree_dual_var).
// h[d] = (f'/eps + log gamma_owner) * log2(e); the apply therefore returns the
// message plus Z of the neighbour, which the node update subtracts.
struct NodeArgs {
  const NodeChunk* chunks;   // CTAs of this launch: (node, chunk) pairs of the colour
  int32_t nchunks;
  int32_t colour;
  const NodeD* nodes;
  const DEdgeD* dedges;
  const int32_t* node_dedges;
  const ProbD* probs;
  int32_t nprob;
  int32_t* done;
  int64_t* done_at;
  double* f;
  double* m;                 // raw merged message (before subtracting Z of the neighbour)
  float* hh;
  float* hl;
  double* Z;                 // per node
  double* rho;               // per node
  const float2* part32;
  const double2* part64;
  const double* logg;
  const double* mu;
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
  int32_t tol_kind;
  int32_t retire;            // 1: retire problems whose stopping quantity < tol
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
};

// ---- launchers (defined in the .cu files) --------------------------------
// slot 0: stored-cost tasks (ROW/COL); slot D (1..3): recomputed squared-Euclidean tasks
cudaError_t launch_apply_f32(const ApplyArgs& a, int slot, int grid, cudaStream_t s);
cudaError_t launch_apply_f64(const ApplyArgs& a, int grid, cudaStream_t s);
cudaError_t launch_node_update(const NodeArgs& a, bool fp64, cudaStream_t s);
// v = (f'/eps - Z_owner + log gamma) * scale as FP32 (hi, lo); Z may be null.
// quantize: hi on the 2^-10 grid (the apply operand), else hi = nearest float.
cudaError_t launch_operand(const double* f, const double* Z, const double* logg, const DEdgeD* dedges,
                           const NodeD* nodes, const ProbD* probs, int32_t ndedges, double scale, bool quantize,
                           float* vh, float* vl, cudaStream_t s);
cudaError_t launch_check64(const CheckArgs& a, cudaStream_t s);
cudaError_t launch_scan_cost(const float* C, int64_t ld, int32_t rows, int32_t cols, int32_t* bad, cudaStream_t s);
cudaError_t launch_check(const CheckArgs& a, cudaStream_t s);
cudaError_t launch_fill_f32(float* p, int64_t n, float v, cudaStream_t s);
cudaError_t launch_pad_copy(const float* src, int64_t src_ld, float* dst, int64_t dst_ld, int32_t rows,
                            int32_t cols, cudaStream_t s);
int apply_ctas_per_sm(int slot);
// allocation-free single-matrix row apply (scratch in a file-scope device array)
cudaError_t noalloc_scratch(float** out, int64_t* capacity_floats);
int64_t noalloc_scratch_floats_needed(int32_t n_rows, int32_t n_cols);
cudaError_t launch_edge_apply_noalloc(const float* C, int64_t ld, int32_t n_rows, int32_t n_cols, const double* g,
                                      float shi, float slo, double* m_out, float* scratch, cudaStream_t s);
constexpr int kApplySlots = 4;

}  // namespace treeot
