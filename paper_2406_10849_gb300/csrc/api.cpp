// C ABI of the tree solver: validation, two-colouring, device plan, the solve
// loop (CUDA-graph chunks of half-steps with device-side retirement), and the
// host side of the final check.  See include/tree_ot.h for the contract.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <deque>
#include <limits>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/tree_ot.h"
#include "forest.h"
#include "internal.h"
#include "round.h"
#include "sk.h"

using namespace treeot;

namespace {

// node update: the largest dynamic shared memory a CTA may take (a chunk needs
// about 12 KB plus 70-90 bytes per edge of its node)
constexpr uint32_t kNodeSmemMax = 200u * 1024;

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? TREE_OT_ERR_OOM : TREE_OT_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define CUDA_TRY(call)                                 \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

int64_t align_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

// v = hi + lo with hi the largest float strictly below v, so lo > 0: with an
// infinite cost c the apply's second product c * lo then stays -inf (a zero or
// negative lo would turn inf * lo into NaN)
void split_positive(double v, float* hi, float* lo) {
  float h = (float)v;
  if ((double)h >= v) h = std::nextafter(h, 0.0f);
  *hi = h;
  *lo = (float)(v - (double)h);
  if (!(*lo > 0.0f)) *lo = std::numeric_limits<float>::denorm_min();
}

// ---------------------------------------------------------------------------
// host-only checks (Sec. 3 assumptions)
// ---------------------------------------------------------------------------

int check_tree(int32_t J, const int32_t* edges, std::vector<std::vector<int32_t>>* adj_out) {
  if (J < 2) return fail(TREE_OT_ERR_NOT_TREE, "a tree needs at least two nodes");
  if (!edges) return fail(TREE_OT_ERR_ARG, "edges is NULL");
  std::vector<std::vector<int32_t>> adj(J);
  for (int32_t e = 0; e < J - 1; ++e) {
    const int32_t a = edges[2 * e], b = edges[2 * e + 1];
    if (a < 0 || b < 0 || a >= J || b >= J || a == b)
      return fail(TREE_OT_ERR_NOT_TREE, "edge " + std::to_string(e) + " has an invalid endpoint or is a self loop");
    adj[a].push_back(b);
    adj[b].push_back(a);
  }
  std::vector<uint8_t> seen(J, 0);
  std::deque<int32_t> q{0};
  seen[0] = 1;
  int32_t count = 1;
  while (!q.empty()) {
    const int32_t v = q.front();
    q.pop_front();
    for (int32_t w : adj[v])
      if (!seen[w]) {
        seen[w] = 1;
        ++count;
        q.push_back(w);
      }
  }
  // J-1 edges + connected <=> tree (also rules out duplicate edges / cycles)
  if (count != J) return fail(TREE_OT_ERR_NOT_TREE, "the edges do not connect all nodes (cycle or forest)");
  if (adj_out) *adj_out = std::move(adj);
  return TREE_OT_OK;
}

void colour_tree(int32_t J, const std::vector<std::vector<int32_t>>& adj, uint8_t* colour) {
  std::vector<int8_t> c(J, -1);
  c[0] = 0;
  std::deque<int32_t> q{0};
  while (!q.empty()) {
    const int32_t v = q.front();
    q.pop_front();
    for (int32_t w : adj[v])
      if (c[w] < 0) {
        c[w] = (int8_t)(1 - c[v]);
        q.push_back(w);
      }
  }
  for (int32_t j = 0; j < J; ++j) colour[j] = (uint8_t)c[j];
}

int validate_problem(const tree_ot_problem* p, std::vector<std::vector<int32_t>>* adj_out) {
  if (!p) return fail(TREE_OT_ERR_ARG, "problem is NULL");
  if (!p->support_size || !p->is_fixed) return fail(TREE_OT_ERR_ARG, "support_size / is_fixed is NULL");
  std::vector<std::vector<int32_t>> adj;
  int rc = check_tree(p->num_nodes, p->edges, &adj);
  if (rc) return rc;
  const int32_t J = p->num_nodes;
  for (int32_t j = 0; j < J; ++j)
    if (p->support_size[j] < 1) return fail(TREE_OT_ERR_ARG, "support size of node " + std::to_string(j) + " < 1");
  if (!(p->eps > 0.0) || !std::isfinite(p->eps)) return fail(TREE_OT_ERR_EPS, "eps must be positive and finite");
  for (int32_t j = 0; j < J; ++j) {
    if (!p->is_fixed[j]) continue;
    if (adj[j].size() != 1) return fail(TREE_OT_ERR_FIXED_NOT_LEAF, "fixed node " + std::to_string(j) + " is not a leaf");
    if (p->is_fixed[adj[j][0]])
      return fail(TREE_OT_ERR_FIXED_ADJACENT,
                  "edge joins fixed nodes " + std::to_string(j) + " and " + std::to_string(adj[j][0]));
    if (!p->marginal || !p->marginal[j]) return fail(TREE_OT_ERR_ARG, "marginal of fixed node " + std::to_string(j) + " is NULL");
    double s = 0.0;
    for (int32_t x = 0; x < p->support_size[j]; ++x) {
      const double v = p->marginal[j][x];
      if (!(v >= 0.0) || !std::isfinite(v))
        return fail(TREE_OT_ERR_MARGINAL, "marginal of node " + std::to_string(j) + " has a negative or non-finite entry");
      s += v;
    }
    if (std::fabs(s - 1.0) > 1e-9)
      return fail(TREE_OT_ERR_MARGINAL, "marginal of node " + std::to_string(j) + " does not sum to 1");
  }
  if (p->cost_kind == TREE_OT_COST_SQEUCLID) {
    if (p->dim < 1 || p->dim > 3) return fail(TREE_OT_ERR_ARG, "dim must be 1..3 for the squared-Euclidean cost");
    if (!p->coords) return fail(TREE_OT_ERR_ARG, "coords is NULL");
    for (int32_t j = 0; j < J; ++j)
      if (!p->coords[j]) return fail(TREE_OT_ERR_ARG, "coords of node " + std::to_string(j) + " is NULL");
    if (!(p->cost_scale > 0.0) || !std::isfinite(p->cost_scale)) return fail(TREE_OT_ERR_ARG, "cost_scale must be > 0");
    if (!(p->flags & TREE_OT_INPUT_DEVICE)) {
      for (int32_t j = 0; j < J; ++j)
        for (int64_t i = 0; i < (int64_t)p->support_size[j] * p->dim; ++i)
          if (!std::isfinite(p->coords[j][i]))
            return fail(TREE_OT_ERR_NONFINITE, "coordinates of node " + std::to_string(j) + " are not finite");
    }
  } else if (p->cost_kind == TREE_OT_COST_DENSE_F32) {
    if (!p->dense_cost) return fail(TREE_OT_ERR_ARG, "dense_cost is NULL");
    for (int32_t e = 0; e < J - 1; ++e)
      if (!p->dense_cost[e]) return fail(TREE_OT_ERR_ARG, "dense cost of edge " + std::to_string(e) + " is NULL");
    if (p->coords && (p->dim < 0 || p->dim > 3)) return fail(TREE_OT_ERR_ARG, "dim must be 0..3");
  } else {
    return fail(TREE_OT_ERR_ARG, "unknown cost_kind");
  }
  if (adj_out) *adj_out = std::move(adj);
  return TREE_OT_OK;
}

}  // namespace

void treeot::set_last_error(const std::string& msg) { g_err = msg; }


// ---------------------------------------------------------------------------
// the handle
// ---------------------------------------------------------------------------

struct tree_ot_handle {
  tree_ot_options opt{};
  bool fp64 = false;
  int nprob = 0;
  std::vector<ProbD> probs;
  std::vector<NodeD> nodes;
  std::vector<EdgeD> edges;
  std::vector<DEdgeD> dedges;
  std::vector<int32_t> node_dedges;
  std::vector<Task> tasks[2];              // per colour, grouped by kernel slot
  int32_t slot_begin[2][kApplySlots] = {};
  int32_t slot_count[2][kApplySlots] = {};
  std::vector<NodeChunk> chunks[2];
  uint32_t node_smem[2] = {0, 0};  // node update: dynamic shared memory per CTA, per colour
  std::vector<Task> check_tasks;
  std::vector<Task> btasks[2];             // absorbed BF16 apply tasks per colour
  std::vector<Task> atasks;                // absorption blocks (dedge 2e, 64 rows)
  bool lowp = false;                       // handle built for a BF16 phase (absorbed or shared-kernel)
  // shared-kernel BF16 phase (squared-Euclidean costs): groups of directed edges
  // with one Gibbs kernel, their columns per colour, and the problems all of
  // whose directed edges are grouped (only those enter the phase)
  struct SkGroup {
    std::vector<SkCol> cols[2];
    int32_t owner_rep = 0, nbr_rep = 0, prob_rep = 0;  // representative nodes / problem
    SkArgs args[2]{};
    SkMaps maps[2]{};  // tensor maps of the tcgen05 product's operands, per colour
  };
  std::vector<SkGroup> sk;
  std::vector<uint8_t> sk_prob;
  std::vector<int32_t> prob_node_base, prob_edge_base, prob_nodes;
  std::vector<std::vector<double>> mu;  // per global node (fixed nodes), host copy
  int64_t vec_len = 0, node_len = 0, part_len = 0, coord_len = 0;
  int32_t nzchunks = 0;
  int64_t elems = 0, matrix_bytes = 0, device_bytes = 0;

  ProbD* d_probs = nullptr;
  NodeD* d_nodes = nullptr;
  EdgeD* d_edges = nullptr;
  DEdgeD* d_dedges = nullptr;
  int32_t* d_node_dedges = nullptr;
  Task* d_tasks[2] = {nullptr, nullptr};
  NodeChunk* d_chunks[2] = {nullptr, nullptr};
  Task* d_check_tasks = nullptr;
  Task* d_btasks[2] = {nullptr, nullptr};
  int32_t* d_queue = nullptr;              // [colour][slot][2] work-queue counters
  int32_t rec_ob = kRecOut;                // recomputed-cost output block (autotuned)
  int32_t grid_mult = 0;                   // 0: occupancy-derived grid; else CTAs per SM (autotuned)
  int32_t rec_variant = 0;                 // recomputed-cost kernel register budget (autotuned)
  int32_t dense_tma = 0;                   // stored-cost tasks on the bulk-copy staged kernel
  bool use_ct = false;                     // stored costs also kept transposed (column owners stream rows)
  StreamTask* d_stasks[2] = {nullptr, nullptr};  // slot-0 tasks of each colour, resolved for that kernel
  void* d_setbuf = nullptr;                // batched potential set: directed-edge list + records
  int64_t setbuf_cap = 0;                  // items d_setbuf holds
  int rec_grid[2][kApplySlots] = {};       // occupancy-derived grids per variant
  int64_t task_cap[2] = {0, 0};            // device capacity of d_tasks
  Task* d_atasks = nullptr;
  int32_t *d_lowp = nullptr, *d_drift = nullptr;
  int64_t* d_lowp_span = nullptr;          // per problem: [begin, end) half-steps of the BF16 phase (-1: none)
  double* d_lowp_best = nullptr;           // per problem: the phase's stall detector (node update)
  int64_t* d_lowp_best_t = nullptr;
  unsigned long long* d_absorb_count = nullptr;
  std::vector<int64_t> h_lowp_span;
  unsigned long long h_absorb_count = 0;
  float *d_bh = nullptr, *d_bl = nullptr, *d_arho = nullptr;
  int bf16_grid = 1;
  float* d_fr = nullptr;                   // frames of the messages (FP32, log2 on the 2^-10 grid)
  double *d_f = nullptr, *d_Z = nullptr, *d_rho = nullptr, *d_logg = nullptr, *d_mu = nullptr;
  float4* d_lgf = nullptr;                 // per node point: log2 mu (hi on the grid, lo), mu (FP32 node update)
  double *d_resid_acc = nullptr, *d_resid_dedge = nullptr, *d_res_sum = nullptr, *d_marg = nullptr;
  double *d_edge_tc = nullptr, *d_edge_mass = nullptr;
  float *d_hh = nullptr, *d_hl = nullptr, *d_ah = nullptr, *d_al = nullptr, *d_coords = nullptr;
  float *d_coords_hi = nullptr, *d_coords_lo = nullptr;  // coordinates split hi + lo (exact distances)
  uint32_t* d_cmax = nullptr;              // per problem max |coordinate| (split scratch)
  int32_t* d_exact = nullptr;              // per problem: exact squared distances (recomputed costs)
  std::vector<int32_t> h_exact;
  int32_t any_exact = 0;
  float2* d_part32 = nullptr;
  double2* d_part64 = nullptr;
  double2* d_zpart = nullptr;
  unsigned long long* d_res_max = nullptr;
  int32_t *d_done = nullptr, *d_node_arrive = nullptr, *d_node_count = nullptr, *d_launch_count = nullptr;
  int32_t *d_err = nullptr, *d_scan = nullptr, *d_chk_mask = nullptr;
  int64_t *d_done_at = nullptr, *d_hs = nullptr;
  double* d_ptol = nullptr;                // per-problem retirement threshold
  std::vector<double> h_ptol;
  int64_t* d_deadline = nullptr;           // per-problem latest retirement half-step
  std::vector<int64_t> h_deadline;
  std::vector<void*> owned;
  // rounding (tree_ot_round): buffers allocated on first use, the last rounding's tasks
  double *d_rsum = nullptr, *d_rtgt = nullptr, *d_rxy = nullptr, *d_rs2 = nullptr, *d_rer = nullptr;
  double *d_racc = nullptr, *d_rnmass = nullptr;
  int32_t* d_rside = nullptr;
  RoundTask* d_rtasks = nullptr;
  int64_t rtask_cap = 0;
  std::vector<RoundTask> rtasks;
  std::vector<int32_t> rt_begin, rt_count;  // per edge: its tasks in rtasks
  // launch timing (tree_ot_profile): CUDA events around launches queued outside graph capture
  bool prof_on = false, prof_capturing = false;
  std::vector<cudaEvent_t> prof_ev;
  size_t prof_used = 0;
  struct Span {
    int32_t cat, i0, i1;
  };
  std::vector<Span> prof_spans;
  // persistent forest launch (TREE_OT_OPT_PERSISTENT): 0 = off, else the register
  // budget in CTAs per SM (2 or 3) the create-time timing chose
  int32_t* d_live = nullptr;               // problems the FP32 applies process (see ApplyArgs::fp32_live)
  int32_t nfixed_chunks[2] = {0, 0};       // per colour: its first chunks belong to fixed nodes
  bool node_defer[2] = {false, false};     // per colour: bookkeeping in node_finish_kernel
  int32_t chunk_pairs[2] = {0, 0};         // per colour: (edge, point) pairs per node-update chunk
  SkRefD* d_skref = nullptr;               // per directed edge: its shared-kernel product's output
  FixedChunkD* d_fixed[2] = {nullptr, nullptr};  // per colour: records of its fixed-leaf chunks
  int32_t* d_fin[2] = {nullptr, nullptr};  // per colour: the FinishList arrays, one allocation
  FinishList fin[2] = {};
  int persistent = 0;
  int forest_D = 0;
  uint32_t forest_smem = 0;
  int forest_grid[2] = {0, 0};             // grids at 2 and 3 CTAs per SM
  int forest_grid_exact = 0;
  int32_t *d_fcnt = nullptr, *d_fdone = nullptr, *d_fctl = nullptr;
  int64_t pot_version = 0;                  // bumped by every call that changes potentials
  int64_t round_version = -1;               // pot_version the last rounding saw

  int64_t hs_host = 0;
  cudaStream_t hstream = nullptr;
  cudaGraphExec_t graph = nullptr;
  int graph_len = 0;
  int apply_grid[kApplySlots] = {1, 1, 1, 1};
  int sms = 1;

  bool have_check = false;
  bool f_stale = false;  // FP32 handles: the node update has advanced the operand past d_f
  std::vector<double> h_marg, h_f, h_Z, h_rho, h_tc, h_mass;
  std::vector<int32_t> h_done;
  std::vector<int64_t> h_done_at;
  double last_wall_ms = 0.0;
  std::vector<int32_t> last_status;

  template <class T>
  int alloc(T** p, int64_t count) {
    *p = nullptr;
    if (count <= 0) count = 1;
    const size_t bytes = sizeof(T) * (size_t)count;
    cudaError_t e = cudaMalloc((void**)p, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    owned.push_back(*p);
    device_bytes += (int64_t)bytes;
    return TREE_OT_OK;
  }
};

namespace {

#define RC_TRY(call)      \
  do {                    \
    int rc_ = (call);     \
    if (rc_) return rc_;  \
  } while (0)

// ---- launch timing ----------------------------------------------------------
// an event of the pool (created on demand); -1 when timing is off or capturing
int prof_take(tree_ot_handle* h) {
  if (!h->prof_on || h->prof_capturing) return -1;
  if (h->prof_used == h->prof_ev.size()) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    h->prof_ev.push_back(e);
  }
  return (int)h->prof_used++;
}
int prof_mark(tree_ot_handle* h, cudaStream_t s) {
  const int i = prof_take(h);
  if (i >= 0 && cudaEventRecord(h->prof_ev[i], s) != cudaSuccess) return -1;
  return i;
}
void prof_span(tree_ot_handle* h, int cat, int i0, int i1) {
  if (i0 >= 0 && i1 >= 0) h->prof_spans.push_back({cat, i0, i1});
}
cudaEvent_t prof_event(tree_ot_handle* h, int i) { return i >= 0 ? h->prof_ev[i] : nullptr; }

// Apply tasks of both colours, grouped by kernel slot.  rec_ob: largest output
// block of a recomputed-cost task (256, 512 or 1024 outputs); a task with fewer
// outputs runs its CTA as G warp groups splitting the reduction points.
void build_apply_tasks(tree_ot_handle* h, int32_t rec_ob) {
  for (int c = 0; c < 2; ++c) {
    h->tasks[c].clear();
    for (int s2 = 0; s2 < kApplySlots; ++s2) h->slot_begin[c][s2] = h->slot_count[c][s2] = 0;
  }
  for (size_t di = 0; di < h->dedges.size(); ++di) {
    const DEdgeD& d = h->dedges[di];
    const NodeD& own = h->nodes[d.owner];
    const NodeD& nbn = h->nodes[d.nbr];
    const ProbD& pd = h->probs[d.prob];
    std::vector<Task>& tl = h->tasks[own.colour];
    const bool dense = pd.cost_kind == TREE_OT_COST_DENSE_F32;
    if (h->fp64) {
      for (int32_t o0 = 0; o0 < own.n; o0 += 64)
        tl.push_back(Task{(int32_t)di, dense ? (d.dir == 0 ? TASK_ROW : TASK_COL) : TASK_RECOMP, o0,
                          std::min(64, own.n - o0), 0, nbn.n, 0, 0});
    } else if (dense && (d.dir == 0 || h->use_ct)) {
      // rows of C (owner = row node) or of its transpose (owner = column node; pad = 1)
      for (int32_t o0 = 0; o0 < own.n; o0 += 8 * kRowRowsPerWarp)
        for (int32_t s = 0; s < d.nsplit; ++s)
          tl.push_back(Task{(int32_t)di, TASK_ROW, o0, std::min(8 * kRowRowsPerWarp, own.n - o0), s * kRowCols,
                            std::min(kRowCols, nbn.n - s * kRowCols), s, d.dir == 0 ? 0 : 1});
    } else if (dense) {
      for (int32_t s = 0; s < d.nsplit; ++s)
        for (int32_t o0 = 0; o0 < own.n; o0 += kColCols)
          tl.push_back(Task{(int32_t)di, TASK_COL, o0, std::min(kColCols, own.n - o0), s * kColRows,
                            std::min(kColRows, nbn.n - s * kColRows), s, 0});
    } else {
      for (int32_t o0 = 0; o0 < own.n; o0 += rec_ob) {
        const int32_t oc = std::min(rec_ob, own.n - o0);
        int32_t G = 1;
        while (G < 8 && kRecOut / (2 * G) >= oc) G *= 2;
        for (int32_t s = 0; s < d.nsplit; ++s)
          tl.push_back(Task{(int32_t)di, TASK_RECOMP, o0, oc, s * kRecRed, std::min(kRecRed, nbn.n - s * kRecRed), s,
                            G});
      }
    }
  }
  // group each colour's tasks by kernel slot (stored costs; recomputed costs by
  // dimension); recomputed tasks go largest first for the work queue
  for (int c = 0; c < 2; ++c) {
    auto slot_of = [&](const Task& t) {
      if (h->fp64 || t.kind != TASK_RECOMP) return 0;
      return (int)h->probs[h->dedges[t.dedge].prob].dim;
    };
    auto cost_of = [&](const Task& t) { return (int64_t)t.ocount * t.rcount; };
    std::stable_sort(h->tasks[c].begin(), h->tasks[c].end(), [&](const Task& x, const Task& y) {
      const int sx = slot_of(x), sy = slot_of(y);
      if (sx != sy) return sx < sy;
      return sx != 0 && cost_of(x) > cost_of(y);
    });
    for (const Task& t : h->tasks[c]) h->slot_count[c][slot_of(t)] += 1;
    int32_t b = 0;
    for (int s2 = 0; s2 < kApplySlots; ++s2) {
      h->slot_begin[c][s2] = b;
      b += h->slot_count[c][s2];
    }
  }
  h->rec_ob = rec_ob;
}

ApplyArgs apply_args(tree_ot_handle* h, int colour) {
  ApplyArgs a{};
  a.tasks = h->d_tasks[colour];
  a.ntasks = (int32_t)h->tasks[colour].size();
  a.dedges = h->d_dedges;
  a.edges = h->d_edges;
  a.nodes = h->d_nodes;
  a.probs = h->d_probs;
  a.done = h->d_done;
  a.fr = h->d_fr;
  a.hh = h->d_hh;
  a.hl = h->d_hl;
  a.f = h->d_f;
  a.logg = h->d_logg;
  a.coords = h->d_coords;
  a.coords_hi = h->d_coords_hi;
  a.coords_lo = h->d_coords_lo;
  a.exact = h->d_exact;
  a.any_exact = h->any_exact;
  a.part32 = h->d_part32;
  a.part64 = h->d_part64;
  a.lowp = h->d_lowp;
  a.bh = h->d_bh;
  a.bl = h->d_bl;
  a.arho = h->d_arho;
  a.err = h->d_err;
  a.test_stall = (h->opt.flags & TREE_OT_OPT_TEST_STALL) ? 1 : 0;
  a.fp32_live = h->fp64 ? nullptr : h->d_live;
  return a;
}

NodeArgs node_args(tree_ot_handle* h, int colour, bool retire) {
  NodeArgs a{};
  a.chunks = h->d_chunks[colour];
  a.nchunks = (int32_t)h->chunks[colour].size();
  a.smem = h->node_smem[colour];
  a.colour = colour;
  a.nodes = h->d_nodes;
  a.dedges = h->d_dedges;
  a.node_dedges = h->d_node_dedges;
  a.probs = h->d_probs;
  a.nprob = h->nprob;
  a.done = h->d_done;
  a.done_at = h->d_done_at;
  a.f = h->d_f;
  a.fr = h->d_fr;
  a.hh = h->d_hh;
  a.hl = h->d_hl;
  a.Z = h->d_Z;
  a.rho = h->d_rho;
  a.part32 = h->d_part32;
  a.part64 = h->d_part64;
  a.logg = h->d_logg;
  a.mu = h->d_mu;
  a.lgf = h->d_lgf;
  a.zpart = h->d_zpart;
  a.resid_acc = h->d_resid_acc;
  a.resid_dedge = h->d_resid_dedge;
  a.res_sum = h->d_res_sum;
  a.res_max = h->d_res_max;
  a.node_arrive = h->d_node_arrive;
  a.node_count = h->d_node_count;
  a.launch_count = h->d_launch_count;
  a.hs = h->d_hs;
  a.err = h->d_err;
  a.tol = h->opt.tol;
  a.ptol = h->d_ptol;
  a.deadline = h->d_deadline;
  a.tol_kind = h->opt.tol_kind;
  a.retire = retire ? 1 : 0;
  a.absorbed = h->lowp ? 1 : 0;
  a.lowp = h->d_lowp;
  a.bh = h->d_bh;
  a.bl = h->d_bl;
  a.drift = h->d_drift;
  a.refine_tol = h->opt.refine_tol;
  a.tau = (float)h->opt.absorb_tau;
  a.sk_ref = h->d_skref;
  a.lowp_start = h->opt.lowp_start;
  a.lowp_span = h->d_lowp_span;
  a.lowp_best = h->d_lowp_best;
  a.lowp_best_t = h->d_lowp_best_t;
  a.fp32_live = h->fp64 ? nullptr : h->d_live;
  a.count_launch = 1;
  return a;
}

AbsorbArgs absorb_args(tree_ot_handle* h) {
  AbsorbArgs a{};
  a.tasks = h->d_atasks;
  a.ntasks = (int32_t)h->atasks.size();
  a.dedges = h->d_dedges;
  a.edges = h->d_edges;
  a.probs = h->d_probs;
  a.hh = h->d_hh;
  a.hl = h->d_hl;
  a.bh = h->d_bh;
  a.bl = h->d_bl;
  a.arho = h->d_arho;
  a.lowp = h->d_lowp;
  a.drift = h->d_drift;
  a.nedges = (int32_t)h->edges.size();
  a.count = h->d_absorb_count;
  return a;
}

int launch_absorb_step(tree_ot_handle* h, cudaStream_t s) {
  if (!h->lowp) return TREE_OT_OK;
  AbsorbArgs a = absorb_args(h);
  const int grid = std::max(1, std::min<int>(a.ntasks, h->bf16_grid));
  const int p0 = prof_mark(h, s);
  cudaError_t e = launch_absorb(a, grid, s);
  if (e != cudaSuccess) return cuda_fail(e, "absorption launch");
  prof_span(h, TREE_OT_PROF_ABSORB, p0, prof_mark(h, s));
  return TREE_OT_OK;
}

// only_stored: just the stored-cost (slot 0) kernel, for timing it
int launch_apply(tree_ot_handle* h, int colour, cudaStream_t s, bool only_stored = false) {
  ApplyArgs a = apply_args(h, colour);
  if (h->fp64) {
    const int grid = std::max(1, std::min<int>(a.ntasks, h->apply_grid[0]));
    const int p0 = prof_mark(h, s);
    cudaError_t e = launch_apply_f64(a, grid, s);
    if (e != cudaSuccess) return cuda_fail(e, "edge apply launch");
    prof_span(h, TREE_OT_PROF_APPLY_FP64, p0, prof_mark(h, s));
    return TREE_OT_OK;
  }
  for (int slot = 0; slot < (only_stored ? 1 : kApplySlots); ++slot) {
    const int32_t cnt = h->slot_count[colour][slot];
    if (cnt == 0) continue;
    a.tasks = h->d_tasks[colour] + h->slot_begin[colour][slot];
    a.ntasks = cnt;
    a.queue = h->d_queue + 2 * (colour * kApplySlots + slot);
    const int p0 = prof_mark(h, s);
    if (slot == 0 && h->dense_tma) {
      a.stasks = h->d_stasks[colour];
      cudaError_t e = launch_apply_tma(a, std::max(1, std::min<int>(cnt, h->sms)), s);
      if (e != cudaSuccess) return cuda_fail(e, "staged edge apply launch");
      prof_span(h, TREE_OT_PROF_APPLY_STORED, p0, prof_mark(h, s));
      continue;
    }
    int cap = slot == 0 ? h->apply_grid[0] : h->rec_grid[h->rec_variant][slot];
    if (slot > 0 && h->grid_mult > 0) cap = h->sms * h->grid_mult;
    const int grid = std::max(1, std::min<int>(cnt, cap));
    cudaError_t e = launch_apply_f32(a, slot, slot == 0 ? 0 : h->rec_variant, grid, s);
    if (e != cudaSuccess) return cuda_fail(e, "edge apply launch");
    prof_span(h, slot == 0 ? TREE_OT_PROF_APPLY_STORED : TREE_OT_PROF_APPLY_RECOMPUTE, p0, prof_mark(h, s));
  }
  if (h->lowp && !only_stored && !h->btasks[colour].empty()) {
    a.tasks = h->d_btasks[colour];
    a.ntasks = (int32_t)h->btasks[colour].size();
    const int grid = std::max(1, std::min<int>(a.ntasks, h->bf16_grid));
    const int p0 = prof_mark(h, s);
    cudaError_t e = launch_apply_bf16(a, grid, s);
    if (e != cudaSuccess) return cuda_fail(e, "absorbed apply launch");
    prof_span(h, TREE_OT_PROF_APPLY_BF16, p0, prof_mark(h, s));
  }
  if (!only_stored)
    for (const auto& g : h->sk) {
      const int p0 = prof_mark(h, s), m0 = prof_take(h), m1 = prof_take(h);
      cudaError_t e = launch_sk(g.args[colour], g.args[colour].use_tc ? &g.maps[colour] : nullptr, s,
                                prof_event(h, m0), prof_event(h, m1));
      if (e != cudaSuccess) return cuda_fail(e, "shared-kernel apply launch");
      const int p1 = prof_mark(h, s);
      prof_span(h, TREE_OT_PROF_SK_BUILD, p0, m0);
      prof_span(h, TREE_OT_PROF_SK_PRODUCT, m0, m1);
      prof_span(h, TREE_OT_PROF_SK_FIXUP, m1, p1);
    }
  return TREE_OT_OK;
}

int launch_update(tree_ot_handle* h, int colour, bool retire, cudaStream_t s) {
  const int p0 = prof_mark(h, s);
  NodeArgs a = node_args(h, colour, retire);
  const int32_t nf = h->nfixed_chunks[colour], nall = a.nchunks;
  const bool defer = h->node_defer[colour];
  a.defer = defer ? 1 : 0;
  cudaError_t e = cudaSuccess;
  // The kernel without the free-node path takes the fixed nodes' chunks (listed
  // first) when they fill the GPU on their own, or when there is nothing else;
  // otherwise one launch takes every chunk (two half-empty launches back to
  // back cost more than the leaner kernel saves).
  const bool all_fixed = nf > 0 && nf == nall;
  const bool split = nf > 0 && nf < nall && nf >= 4 * h->sms;
  if (split) {
    a.nchunks = nf;
    a.count_launch = 0;
    a.fixed = defer ? h->d_fixed[colour] : nullptr;
    e = launch_node_update(a, h->fp64, true, s);
    a.fixed = nullptr;
  }
  if (e == cudaSuccess && nall > 0) {
    const int32_t first = split ? nf : 0;
    a.chunks = h->d_chunks[colour] + first;
    a.nchunks = nall - first;
    a.count_launch = defer ? 0 : 1;
    a.fixed = (all_fixed && defer) ? h->d_fixed[colour] : nullptr;
    e = launch_node_update(a, h->fp64, all_fixed, s);
    a.fixed = nullptr;
  }
  if (e == cudaSuccess && defer) {  // the bookkeeping; its last CTA advances the half-step counter
    a.count_launch = 1;
    e = launch_node_finish(a, h->fin[colour], s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "node update launch");
  prof_span(h, TREE_OT_PROF_NODE_UPDATE, p0, prof_mark(h, s));
  if (!h->fp64) h->f_stale = true;
  return TREE_OT_OK;
}

// d_f up to date before anything reads or partly overwrites it (FP32 handles
// keep the potentials in the operand between node updates)
int sync_potentials(tree_ot_handle* h, cudaStream_t s) {
  if (!h->f_stale) return TREE_OT_OK;
  CUDA_TRY(launch_materialise_f(h->d_dedges, (int32_t)h->dedges.size(), h->d_nodes, h->d_probs, h->d_lgf, h->d_hh,
                                h->d_hl, h->d_f, s));
  h->f_stale = false;
  return TREE_OT_OK;
}

// one persistent launch of G half-steps (the forest kernel; see forest.cu)
int launch_forest_chunk(tree_ot_handle* h, int G, bool retire, cudaStream_t s) {
  ForestArgs f{};
  for (int c = 0; c < 2; ++c) {
    f.ap[c] = apply_args(h, c);
    f.ap[c].tasks = h->d_tasks[c] + h->slot_begin[c][h->forest_D];
    f.ap[c].ntasks = h->slot_count[c][h->forest_D];
    f.nd[c] = node_args(h, c, retire);
  }
  f.cnt = h->d_fcnt;
  f.app_done = h->d_fdone;
  f.nod_done = h->d_fdone + h->nprob;
  f.ctl = h->d_fctl;
  f.err = h->d_err;
  f.hs = h->d_hs;
  f.nprob = h->nprob;
  f.G = G;
  f.c0 = (int32_t)(h->hs_host % 2);
  f.test_stall = (h->opt.flags & TREE_OT_OPT_TEST_STALL) ? 1 : 0;
  const bool exact = h->any_exact != 0;
  const int grid = exact ? h->forest_grid_exact : h->forest_grid[h->persistent == 3 ? 1 : 0];
  const int p0 = prof_mark(h, s);
  cudaError_t e = launch_forest(f, h->forest_D, exact, exact ? 2 : h->persistent, h->forest_smem, grid, s);
  if (e != cudaSuccess) return cuda_fail(e, "persistent forest launch");
  prof_span(h, TREE_OT_PROF_FOREST, p0, prof_mark(h, s));
  h->f_stale = true;  // the node updates advanced the operand past the stored potentials
  return TREE_OT_OK;
}

// the count of problems the FP32 applies process, from the done and phase flags
// (after the host changes either)
int recount_live(tree_ot_handle* h, cudaStream_t s) {
  if (h->fp64) return TREE_OT_OK;
  CUDA_TRY(launch_count_live(h->d_done, h->lowp ? h->d_lowp : nullptr, h->nprob, h->d_live, s));
  return TREE_OT_OK;
}

int queue_half_steps(tree_ot_handle* h, int64_t T, bool retire, cudaStream_t s) {
  if (h->persistent) {
    while (T > 0) {
      const int G = (int)std::min<int64_t>(T, 64);
      RC_TRY(launch_forest_chunk(h, G, retire, s));
      h->hs_host += G;
      T -= G;
    }
    return TREE_OT_OK;
  }
  for (int64_t i = 0; i < T; ++i) {
    const int colour = (int)(h->hs_host % 2);
    RC_TRY(launch_apply(h, colour, s));
    RC_TRY(launch_update(h, colour, retire, s));
    RC_TRY(launch_absorb_step(h, s));
    ++h->hs_host;
  }
  return TREE_OT_OK;
}

int reset_state(tree_ot_handle* h, cudaStream_t s) {
  CUDA_TRY(cudaMemsetAsync(h->d_f, 0, sizeof(double) * h->vec_len, s));
  CUDA_TRY(cudaMemsetAsync(h->d_fr, 0, sizeof(float) * h->vec_len, s));
  CUDA_TRY(cudaMemsetAsync(h->d_Z, 0, sizeof(double) * h->nodes.size(), s));
  CUDA_TRY(cudaMemsetAsync(h->d_rho, 0, sizeof(double) * h->nodes.size(), s));
  CUDA_TRY(cudaMemsetAsync(h->d_resid_acc, 0, sizeof(double) * h->dedges.size(), s));
  CUDA_TRY(cudaMemsetAsync(h->d_resid_dedge, 0, sizeof(double) * h->dedges.size(), s));
  CUDA_TRY(cudaMemsetAsync(h->d_res_sum, 0, sizeof(double) * kResidRing * h->nprob, s));
  h->h_ptol.assign(h->nprob, h->opt.tol);
  CUDA_TRY(cudaMemcpyAsync(h->d_ptol, h->h_ptol.data(), sizeof(double) * h->nprob, cudaMemcpyHostToDevice, s));
  h->h_deadline.assign(h->nprob, INT64_MAX);
  CUDA_TRY(
      cudaMemcpyAsync(h->d_deadline, h->h_deadline.data(), sizeof(int64_t) * h->nprob, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaStreamSynchronize(s));  // h_ptol may be rewritten by the next solve
  CUDA_TRY(cudaMemsetAsync(h->d_res_max, 0, sizeof(unsigned long long) * kResidRing * h->nprob, s));
  CUDA_TRY(cudaMemsetAsync(h->d_done, 0, sizeof(int32_t) * h->nprob, s));
  {
    // exact squared distances from the start only when the option asks for them
    const bool force = (h->opt.flags & TREE_OT_OPT_EXACT_DIST) != 0;
    h->h_exact.assign(h->nprob, 0);
    for (int p = 0; p < h->nprob; ++p)
      h->h_exact[p] = force && h->probs[p].cost_kind == TREE_OT_COST_SQEUCLID ? 1 : 0;
    const int32_t any = *std::max_element(h->h_exact.begin(), h->h_exact.end());
    if (any != h->any_exact && h->graph) {  // the captured launches pick the kernel instantiation
      cudaGraphExecDestroy(h->graph);
      h->graph = nullptr;
    }
    h->any_exact = any;
    CUDA_TRY(cudaMemcpyAsync(h->d_exact, h->h_exact.data(), sizeof(int32_t) * h->nprob, cudaMemcpyHostToDevice, s));
  }
  CUDA_TRY(cudaMemsetAsync(h->d_done_at, 0, sizeof(int64_t) * h->nprob, s));
  CUDA_TRY(cudaMemsetAsync(h->d_node_arrive, 0, sizeof(int32_t) * h->nodes.size(), s));
  CUDA_TRY(cudaMemsetAsync(h->d_node_count, 0, sizeof(int32_t) * h->nprob, s));
  CUDA_TRY(cudaMemsetAsync(h->d_launch_count, 0, sizeof(int32_t), s));
  CUDA_TRY(cudaMemsetAsync(h->d_hs, 0, sizeof(int64_t), s));
  CUDA_TRY(cudaMemsetAsync(h->d_err, 0, sizeof(int32_t), s));
  CUDA_TRY(cudaMemsetAsync(h->d_queue, 0, sizeof(int32_t) * 2 * 2 * kApplySlots, s));
  if (h->d_fdone) {  // the persistent launch's counters (its last CTA leaves them at zero)
    CUDA_TRY(cudaMemsetAsync(h->d_fdone, 0, sizeof(int32_t) * 2 * h->nprob, s));
    CUDA_TRY(cudaMemsetAsync(h->d_fctl, 0, sizeof(int32_t) * 2, s));
  }
  // apply operand of u = 1: h = log gamma * log2(e)
  CUDA_TRY(launch_operand(h->d_f, nullptr, h->d_logg, h->d_dedges, h->d_nodes, h->d_probs, (int32_t)h->dedges.size(),
                          kLog2e, true, h->d_hh, h->d_hl, s));
  h->f_stale = false;
  // phase of every problem: absorbed BF16 phase (1), waiting for it (2), or FP32 (0)
  CUDA_TRY(cudaMemsetAsync(h->d_absorb_count, 0, sizeof(unsigned long long), s));
  {
    std::vector<int32_t> lp(h->nprob, 0);
    std::vector<int32_t> dr(h->edges.size(), 0);
    std::vector<int64_t> span(2 * h->nprob, -1), best_t(h->nprob, 0);
    std::vector<double> best(h->nprob, INFINITY);
    for (int p = 0; p < h->nprob; ++p) {
      const bool sk = !h->sk_prob.empty() && h->sk_prob[p];
      if (!h->lowp || (h->probs[p].cost_kind != TREE_OT_COST_DENSE_F32 && !sk)) continue;
      lp[p] = h->opt.lowp_start == 0 ? 1 : 2;
      if (lp[p] == 1) {
        span[2 * p] = 0;
        for (int k = 0; k < h->probs[p].edge_count; ++k) dr[h->probs[p].edge_begin + k] = 1;
      }
    }
    CUDA_TRY(cudaMemcpyAsync(h->d_lowp, lp.data(), sizeof(int32_t) * lp.size(), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(h->d_drift, dr.data(), sizeof(int32_t) * dr.size(), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(h->d_lowp_span, span.data(), sizeof(int64_t) * span.size(), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(h->d_lowp_best, best.data(), sizeof(double) * best.size(), cudaMemcpyHostToDevice, s));
    CUDA_TRY(
        cudaMemcpyAsync(h->d_lowp_best_t, best_t.data(), sizeof(int64_t) * best_t.size(), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    RC_TRY(launch_absorb_step(h, s));
  }
  RC_TRY(recount_live(h, s));
  h->hs_host = 0;
  h->have_check = false;
  return TREE_OT_OK;
}

int build_graph(tree_ot_handle* h, int len) {
  if (h->graph && h->graph_len == len) return TREE_OT_OK;
  if (h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  CUDA_TRY(cudaStreamBeginCapture(h->hstream, cudaStreamCaptureModeThreadLocal));
  const int64_t saved = h->hs_host;
  h->hs_host = 0;
  h->prof_capturing = true;
  int rc = queue_half_steps(h, len, true, h->hstream);
  h->prof_capturing = false;
  h->hs_host = saved;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(h->hstream, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&h->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  h->graph_len = len;
  return TREE_OT_OK;
}

// FP64-grade check of the current potentials.  only (optional, per problem):
// check just the flagged problems and keep the other problems' last results.
int run_check(tree_ot_handle* h, cudaStream_t s, const std::vector<int32_t>* only = nullptr) {
  const int32_t nd = (int32_t)h->dedges.size();
  const bool partial = only != nullptr && h->have_check;
  std::vector<double> keep_marg, keep_tc, keep_mass;
  if (partial) {
    keep_marg = h->h_marg;
    keep_tc = h->h_tc;
    keep_mass = h->h_mass;
    CUDA_TRY(cudaMemcpyAsync(h->d_chk_mask, only->data(), sizeof(int32_t) * h->nprob, cudaMemcpyHostToDevice, s));
  }
  RC_TRY(sync_potentials(h, s));
  CUDA_TRY(launch_operand(h->d_f, h->d_Z, h->d_logg, h->d_dedges, h->d_nodes, h->d_probs, nd, 1.0, false, h->d_ah,
                          h->d_al, s));
  CUDA_TRY(cudaMemsetAsync(h->d_edge_tc, 0, sizeof(double) * h->edges.size(), s));
  CUDA_TRY(cudaMemsetAsync(h->d_edge_mass, 0, sizeof(double) * h->edges.size(), s));
  CUDA_TRY(cudaMemsetAsync(h->d_marg, 0, sizeof(double) * h->vec_len, s));
  CheckArgs c{};
  c.tasks = h->d_check_tasks;
  c.ntasks = (int32_t)h->check_tasks.size();
  c.dedges = h->d_dedges;
  c.edges = h->d_edges;
  c.nodes = h->d_nodes;
  c.probs = h->d_probs;
  c.ah = h->d_ah;
  c.al = h->d_al;
  c.f = h->d_f;
  c.Z = h->d_Z;
  c.logg = h->d_logg;
  c.coords = h->d_coords;
  c.marg = h->d_marg;
  c.edge_tc = h->d_edge_tc;
  c.edge_mass = h->d_edge_mass;
  c.mask = partial ? h->d_chk_mask : nullptr;
  const int p0 = prof_mark(h, s);
  CUDA_TRY(h->fp64 ? launch_check64(c, s) : launch_check(c, s));
  prof_span(h, TREE_OT_PROF_CHECK, p0, prof_mark(h, s));
  h->h_marg.resize(h->vec_len);
  h->h_f.resize(h->vec_len);
  h->h_Z.resize(h->nodes.size());
  h->h_rho.resize(h->nodes.size());
  h->h_tc.resize(h->edges.size());
  h->h_mass.resize(h->edges.size());
  CUDA_TRY(cudaMemcpyAsync(h->h_marg.data(), h->d_marg, sizeof(double) * h->vec_len, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(h->h_f.data(), h->d_f, sizeof(double) * h->vec_len, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(h->h_Z.data(), h->d_Z, sizeof(double) * h->nodes.size(), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(h->h_rho.data(), h->d_rho, sizeof(double) * h->nodes.size(), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(h->h_tc.data(), h->d_edge_tc, sizeof(double) * h->edges.size(), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(
      cudaMemcpyAsync(h->h_mass.data(), h->d_edge_mass, sizeof(double) * h->edges.size(), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (partial) {
    for (int p = 0; p < h->nprob; ++p) {
      if ((*only)[p]) continue;
      const int32_t eb = h->prob_edge_base[p], J = h->prob_nodes[p];
      for (int32_t e = eb; e < eb + J - 1; ++e) {
        h->h_tc[e] = keep_tc[e];
        h->h_mass[e] = keep_mass[e];
        for (int k = 0; k < 2; ++k) {
          const DEdgeD& d = h->dedges[2 * e + k];
          const int32_t n = h->nodes[d.owner].n;
          std::copy(keep_marg.begin() + d.off, keep_marg.begin() + d.off + n, h->h_marg.begin() + d.off);
        }
      }
    }
  }
  h->have_check = true;
  return TREE_OT_OK;
}

// potential of a directed edge from the stored normalised form: f = f' - eps Z_owner
inline double true_f(const tree_ot_handle* h, const DEdgeD& d, int32_t x) {
  return h->h_f[d.off + x] - h->probs[d.prob].eps * h->h_Z[d.owner];
}

void fill_result(tree_ot_handle* h, tree_ot_result* res, int p);

// per-problem results from the check's marginals; problems are independent, so
// large batches are split across host threads
void fill_results(tree_ot_handle* h, tree_ot_result* res) {
  const int64_t work = h->vec_len;
  const unsigned hw = std::thread::hardware_concurrency();
  const int nt = (int)std::min<int64_t>({(int64_t)(hw == 0 ? 1 : hw), 16, (int64_t)h->nprob, work / (1 << 18) + 1});
  if (nt <= 1) {
    for (int p = 0; p < h->nprob; ++p) fill_result(h, res, p);
    return;
  }
  std::vector<std::thread> pool;
  for (int t = 0; t < nt; ++t)
    pool.emplace_back([h, res, t, nt] {
      for (int p = t; p < h->nprob; p += nt) fill_result(h, res, p);
    });
  for (auto& th : pool) th.join();
}

void fill_result(tree_ot_handle* h, tree_ot_result* res, int p) {
  {
    tree_ot_result r{};
    const ProbD& P = h->probs[p];
    double rsum = 0.0, rmax = 0.0, tc = 0.0, pr = 0.0, du = 0.0, mass_total = 0.0;
    const int32_t nb = h->prob_node_base[p], J = h->prob_nodes[p];
    for (int32_t jj = 0; jj < J; ++jj) {
      const int32_t j = nb + jj;
      const NodeD& nd = h->nodes[j];
      if (nd.fixed) {
        const DEdgeD& d = h->dedges[h->node_dedges[nd.dedge_begin]];
        double t = 0.0;
        for (int32_t x = 0; x < nd.n; ++x) t += std::fabs(h->h_marg[d.off + x] - h->mu[j][x]);
        rsum += t;
        rmax = std::max(rmax, t);
        for (int32_t x = 0; x < nd.n; ++x)
          if (h->mu[j][x] > 0.0) du += true_f(h, d, x) * h->mu[j][x];
      } else {
        std::vector<double> qbar(nd.n, 0.0);
        for (int32_t i = 0; i < nd.deg; ++i) {
          const DEdgeD& d = h->dedges[h->node_dedges[nd.dedge_begin + i]];
          for (int32_t x = 0; x < nd.n; ++x) qbar[x] += h->h_marg[d.off + x] / nd.deg;
        }
        double fsum = 0.0;
        for (int32_t i = 0; i < nd.deg; ++i) {
          const DEdgeD& d = h->dedges[h->node_dedges[nd.dedge_begin + i]];
          double t = 0.0;
          for (int32_t x = 0; x < nd.n; ++x) {
            t += std::fabs(h->h_marg[d.off + x] - qbar[x]);
            fsum += true_f(h, d, x);
          }
          rsum += t;
          rmax = std::max(rmax, t);
        }
        du += fsum / nd.n;  // eps * rho_j, rho_j = (1/eps) mean_x sum_k f_(j,k)(x)
      }
    }
    const int32_t eb = h->prob_edge_base[p];
    for (int32_t ee = 0; ee < J - 1; ++ee) {
      const int32_t e = eb + ee;
      tc += h->h_tc[e];
      mass_total += h->h_mass[e];
      for (int k = 0; k < 2; ++k) {
        const DEdgeD& d = h->dedges[2 * e + k];
        const int32_t n = h->nodes[d.owner].n;
        for (int32_t x = 0; x < n; ++x) {
          const double q = h->h_marg[d.off + x];
          if (q > 0.0) pr += true_f(h, d, x) * q;
        }
      }
    }
    pr -= P.eps * mass_total;
    du -= P.eps * mass_total;
    r.residual_sum_l1 = rsum;
    r.max_marginal_l1 = rmax;
    r.transport_cost = tc;
    r.primal = pr;
    r.dual = du;
    const bool done = !h->h_done.empty() && h->h_done[p];
    r.half_steps = done ? h->h_done_at[p] : h->hs_host;
    r.status = (h->last_status.empty() ? TREE_OT_OK : h->last_status[p]);
    r.wall_ms = h->last_wall_ms;
    if (!h->h_lowp_span.empty() && h->h_lowp_span[2 * p] >= 0) {
      const int64_t end = h->h_lowp_span[2 * p + 1] >= 0 ? h->h_lowp_span[2 * p + 1] : r.half_steps;
      r.lowp_half_steps = std::max<int64_t>(0, end - h->h_lowp_span[2 * p]);
    }
    r.absorptions = (int64_t)h->h_absorb_count;
    res[p] = r;
  }
}

// ---------------------------------------------------------------------------
// autotuner for the recomputed-cost apply: output block (256/512/1024, which
// sets the warp groups per task) x {2 CTAs per SM register budget, 3 CTAs per
// SM register budget, 1 CTA per SM}.  It
// times both colours' apply launches, which write only the partial sums, so
// the solver state is untouched.  Results are cached per problem-shape
// signature for the life of the process.
// ---------------------------------------------------------------------------
std::mutex g_tune_mu;
struct TuneCfg {
  int32_t ob, gm, variant;
};
std::map<uint64_t, TuneCfg> g_tune_cache;

uint64_t shape_signature(const tree_ot_handle* h) {
  uint64_t sig = 1469598103934665603ull;
  auto mix = [&](uint64_t v) {
    sig ^= v;
    sig *= 1099511628211ull;
  };
  for (const DEdgeD& d : h->dedges) {
    if (h->probs[d.prob].cost_kind == TREE_OT_COST_DENSE_F32) continue;
    mix((uint64_t)h->nodes[d.owner].n);
    mix((uint64_t)h->nodes[d.nbr].n);
    mix((uint64_t)h->probs[d.prob].dim);
    mix((uint64_t)h->nodes[d.owner].colour);
  }
  return sig;
}

int upload_tasks(tree_ot_handle* h, cudaStream_t s) {
  for (int c = 0; c < 2; ++c) {
    if ((int64_t)h->tasks[c].size() > h->task_cap[c]) return fail(TREE_OT_ERR_STATE, "task capacity exceeded");
    if (!h->tasks[c].empty())
      CUDA_TRY(cudaMemcpyAsync(h->d_tasks[c], h->tasks[c].data(), sizeof(Task) * h->tasks[c].size(),
                               cudaMemcpyHostToDevice, s));
  }
  return TREE_OT_OK;
}

int autotune_recompute(tree_ot_handle* h, cudaStream_t s) {
  bool any = false;
  for (int c = 0; c < 2; ++c)
    for (int slot = 1; slot < kApplySlots; ++slot) any = any || h->slot_count[c][slot] > 0;
  if (!any) return TREE_OT_OK;
  const uint64_t sig = shape_signature(h);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(sig);
    if (it != g_tune_cache.end()) {
      build_apply_tasks(h, it->second.ob);
      h->grid_mult = it->second.gm;
      h->rec_variant = it->second.variant;
      return upload_tasks(h, s);
    }
  }
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  float best = 1e30f;
  TuneCfg best_cfg{kRecOut, 0, 0};
  for (int32_t ob : {1024, 512, 256}) {
    build_apply_tasks(h, ob);
    RC_TRY(upload_tasks(h, s));
    for (int32_t cfg = 0; cfg < 3; ++cfg) {
      const int32_t gm = cfg == 2 ? 1 : 0;
      const int32_t variant = cfg == 1 ? 1 : 0;
      h->grid_mult = gm;
      h->rec_variant = variant;
      RC_TRY(launch_apply(h, 0, s));  // warm-up
      RC_TRY(launch_apply(h, 1, s));
      CUDA_TRY(cudaEventRecord(e0, s));
      for (int rep = 0; rep < 2; ++rep) {
        RC_TRY(launch_apply(h, 0, s));
        RC_TRY(launch_apply(h, 1, s));
      }
      CUDA_TRY(cudaEventRecord(e1, s));
      CUDA_TRY(cudaEventSynchronize(e1));
      float ms = 0.f;
      CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) {
        best = ms;
        best_cfg = {ob, gm, variant};
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  build_apply_tasks(h, best_cfg.ob);
  h->grid_mult = best_cfg.gm;
  h->rec_variant = best_cfg.variant;
  RC_TRY(upload_tasks(h, s));
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_cache[sig] = best_cfg;
  return TREE_OT_OK;
}

// Slot-0 (stored-cost) tasks of both colours with their addresses resolved,
// for the bulk-copy staged kernel.  Slot-0 tasks do not depend on the
// recomputed-cost tile shape, so this is built once.
int upload_stream_tasks(tree_ot_handle* h, cudaStream_t s) {
  for (int c = 0; c < 2; ++c) {
    const int32_t cnt = h->slot_count[c][0];
    if (cnt == 0) continue;
    std::vector<StreamTask> st;
    st.reserve(cnt);
    for (int32_t i = 0; i < cnt; ++i) {
      const Task& t = h->tasks[c][h->slot_begin[c][0] + i];
      const DEdgeD& d = h->dedges[t.dedge];
      const EdgeD& e = h->edges[d.edge];
      const ProbD& pd = h->probs[d.prob];
      StreamTask x{};
      x.kind = t.kind;
      x.prob = d.prob;
      x.ocount = t.ocount;
      x.rcount = t.rcount;
      if (t.kind == TASK_ROW && t.pad == 1) {  // rows of the transpose
        x.ld = e.ldt;
        x.C = e.CT + (int64_t)t.o0 * e.ldt + t.r0;
      } else {
        x.ld = e.ld;
        x.C = t.kind == TASK_ROW ? e.C + (int64_t)t.o0 * e.ld + t.r0 : e.C + (int64_t)t.r0 * e.ld + t.o0;
      }
      x.m_off = d.off + t.o0;
      x.h_off = d.rev_off + t.r0;
      x.out_off = d.part_off + (int64_t)t.split * h->nodes[d.owner].n + t.o0;
      x.s2 = pd.s2;
      x.s2_lo = pd.s2_lo;
      st.push_back(x);
    }
    if (!h->d_stasks[c]) RC_TRY(h->alloc(&h->d_stasks[c], cnt));
    CUDA_TRY(cudaMemcpyAsync(h->d_stasks[c], st.data(), sizeof(StreamTask) * cnt, cudaMemcpyHostToDevice, s));
  }
  return TREE_OT_OK;
}

// Stored-cost kernel choice: time the plain-load and the bulk-copy staged
// kernels on both colours' stored-cost tasks (they write only partial sums)
// and keep the faster.
int autotune_dense(tree_ot_handle* h, cudaStream_t s) {
  if (h->slot_count[0][0] + h->slot_count[1][0] == 0 || !apply_tma_available()) return TREE_OT_OK;
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  float ms[2] = {0.f, 0.f};
  for (int32_t tma = 0; tma < 2; ++tma) {
    h->dense_tma = tma;
    for (int rep = 0; rep < 4; ++rep) {
      if (rep == 1) CUDA_TRY(cudaEventRecord(e0, s));
      RC_TRY(launch_apply(h, 0, s, true));
      RC_TRY(launch_apply(h, 1, s, true));
    }
    CUDA_TRY(cudaEventRecord(e1, s));
    CUDA_TRY(cudaEventSynchronize(e1));
    CUDA_TRY(cudaEventElapsedTime(&ms[tma], e0, e1));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int32_t err = 0;
  CUDA_TRY(cudaMemcpyAsync(&err, h->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (err & 2) return fail(TREE_OT_ERR_TIMEOUT, "a bounded wait in the staged edge apply ran out");
  h->dense_tma = ms[1] < ms[0] ? 1 : 0;
  return TREE_OT_OK;
}

// Shared-kernel BF16 phase: group the directed edges of squared-Euclidean
// problems by (owner support, neighbour support, cost scale, eps) — equal
// supports compared by value — and keep the problems all of whose directed
// edges found a group of at least kSkMinCols.  Columns are listed per colour
// of the owner.
constexpr int kSkMinCols = 8;

int plan_shared_kernels(tree_ot_handle* h, const tree_ot_problem* probs, int32_t num_probs) {
  h->sk.clear();
  h->sk_prob.assign(num_probs, 0);
  const size_t NN = h->nodes.size();
  std::vector<std::vector<float>> pts(NN);
  std::vector<uint64_t> hash(NN, 0);
  for (int32_t p = 0; p < num_probs; ++p) {
    const tree_ot_problem& P = probs[p];
    const ProbD& pd = h->probs[p];
    if (P.cost_kind != TREE_OT_COST_SQEUCLID || !P.coords || pd.dim <= 0) continue;
    for (int32_t j = 0; j < P.num_nodes; ++j) {
      const int32_t g = h->prob_node_base[p] + j;
      const size_t cnt = (size_t)h->nodes[g].n * (size_t)pd.dim;
      pts[g].resize(cnt);
      if (P.flags & TREE_OT_INPUT_DEVICE) {
        cudaError_t e = cudaMemcpy(pts[g].data(), P.coords[j], cnt * sizeof(float), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(supports for grouping)");
      } else {
        std::memcpy(pts[g].data(), P.coords[j], cnt * sizeof(float));
      }
      uint64_t hv = 1469598103934665603ull;  // FNV-1a over 32-bit words
      for (size_t i = 0; i < cnt; ++i) {
        uint32_t w;
        std::memcpy(&w, &pts[g][i], 4);
        hv = (hv ^ w) * 1099511628211ull;
      }
      hash[g] = hv;
    }
  }
  using Key = std::tuple<int32_t, int32_t, int32_t, uint64_t, uint64_t, uint64_t, uint64_t>;
  std::map<Key, int> index;
  std::vector<int> dgroup(h->dedges.size(), -1);
  for (size_t di = 0; di < h->dedges.size(); ++di) {
    const DEdgeD& d = h->dedges[di];
    if (pts[d.owner].empty() || pts[d.nbr].empty()) continue;
    const ProbD& pd = h->probs[d.prob];
    uint64_t sb, eb;
    std::memcpy(&sb, &pd.cost_scale, 8);
    std::memcpy(&eb, &pd.eps, 8);
    const Key key{h->nodes[d.owner].n, h->nodes[d.nbr].n, pd.dim, hash[d.owner], hash[d.nbr], sb, eb};
    auto it = index.find(key);
    int gi;
    if (it == index.end()) {
      gi = (int)h->sk.size();
      index.emplace(key, gi);
      h->sk.emplace_back();
      h->sk[gi].owner_rep = d.owner;
      h->sk[gi].nbr_rep = d.nbr;
      h->sk[gi].prob_rep = d.prob;
    } else {
      gi = it->second;
      const auto& G = h->sk[gi];
      if (pts[d.owner] != pts[G.owner_rep] || pts[d.nbr] != pts[G.nbr_rep]) continue;  // equal hashes only
    }
    dgroup[di] = gi;
  }
  // a kernel shared by fewer than kSkMinCols directed edges is cheaper recomputed
  std::vector<int> gsize(h->sk.size(), 0);
  for (int g : dgroup)
    if (g >= 0) ++gsize[g];
  for (int& g : dgroup)
    if (g >= 0 && gsize[g] < kSkMinCols) g = -1;
  std::vector<uint8_t> ok(num_probs, 0);
  for (int32_t p = 0; p < num_probs; ++p)
    ok[p] = probs[p].cost_kind == TREE_OT_COST_SQEUCLID && probs[p].coords && h->probs[p].dim > 0;
  for (size_t di = 0; di < h->dedges.size(); ++di)
    if (dgroup[di] < 0) ok[h->dedges[di].prob] = 0;
  for (size_t di = 0; di < h->dedges.size(); ++di) {
    const DEdgeD& d = h->dedges[di];
    if (!ok[d.prob]) continue;
    h->sk[dgroup[di]].cols[h->nodes[d.owner].colour].push_back(SkCol{d.rev_off, d.part_off, d.prob, (int32_t)di});
  }
  std::vector<tree_ot_handle::SkGroup> kept;
  for (auto& g : h->sk)
    if (!g.cols[0].empty() || !g.cols[1].empty()) kept.push_back(std::move(g));
  h->sk = std::move(kept);
  h->sk_prob = ok;
  return TREE_OT_OK;
}

// device buffers and launch arguments of the shared-kernel groups
int setup_shared_kernels(tree_ot_handle* h, cudaStream_t s) {
  int rc;
  for (auto& g : h->sk) {
    const NodeD& own = h->nodes[g.owner_rep];
    const NodeD& nbn = h->nodes[g.nbr_rep];
    const ProbD& pd = h->probs[g.prob_rep];
    const int32_t mp = (int32_t)align_up(own.n, kSkTileM), kd = (int32_t)align_up(nbn.n, kSkPadK);
    const int64_t maxc = (int64_t)std::max(g.cols[0].size(), g.cols[1].size());
    float *b = nullptr, *rf = nullptr, *cmax = nullptr, *sout = nullptr, *benv = nullptr;
    __nv_bfloat16 *khi = nullptr, *klo = nullptr, *vhi = nullptr, *vlo = nullptr;
    SkCol* dc[2] = {nullptr, nullptr};
    int32_t* fix_count = nullptr;
    int2* fix_list = nullptr;
    if ((rc = h->alloc(&b, kd)) || (rc = h->alloc(&rf, mp)) || (rc = h->alloc(&cmax, maxc)) ||
        (rc = h->alloc(&khi, (int64_t)mp * kd)) ||
        (rc = h->alloc(&klo, (int64_t)mp * kd)) || (rc = h->alloc(&vhi, maxc * kd)) ||
        (rc = h->alloc(&vlo, maxc * kd)) || (rc = h->alloc(&sout, maxc * align_up(own.n, 32))) ||
        (rc = h->alloc(&benv, ((maxc + kSkEnvCols - 1) / kSkEnvCols) * kd)) ||
        (rc = h->alloc(&dc[0], (int64_t)g.cols[0].size())) ||
        (rc = h->alloc(&dc[1], (int64_t)g.cols[1].size())) || (rc = h->alloc(&fix_count, 1)) ||
        (rc = h->alloc(&fix_list, (int64_t)own.n * maxc)))
      return rc;
    CUDA_TRY(cudaMemsetAsync(fix_count, 0, sizeof(int32_t), s));
    for (int c = 0; c < 2; ++c) {
      if (!g.cols[c].empty())
        CUDA_TRY(cudaMemcpyAsync(dc[c], g.cols[c].data(), sizeof(SkCol) * g.cols[c].size(), cudaMemcpyHostToDevice,
                                 s));
      SkArgs& a = g.args[c];
      a.cols = dc[c];
      a.ncols = (int32_t)g.cols[c].size();
      a.nx = own.n;
      a.ny = nbn.n;
      a.dim = pd.dim;
      a.mp = mp;
      a.kd = kd;
      a.hh = h->d_hh;
      a.hl = h->d_hl;
      a.done = h->d_done;
      a.lowp = h->d_lowp;
      a.xc = h->d_coords + own.coord_off;
      a.yc = h->d_coords + nbn.coord_off;
      a.s_hi = pd.s2_scaled;
      a.s_lo = pd.s2_scaled_lo;
      a.b = b;
      a.benv = benv;
      a.cmax = cmax;
      a.rf = rf;
      a.khi = khi;
      a.klo = klo;
      a.vhi = vhi;
      a.vlo = vlo;
      a.part32 = h->d_part32;
      a.sout = sout;
      a.ldo = (int32_t)align_up(own.n, 32);
      a.fix_count = fix_count;
      a.fix_list = fix_list;
      a.err = h->d_err;
      a.use_tc = !(h->opt.flags & TREE_OT_OPT_SK_MMA_SYNC) && sk_tc_available() ? 1 : 0;
      a.tc_pair = a.use_tc && !(h->opt.flags & TREE_OT_OPT_SK_ONE_CTA) && sk_tc_pair_available() ? 1 : 0;
    }
    // the tcgen05 product needs tensor maps of its operands; without them both colours use mma.sync.
    // Its sums leave through a TMA tensor map too where the shapes allow (else plain stores).
    bool tc = g.args[0].use_tc != 0;
    for (int c = 0; c < 2 && tc; ++c) {
      if (g.args[c].ncols <= 0) continue;
      g.args[c].store_tma = (g.args[c].nx >= 32 && g.args[c].ncols >= 16) ? 1 : 0;
      if (sk_encode_maps(g.args[c], &g.maps[c])) continue;
      g.args[c].store_tma = 0;
      if (!sk_encode_maps(g.args[c], &g.maps[c])) tc = false;
    }
    for (int c = 0; c < 2; ++c) g.args[c].use_tc = tc ? 1 : 0;
    CUDA_TRY(launch_sk_reset(b, kd, s));
  }
  if (!h->sk.empty()) {  // per directed edge: where its colour's product leaves the message
    std::vector<SkRefD> ref(h->dedges.size(), SkRefD{nullptr, nullptr, nullptr});
    for (auto& g : h->sk)
      for (int c = 0; c < 2; ++c)
        for (size_t j = 0; j < g.cols[c].size(); ++j)
          ref[g.cols[c][j].dedge] =
              SkRefD{g.args[c].sout + (int64_t)j * g.args[c].ldo, g.args[c].rf, g.args[c].cmax + j};
    if ((rc = h->alloc(&h->d_skref, (int64_t)ref.size()))) return rc;
    CUDA_TRY(cudaMemcpyAsync(h->d_skref, ref.data(), sizeof(SkRefD) * ref.size(), cudaMemcpyHostToDevice, s));
  }
  return TREE_OT_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// exported entry points
// ---------------------------------------------------------------------------

namespace {
// The persistent forest launch: eligible when every problem's costs are
// recomputed from points of one dimension in FP32 with no BF16 phase.  Builds
// the per-problem item counts, then times G = 8 half-steps of the per-half-step
// launches and of the persistent kernel at 2 and 3 CTAs per SM (after 2
// warm-up half-steps each) and keeps the fastest; the state goes back to u = 1.
int setup_forest(tree_ot_handle* h, cudaStream_t s) {
  h->persistent = 0;
  if (h->fp64 || h->lowp || !(h->opt.flags & TREE_OT_OPT_PERSISTENT)) return TREE_OT_OK;
  int D = 0;
  for (int c = 0; c < 2; ++c) {
    if (h->slot_count[c][0] > 0) return TREE_OT_OK;
    for (int slot = 1; slot < kApplySlots; ++slot) {
      if (h->slot_count[c][slot] == 0) continue;
      if (D && D != slot) return TREE_OT_OK;
      D = slot;
    }
  }
  if (D == 0) return TREE_OT_OK;
  std::vector<int32_t> cnt(4 * (size_t)h->nprob, 0);
  for (int c = 0; c < 2; ++c) {
    for (int32_t i = 0; i < h->slot_count[c][D]; ++i)
      ++cnt[4 * h->dedges[h->tasks[c][h->slot_begin[c][D] + i].dedge].prob + c];
    for (const NodeChunk& ch : h->chunks[c]) ++cnt[4 * h->nodes[ch.node].prob + 2 + c];
  }
  if (!h->d_fcnt) {
    int rc = 0;
    if ((rc = h->alloc(&h->d_fcnt, 4 * (int64_t)h->nprob)) || (rc = h->alloc(&h->d_fdone, 2 * (int64_t)h->nprob)) ||
        (rc = h->alloc(&h->d_fctl, 2)))
      return rc;
  }
  CUDA_TRY(cudaMemcpyAsync(h->d_fcnt, cnt.data(), sizeof(int32_t) * cnt.size(), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemsetAsync(h->d_fdone, 0, sizeof(int32_t) * 2 * h->nprob, s));
  CUDA_TRY(cudaMemsetAsync(h->d_fctl, 0, sizeof(int32_t) * 2, s));
  h->forest_D = D;
  h->forest_smem = std::max(h->node_smem[0], h->node_smem[1]);
  h->forest_grid[0] = h->sms * forest_ctas_per_sm(D, false, 2, h->forest_smem);
  h->forest_grid[1] = h->sms * forest_ctas_per_sm(D, false, 3, h->forest_smem);
  h->forest_grid_exact = h->sms * forest_ctas_per_sm(D, true, 2, h->forest_smem);
  if (h->forest_grid[0] < 1 || h->forest_grid_exact < 1) return TREE_OT_OK;
  if (!h->opt.autotune) {  // no timing: the persistent kernel at 2 CTAs per SM
    h->persistent = 2;
    return TREE_OT_OK;
  }
  // time the three forms from u = 1
  constexpr int kWarm = 2, kTimed = 8;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  float best = INFINITY;
  int choice = 0;
  for (int form : {0, 2, 3}) {
    if (form == 3 && h->forest_grid[1] < 1) continue;
    RC_TRY(reset_state(h, s));
    h->persistent = form;
    int rc = queue_half_steps(h, kWarm, false, s);
    if (!rc && cudaEventRecord(e0, s) != cudaSuccess) rc = TREE_OT_ERR_CUDA;
    if (!rc) rc = queue_half_steps(h, kTimed, false, s);
    if (!rc && cudaEventRecord(e1, s) != cudaSuccess) rc = TREE_OT_ERR_CUDA;
    float ms = INFINITY;
    if (!rc && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
      rc = TREE_OT_ERR_CUDA;
    if (rc) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      h->persistent = 0;
      return rc == TREE_OT_ERR_CUDA ? cuda_fail(cudaGetLastError(), "timing the persistent forest launch") : rc;
    }
    if (ms < best) {
      best = ms;
      choice = form;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->persistent = choice;
  return reset_state(h, s);
}

// device tables of the last rounding (see tree_ot_round)
RoundArgs round_args(const tree_ot_handle* h) {
  RoundArgs a{};
  a.tasks = h->d_rtasks;
  a.ntasks = (int32_t)h->rtasks.size();
  a.dedges = h->d_dedges;
  a.ndedges = (int32_t)h->dedges.size();
  a.edges = h->d_edges;
  a.nodes = h->d_nodes;
  a.probs = h->d_probs;
  a.node_dedges = h->d_node_dedges;
  a.side = h->d_rside;
  a.nmass = h->d_rnmass;
  a.ah = h->d_ah;
  a.al = h->d_al;
  a.f = h->d_f;
  a.Z = h->d_Z;
  a.logg = h->d_logg;
  a.mu = h->d_mu;
  a.coords = h->d_coords;
  a.rsum = h->d_rsum;
  a.tgt = h->d_rtgt;
  a.xy = h->d_rxy;
  a.s2 = h->d_rs2;
  a.er = h->d_rer;
  a.edge_acc = h->d_racc;
  return a;
}
}  // namespace

extern "C" {

void tree_ot_default_options(tree_ot_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->precision = TREE_OT_PREC_FP32;
  opt->apply_mode = TREE_OT_APPLY_AUTO;
  opt->tol = 1e-6;
  opt->tol_kind = TREE_OT_TOL_SUM;
  opt->max_half_steps = 100000;
  opt->check_every = 32;
  opt->use_graph = 1;
  opt->flags = 0;
  opt->refine_tol = 1e-5;
  opt->absorb_tau = 48.0;
  opt->lowp_start = 16;
  opt->autotune = 1;
}

const char* tree_ot_error_string(int code) {
  switch (code) {
    case TREE_OT_OK: return "ok";
    case TREE_OT_NOT_CONVERGED: return "not converged (iteration cap reached)";
    case TREE_OT_ERR_ARG: return "invalid argument";
    case TREE_OT_ERR_NOT_TREE: return "edges do not form a tree";
    case TREE_OT_ERR_FIXED_NOT_LEAF: return "fixed node is not a leaf";
    case TREE_OT_ERR_FIXED_ADJACENT: return "edge joins two fixed nodes";
    case TREE_OT_ERR_MARGINAL: return "invalid marginal";
    case TREE_OT_ERR_NONFINITE: return "non-finite input or potential";
    case TREE_OT_ERR_EPS: return "invalid eps";
    case TREE_OT_ERR_CUDA: return "CUDA error";
    case TREE_OT_ERR_OOM: return "out of device memory";
    case TREE_OT_ERR_TIMEOUT: return "device wait timed out";
    case TREE_OT_ERR_STATE: return "invalid state";
    default: return "unknown error";
  }
}

const char* tree_ot_last_error(void) { return g_err.c_str(); }

int tree_ot_validate(const tree_ot_problem* prob) {
  g_err.clear();
  return validate_problem(prob, nullptr);
}

int tree_ot_bipartition(int32_t num_nodes, const int32_t* edges, uint8_t* colour_out) {
  g_err.clear();
  if (!colour_out) return fail(TREE_OT_ERR_ARG, "colour_out is NULL");
  std::vector<std::vector<int32_t>> adj;
  int rc = check_tree(num_nodes, edges, &adj);
  if (rc) return rc;
  colour_tree(num_nodes, adj, colour_out);
  return TREE_OT_OK;
}

int tree_ot_create(const tree_ot_problem* probs, int32_t num_probs, const tree_ot_options* opt, void* cuda_stream,
                   tree_ot_handle** out) {
  g_err.clear();
  if (!out) return fail(TREE_OT_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!probs || num_probs < 1) return fail(TREE_OT_ERR_ARG, "need at least one problem");
  tree_ot_options o;
  tree_ot_default_options(&o);
  if (opt) o = *opt;
  if (o.precision != TREE_OT_PREC_FP32 && o.precision != TREE_OT_PREC_FP64)
    return fail(TREE_OT_ERR_ARG, "unknown precision");
  if (o.apply_mode != TREE_OT_APPLY_AUTO && o.apply_mode != TREE_OT_APPLY_LSE && o.apply_mode != TREE_OT_APPLY_BF16)
    return fail(TREE_OT_ERR_ARG, "unknown apply_mode");
  if (o.apply_mode == TREE_OT_APPLY_BF16 &&
      (!(o.refine_tol >= 0.0) || !(o.absorb_tau > 0.0) || o.absorb_tau > 100.0 || o.lowp_start < 0))
    return fail(TREE_OT_ERR_ARG, "BF16 mode needs refine_tol >= 0, 0 < absorb_tau <= 100 and lowp_start >= 0");
  if (!(o.tol >= 0.0) || o.max_half_steps < 0 || o.check_every < 2 || (o.check_every & 1))
    return fail(TREE_OT_ERR_ARG, "tol >= 0, max_half_steps >= 0 and an even check_every >= 2 are required");
  if (o.tol_kind != TREE_OT_TOL_SUM && o.tol_kind != TREE_OT_TOL_MAX) return fail(TREE_OT_ERR_ARG, "unknown tol_kind");
  std::vector<std::vector<std::vector<int32_t>>> adjs(num_probs);
  for (int32_t p = 0; p < num_probs; ++p) {
    int rc = validate_problem(&probs[p], &adjs[p]);
    if (rc) {
      g_err = "problem " + std::to_string(p) + ": " + g_err;
      return rc;
    }
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  tree_ot_handle* h = new tree_ot_handle();
  h->opt = o;
  h->fp64 = o.precision == TREE_OT_PREC_FP64;
  h->nprob = num_probs;
  int rc = TREE_OT_OK;
  // Stored costs: the column owner's apply reduces down columns, which streams
  // short row pieces at a large stride.  When the device has the room, each edge
  // also keeps its cost transposed so both directions stream contiguous rows.
  if (!h->fp64 && !(o.flags & TREE_OT_OPT_NO_TRANSPOSE)) {
    int64_t ct_bytes = 0;
    for (int32_t p = 0; p < num_probs; ++p) {
      if (probs[p].cost_kind != TREE_OT_COST_DENSE_F32) continue;
      for (int32_t e = 0; e < probs[p].num_nodes - 1; ++e) {
        const int64_t na = probs[p].support_size[probs[p].edges[2 * e]];
        const int64_t nb = probs[p].support_size[probs[p].edges[2 * e + 1]];
        ct_bytes += 4 * nb * align_up(na, 4) * 2;  // the transpose, and room for a padded copy of C
      }
    }
    size_t free_b = 0, total_b = 0;
    if (ct_bytes > 0 && cudaMemGetInfo(&free_b, &total_b) == cudaSuccess &&
        (int64_t)free_b > ct_bytes + (int64_t(1) << 30))
      h->use_ct = true;
    cudaGetLastError();
  }
  auto bail = [&](int code) {
    tree_ot_destroy(h);
    return code;
  };

  // ---- host plan ---------------------------------------------------------
  int64_t vec_off = 0, node_off = 0, coord_off = 0, part_off = 0;
  int32_t chunk_base = 0;
  std::vector<std::vector<int32_t>> owned_by;  // per global node: owned dedges
  for (int32_t p = 0; p < num_probs; ++p) {
    const tree_ot_problem& P = probs[p];
    const int32_t J = P.num_nodes;
    const int32_t nbase = (int32_t)h->nodes.size();
    const int32_t ebase = (int32_t)h->edges.size();
    h->prob_node_base.push_back(nbase);
    h->prob_edge_base.push_back(ebase);
    h->prob_nodes.push_back(J);
    std::vector<uint8_t> col(J);
    colour_tree(J, adjs[p], col.data());
    ProbD pd{};
    pd.eps = P.eps;
    pd.inv_eps = 1.0 / P.eps;
    pd.cost_scale = P.cost_kind == TREE_OT_COST_SQEUCLID ? P.cost_scale : 1.0;
    split_positive(kLog2e / P.eps, &pd.s2, &pd.s2_lo);
    split_positive(pd.cost_scale * kLog2e / P.eps, &pd.s2_scaled, &pd.s2_scaled_lo);
    pd.dim = P.cost_kind == TREE_OT_COST_SQEUCLID ? P.dim : (P.coords ? P.dim : 0);
    pd.cost_kind = P.cost_kind;
    const bool have_coords = P.coords != nullptr && pd.dim > 0;
    for (int32_t j = 0; j < J; ++j) {
      NodeD nd{};
      nd.n = P.support_size[j];
      nd.deg = (int32_t)adjs[p][j].size();
      nd.prob = p;
      nd.fixed = P.is_fixed[j] ? 1 : 0;
      nd.colour = col[j];
      nd.node_off = node_off;
      node_off += align_up(nd.n, 32);
      nd.coord_off = have_coords ? coord_off : -1;
      if (have_coords) coord_off += align_up((int64_t)nd.n * pd.dim, 4);
      pd.nodes_in_colour[nd.colour] += 1;
      h->nodes.push_back(nd);
      owned_by.emplace_back();
      std::vector<double> mu;
      if (nd.fixed) mu.assign(P.marginal[j], P.marginal[j] + nd.n);
      h->mu.push_back(std::move(mu));
    }
    pd.edge_begin = ebase;
    pd.edge_count = J - 1;
    h->probs.push_back(pd);
    for (int32_t e = 0; e < J - 1; ++e) {
      EdgeD ed{};
      ed.a = nbase + P.edges[2 * e];
      ed.b = nbase + P.edges[2 * e + 1];
      ed.na = h->nodes[ed.a].n;
      ed.nb = h->nodes[ed.b].n;
      ed.ld = align_up(ed.nb, 4);
      ed.C = nullptr;
      h->edges.push_back(ed);
      h->elems += (int64_t)ed.na * ed.nb;
      const int32_t ge = ebase + e;
      for (int k = 0; k < 2; ++k) {
        DEdgeD d{};
        d.owner = k == 0 ? ed.a : ed.b;
        d.nbr = k == 0 ? ed.b : ed.a;
        d.edge = ge;
        d.dir = k;
        d.prob = p;
        const int32_t n_own = h->nodes[d.owner].n, n_nbr = h->nodes[d.nbr].n;
        if (h->fp64)
          d.nsplit = 1;
        else if (P.cost_kind == TREE_OT_COST_DENSE_F32)
          d.nsplit = (k == 0 || h->use_ct) ? (n_nbr + kRowCols - 1) / kRowCols : (n_nbr + kColRows - 1) / kColRows;
        else
          d.nsplit = (n_nbr + kRecRed - 1) / kRecRed;
        d.off = vec_off;
        vec_off += align_up(n_own, 32);
        d.part_off = part_off;
        part_off += (int64_t)d.nsplit * n_own;
        h->dedges.push_back(d);
        owned_by[d.owner].push_back(2 * ge + k);
      }
      h->dedges[2 * ge].rev_off = h->dedges[2 * ge + 1].off;
      h->dedges[2 * ge + 1].rev_off = h->dedges[2 * ge].off;
      if (P.cost_kind == TREE_OT_COST_DENSE_F32) h->matrix_bytes += 4 * (int64_t)ed.na * ed.nb;
    }
  }
  for (size_t j = 0; j < h->nodes.size(); ++j) {
    h->nodes[j].dedge_begin = (int32_t)h->node_dedges.size();
    for (int32_t d : owned_by[j]) h->node_dedges.push_back(d);
  }
  h->vec_len = vec_off;
  h->node_len = node_off;
  h->coord_len = coord_off;
  h->part_len = part_off;
  // node-update chunks: kNodePairs (edge, point) pairs per CTA where a colour has
  // many of them (fewer CTAs, each CTA's metadata loads amortised over more
  // pairs), kNodePairsSmall where its pairs fill few waves of CTAs anyway
  {
    int64_t pairs[2] = {0, 0};
    for (const NodeD& nd : h->nodes) pairs[nd.colour] += (int64_t)nd.n * std::max(nd.deg, 1);
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    for (int c = 0; c < 2; ++c)
      h->chunk_pairs[c] = pairs[c] > (int64_t)kNodePairsSmall * 8 * nsm ? kNodePairs : kNodePairsSmall;
    for (NodeD& nd : h->nodes) {
      const int32_t cp = node_chunk_points(nd.n, nd.deg, h->chunk_pairs[nd.colour]);
      nd.nchunks = (nd.n + cp - 1) / cp;
      nd.chunk_base = chunk_base;
      chunk_base += nd.nchunks;
    }
  }
  h->nzchunks = chunk_base;

  // device task arrays are sized for the finest output blocking the autotuner may pick
  build_apply_tasks(h, 256);
  h->task_cap[0] = (int64_t)h->tasks[0].size();
  h->task_cap[1] = (int64_t)h->tasks[1].size();
  build_apply_tasks(h, kRecOut);
  // absorbed BF16 phase: apply tasks per colour and absorption blocks (stored-cost edges only)
  h->lowp = o.apply_mode == TREE_OT_APPLY_BF16 && !h->fp64;
  if (h->lowp) {
    bool any = false;
    for (size_t di = 0; di < h->dedges.size(); ++di) {
      const DEdgeD& d = h->dedges[di];
      if (h->probs[d.prob].cost_kind != TREE_OT_COST_DENSE_F32) continue;
      any = true;
      const NodeD& own = h->nodes[d.owner];
      const NodeD& nbn = h->nodes[d.nbr];
      std::vector<Task>& tl = h->btasks[own.colour];
      if (d.dir == 0) {
        // taller than the FP32 row tasks: a BF16 row is half the bytes, and every task
        // first forms its columns' weights
        for (int32_t o0 = 0; o0 < own.n; o0 += kBfRowTask)
          for (int32_t s = 0; s < d.nsplit; ++s)
            tl.push_back(Task{(int32_t)di, TASK_ROW, o0, std::min(kBfRowTask, own.n - o0), s * kRowCols,
                              std::min(kRowCols, nbn.n - s * kRowCols), s, 0});
        for (int32_t o0 = 0; o0 < own.n; o0 += 64)
          h->atasks.push_back(Task{(int32_t)di, TASK_ROW, o0, std::min(64, own.n - o0), 0, nbn.n, 0, 0});
      } else {
        // column sums of K~ (measured faster than rows of a transposed BF16 copy:
        // 0.46 against 0.54 ms per launch on the 64-node tree)
        const int32_t rows = h->use_ct ? kRowCols : kColRows;  // reduction rows per split (see nsplit)
        for (int32_t s = 0; s < d.nsplit; ++s)
          for (int32_t o0 = 0; o0 < own.n; o0 += kBfCols)
            tl.push_back(Task{(int32_t)di, TASK_COL, o0, std::min(kBfCols, own.n - o0), s * rows,
                              std::min(rows, nbn.n - s * rows), s, 0});
      }
    }
    h->lowp = any;
  }
  if (o.apply_mode == TREE_OT_APPLY_BF16 && !h->fp64) {
    if ((rc = plan_shared_kernels(h, probs, num_probs))) return bail(rc);
    if (!h->sk.empty()) h->lowp = true;
  }
  h->node_smem[0] = h->node_smem[1] = 0;
  for (int pass = 0; pass < 2; ++pass)  // per colour: the fixed nodes' chunks, then the free nodes'
    for (size_t j = 0; j < h->nodes.size(); ++j) {
      const NodeD& nd = h->nodes[j];
      if ((pass == 0) != (nd.fixed != 0)) continue;
      const int32_t cp = node_chunk_points(nd.n, nd.deg, h->chunk_pairs[nd.colour]);
      for (int32_t c = 0; c < nd.nchunks; ++c)
        h->chunks[nd.colour].push_back(NodeChunk{(int32_t)j, c, c * cp, std::min(cp, nd.n - c * cp)});
      if (pass == 0) h->nfixed_chunks[nd.colour] += nd.nchunks;
      const uint32_t b = node_smem_layout(nd.deg, std::min(cp, nd.n), h->fp64).bytes;
      h->node_smem[nd.colour] = std::max(h->node_smem[nd.colour], b);
    }
  if (std::max(h->node_smem[0], h->node_smem[1]) > kNodeSmemMax)
    return bail(fail(TREE_OT_ERR_ARG, "a node's degree is too high for the node update"));

  for (size_t e = 0; e < h->edges.size(); ++e) {
    const EdgeD& ed = h->edges[e];
    for (int32_t o0 = 0; o0 < ed.na; o0 += 64)
      h->check_tasks.push_back(Task{(int32_t)(2 * e), TASK_ROW, o0, std::min(64, ed.na - o0), 0, ed.nb, 0, 0});
    for (int32_t o0 = 0; o0 < ed.nb; o0 += 256)
      h->check_tasks.push_back(Task{(int32_t)(2 * e + 1), TASK_COL, o0, std::min(256, ed.nb - o0), 0, ed.na, 0, 0});
  }

  // ---- device memory -----------------------------------------------------
  const int64_t NN = (int64_t)h->nodes.size(), NE = (int64_t)h->edges.size(), ND = (int64_t)h->dedges.size();
  if ((rc = h->alloc(&h->d_probs, num_probs)) || (rc = h->alloc(&h->d_nodes, NN)) ||
      (rc = h->alloc(&h->d_edges, NE)) || (rc = h->alloc(&h->d_dedges, ND)) ||
      (rc = h->alloc(&h->d_node_dedges, (int64_t)h->node_dedges.size())) ||
      (rc = h->alloc(&h->d_tasks[0], h->task_cap[0])) || (rc = h->alloc(&h->d_tasks[1], h->task_cap[1])) ||
      (rc = h->alloc(&h->d_queue, 2 * 2 * kApplySlots)) ||
      (rc = h->alloc(&h->d_chunks[0], (int64_t)h->chunks[0].size())) ||
      (rc = h->alloc(&h->d_chunks[1], (int64_t)h->chunks[1].size())) ||
      (rc = h->alloc(&h->d_check_tasks, (int64_t)h->check_tasks.size())) || (rc = h->alloc(&h->d_f, h->vec_len)) ||
      (rc = h->alloc(&h->d_fr, h->vec_len)) || (rc = h->alloc(&h->d_hh, h->vec_len)) ||
      (rc = h->alloc(&h->d_hl, h->vec_len)) || (rc = h->alloc(&h->d_ah, h->vec_len)) ||
      (rc = h->alloc(&h->d_al, h->vec_len)) || (rc = h->alloc(&h->d_marg, h->vec_len)) ||
      (rc = h->alloc(&h->d_Z, NN)) || (rc = h->alloc(&h->d_rho, NN)) || (rc = h->alloc(&h->d_logg, h->node_len)) ||
      (rc = h->alloc(&h->d_mu, h->node_len)) || (rc = h->alloc(&h->d_lgf, h->node_len)) ||
      (rc = h->alloc(&h->d_coords, h->coord_len)) ||
      (rc = h->alloc(&h->d_coords_hi, h->coord_len)) || (rc = h->alloc(&h->d_coords_lo, h->coord_len)) ||
      (rc = h->alloc(&h->d_cmax, num_probs)) || (rc = h->alloc(&h->d_exact, num_probs)) ||
      (rc = h->alloc(&h->d_zpart, h->nzchunks)) || (rc = h->alloc(&h->d_resid_acc, ND)) ||
      (rc = h->alloc(&h->d_resid_dedge, ND)) || (rc = h->alloc(&h->d_res_sum, (int64_t)kResidRing * num_probs)) ||
      (rc = h->alloc(&h->d_res_max, (int64_t)kResidRing * num_probs)) || (rc = h->alloc(&h->d_done, num_probs)) ||
      (rc = h->alloc(&h->d_live, 1)) ||
      (rc = h->alloc(&h->d_done_at, num_probs)) || (rc = h->alloc(&h->d_node_arrive, NN)) ||
      (rc = h->alloc(&h->d_node_count, num_probs)) || (rc = h->alloc(&h->d_launch_count, 1)) ||
      (rc = h->alloc(&h->d_hs, 1)) || (rc = h->alloc(&h->d_ptol, num_probs)) ||
      (rc = h->alloc(&h->d_deadline, num_probs)) ||
      (rc = h->alloc(&h->d_chk_mask, num_probs)) || (rc = h->alloc(&h->d_err, 1)) || (rc = h->alloc(&h->d_scan, 1)) ||
      (rc = h->alloc(&h->d_edge_tc, NE)) || (rc = h->alloc(&h->d_edge_mass, NE)))
    return bail(rc);
  if (h->fp64) {
    if ((rc = h->alloc(&h->d_part64, h->part_len))) return bail(rc);
  } else {
    if ((rc = h->alloc(&h->d_part32, h->part_len))) return bail(rc);
  }
  if ((rc = h->alloc(&h->d_lowp, num_probs)) || (rc = h->alloc(&h->d_drift, NE)) ||
      (rc = h->alloc(&h->d_lowp_span, 2 * (int64_t)num_probs)) || (rc = h->alloc(&h->d_absorb_count, 1)) ||
      (rc = h->alloc(&h->d_lowp_best, num_probs)) || (rc = h->alloc(&h->d_lowp_best_t, num_probs)))
    return bail(rc);
  if (h->lowp) {
    if ((rc = h->alloc(&h->d_bh, h->vec_len)) || (rc = h->alloc(&h->d_bl, h->vec_len)) ||
        (rc = h->alloc(&h->d_arho, h->vec_len)) ||
        (rc = h->alloc(&h->d_btasks[0], (int64_t)h->btasks[0].size())) ||
        (rc = h->alloc(&h->d_btasks[1], (int64_t)h->btasks[1].size())) ||
        (rc = h->alloc(&h->d_atasks, (int64_t)h->atasks.size())))
      return bail(rc);
    for (EdgeD& ed : h->edges) {
      if (h->probs[h->nodes[ed.a].prob].cost_kind != TREE_OT_COST_DENSE_F32) continue;
      ed.ldk = align_up(ed.nb, 8);
      if ((rc = h->alloc(&ed.K, (int64_t)ed.na * ed.ldk))) return bail(rc);
    }
  }
  if ((rc = setup_shared_kernels(h, s))) return bail(rc);
  if (!h->fp64) {  // host-resolved records of the fixed leaves' chunks, per colour
    std::vector<SkRefD> skref(h->dedges.size(), SkRefD{nullptr, nullptr, nullptr});
    if (h->d_skref) {
      cudaError_t ce = cudaMemcpyAsync(skref.data(), h->d_skref, sizeof(SkRefD) * skref.size(), cudaMemcpyDeviceToHost, s);
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
      if (ce != cudaSuccess) return bail(cuda_fail(ce, "read shared-kernel references"));
    }
    for (int c = 0; c < 2; ++c) {
      std::vector<FixedChunkD> fr;
      for (int32_t k = 0; k < h->nfixed_chunks[c]; ++k) {
        const NodeChunk& ch = h->chunks[c][k];
        const NodeD& nd = h->nodes[ch.node];
        const int32_t di = h->node_dedges[nd.dedge_begin];
        const DEdgeD& d = h->dedges[di];
        const ProbD& pd = h->probs[nd.prob];
        fr.push_back(FixedChunkD{d.off, d.part_off, nd.node_off, ch.node, ch.x0, ch.cnt, nd.n, nd.prob, di, d.nbr,
                                 d.edge, d.nsplit, pd.cost_kind, pd.eps * 0.69314718055994530942, skref[di]});
      }
      if (fr.empty()) continue;
      if ((rc = h->alloc(&h->d_fixed[c], (int64_t)fr.size()))) return bail(rc);
      const cudaError_t ce =
          cudaMemcpyAsync(h->d_fixed[c], fr.data(), sizeof(FixedChunkD) * fr.size(), cudaMemcpyHostToDevice, s);
      if (ce != cudaSuccess) return bail(cuda_fail(ce, "upload fixed-leaf chunk records"));
    }
  }

  auto up = [&](void* dst, const void* src, size_t bytes) -> int {
    if (bytes == 0) return TREE_OT_OK;
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
    return e == cudaSuccess ? TREE_OT_OK : cuda_fail(e, "cudaMemcpyAsync(upload)");
  };

  // node vectors: log gamma and mu (FP64)
  {
    std::vector<double> lg(h->node_len, 0.0), mu(h->node_len, 0.0);
    std::vector<float4> lgf(h->node_len, float4{0.f, 0.f, 0.f, 0.f});
    for (size_t j = 0; j < h->nodes.size(); ++j) {
      const NodeD& nd = h->nodes[j];
      if (!nd.fixed) continue;
      for (int32_t x = 0; x < nd.n; ++x) {
        const double v = h->mu[j][x];
        mu[nd.node_off + x] = v;
        lg[nd.node_off + x] = v > 0.0 ? std::log(v) : -INFINITY;
        // log2 mu as (hi on the 2^-10 grid, lo), as the device splits values
        float4& g = lgf[nd.node_off + x];
        if (v > 0.0) {
          const double l2 = std::log(v) * kLog2e;
          const float hi = std::rint((float)l2 * 1024.f) * (1.f / 1024.f);
          g = float4{hi, (float)(l2 - (double)hi), (float)v, 0.f};
        } else {
          g = float4{-INFINITY, 0.f, 0.f, 0.f};
        }
      }
    }
    if ((rc = up(h->d_logg, lg.data(), sizeof(double) * lg.size())) ||
        (rc = up(h->d_mu, mu.data(), sizeof(double) * mu.size())) ||
        (rc = up(h->d_lgf, lgf.data(), sizeof(float4) * lgf.size())))
      return bail(rc);
    CUDA_TRY(cudaStreamSynchronize(s));
  }
  // coordinates
  for (int32_t p = 0; p < num_probs; ++p) {
    const tree_ot_problem& P = probs[p];
    const ProbD& pd = h->probs[p];
    if (!P.coords || pd.dim == 0) continue;
    const cudaMemcpyKind kind =
        (P.flags & TREE_OT_INPUT_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    for (int32_t j = 0; j < P.num_nodes; ++j) {
      const NodeD& nd = h->nodes[h->prob_node_base[p] + j];
      cudaError_t e = cudaMemcpyAsync(h->d_coords + nd.coord_off, P.coords[j], sizeof(float) * nd.n * pd.dim, kind, s);
      if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMemcpyAsync(coords)"));
    }
  }
  // dense costs: borrow aligned device matrices, otherwise copy into a padded buffer
  CUDA_TRY(cudaMemsetAsync(h->d_scan, 0, sizeof(int32_t), s));
  for (int32_t p = 0; p < num_probs; ++p) {
    const tree_ot_problem& P = probs[p];
    if (P.cost_kind != TREE_OT_COST_DENSE_F32) continue;
    for (int32_t e = 0; e < P.num_nodes - 1; ++e) {
      EdgeD& ed = h->edges[h->prob_edge_base[p] + e];
      const float* src = P.dense_cost[e];
      const bool dev = (P.flags & TREE_OT_INPUT_DEVICE) != 0;
      if (dev && ed.nb % 4 == 0 && ((uintptr_t)src % 16) == 0) {
        ed.C = src;
        ed.ld = ed.nb;
      } else {
        float* dst = nullptr;
        if ((rc = h->alloc(&dst, (int64_t)ed.na * ed.ld))) return bail(rc);
        if (dev) {
          cudaError_t ce = launch_pad_copy(src, ed.nb, dst, ed.ld, ed.na, ed.nb, s);
          if (ce != cudaSuccess) return bail(cuda_fail(ce, "pad copy"));
        } else {
          if (ed.ld != ed.nb) {
            cudaError_t ce = launch_fill_f32(dst, (int64_t)ed.na * ed.ld, INFINITY, s);
            if (ce != cudaSuccess) return bail(cuda_fail(ce, "fill"));
          }
          cudaError_t ce = cudaMemcpy2DAsync(dst, sizeof(float) * ed.ld, src, sizeof(float) * ed.nb,
                                             sizeof(float) * ed.nb, ed.na, cudaMemcpyHostToDevice, s);
          if (ce != cudaSuccess) return bail(cuda_fail(ce, "cudaMemcpy2DAsync(cost)"));
        }
        ed.C = dst;
      }
      cudaError_t ce = launch_scan_cost(ed.C, ed.ld, ed.na, ed.nb, h->d_scan, s);
      if (ce != cudaSuccess) return bail(cuda_fail(ce, "cost scan"));
      if (h->use_ct) {
        float* ct = nullptr;
        ed.ldt = align_up(ed.na, 4);
        if ((rc = h->alloc(&ct, (int64_t)ed.nb * ed.ldt))) return bail(rc);
        ce = launch_transpose_pad(ed.C, ed.ld, ed.na, ed.nb, ct, ed.ldt, s);
        if (ce != cudaSuccess) return bail(cuda_fail(ce, "cost transpose"));
        ed.CT = ct;
      }
    }
  }
  // plan tables
  if ((rc = up(h->d_probs, h->probs.data(), sizeof(ProbD) * h->probs.size())) ||
      (rc = up(h->d_nodes, h->nodes.data(), sizeof(NodeD) * h->nodes.size())) ||
      (rc = up(h->d_edges, h->edges.data(), sizeof(EdgeD) * h->edges.size())) ||
      (rc = up(h->d_dedges, h->dedges.data(), sizeof(DEdgeD) * h->dedges.size())) ||
      (rc = up(h->d_node_dedges, h->node_dedges.data(), sizeof(int32_t) * h->node_dedges.size())) ||
      (rc = up(h->d_tasks[0], h->tasks[0].data(), sizeof(Task) * h->tasks[0].size())) ||
      (rc = up(h->d_tasks[1], h->tasks[1].data(), sizeof(Task) * h->tasks[1].size())) ||
      (rc = up(h->d_chunks[0], h->chunks[0].data(), sizeof(NodeChunk) * h->chunks[0].size())) ||
      (rc = up(h->d_chunks[1], h->chunks[1].data(), sizeof(NodeChunk) * h->chunks[1].size())) ||
      (rc = up(h->d_check_tasks, h->check_tasks.data(), sizeof(Task) * h->check_tasks.size())))
    return bail(rc);
  if (h->coord_len > 0) {  // needs the node and problem tables on the device
    cudaError_t e = launch_split_coords(h->d_coords, h->d_nodes, (int32_t)h->nodes.size(), h->d_probs, h->d_cmax,
                                        num_probs, h->d_coords_hi, h->d_coords_lo, s);
    if (e != cudaSuccess) return bail(cuda_fail(e, "coordinate split"));
  }
  if (h->lowp && ((rc = up(h->d_btasks[0], h->btasks[0].data(), sizeof(Task) * h->btasks[0].size())) ||
                  (rc = up(h->d_btasks[1], h->btasks[1].data(), sizeof(Task) * h->btasks[1].size())) ||
                  (rc = up(h->d_atasks, h->atasks.data(), sizeof(Task) * h->atasks.size()))))
    return bail(rc);
  int32_t bad = 0;
  {
    cudaError_t ce = cudaMemcpyAsync(&bad, h->d_scan, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (ce != cudaSuccess) return bail(cuda_fail(ce, "scan read-back"));
    ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return bail(cuda_fail(ce, "cudaStreamSynchronize(create)"));
  }
  if (bad) return bail(fail(TREE_OT_ERR_NONFINITE, "a dense cost holds NaN or -inf"));

  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  h->sms = sms;
  for (int slot = 0; slot < kApplySlots; ++slot) {
    h->apply_grid[slot] = sms * apply_ctas_per_sm(slot, 0);
    for (int v = 0; v < 2; ++v) h->rec_grid[v][slot] = sms * apply_ctas_per_sm(slot, v);
  }
  h->bf16_grid = sms * apply_bf16_ctas_per_sm();
  for (int c = 0; c < 2; ++c) {  // deferred node bookkeeping: where, and what it reads
    if (o.flags & TREE_OT_OPT_NODE_DEFER)
      h->node_defer[c] = true;
    else if (o.flags & TREE_OT_OPT_NODE_ARRIVE)
      h->node_defer[c] = false;
    else
      h->node_defer[c] = (int64_t)h->chunks[c].size() > 4 * (int64_t)sms;
    // per problem: the colour's owned directed edges, then its free nodes
    const int32_t np = h->nprob;
    std::vector<std::vector<int32_t>> dl(np), nl(np);
    for (size_t j = 0; j < h->nodes.size(); ++j) {
      const NodeD& nd = h->nodes[j];
      if (nd.colour != c) continue;
      for (int32_t i = 0; i < nd.deg; ++i) dl[nd.prob].push_back(h->node_dedges[nd.dedge_begin + i]);
      if (!nd.fixed) nl[nd.prob].push_back((int32_t)j);
    }
    // one array: dbeg [np + 1], dedges, nbeg [np + 1], nodes
    std::vector<int32_t> buf(np + 1, 0);
    for (int32_t p = 0; p < np; ++p) {
      buf[p + 1] = buf[p] + (int32_t)dl[p].size();
      buf.insert(buf.end(), dl[p].begin(), dl[p].end());
    }
    const size_t nb = buf.size();
    buf.resize(nb + np + 1, 0);
    for (int32_t p = 0; p < np; ++p) {
      buf[nb + p + 1] = buf[nb + p] + (int32_t)nl[p].size();
      buf.insert(buf.end(), nl[p].begin(), nl[p].end());
    }
    if ((rc = h->alloc(&h->d_fin[c], (int64_t)buf.size())) ||
        (rc = up(h->d_fin[c], buf.data(), sizeof(int32_t) * buf.size())))
      return bail(rc);
    h->fin[c] = FinishList{h->d_fin[c], h->d_fin[c] + (np + 1), h->d_fin[c] + nb, h->d_fin[c] + nb + (np + 1)};
  }
  {
    cudaError_t ce = cudaStreamCreateWithFlags(&h->hstream, cudaStreamNonBlocking);
    if (ce != cudaSuccess) return bail(cuda_fail(ce, "cudaStreamCreate"));
  }
  {
    // the staged kernel rounds operand copies up to 16 bytes: the arena pads stay zero
    cudaError_t ce = cudaMemsetAsync(h->d_hh, 0, sizeof(float) * h->vec_len, s);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(h->d_hl, 0, sizeof(float) * h->vec_len, s);
    if (ce != cudaSuccess) return bail(cuda_fail(ce, "operand memset"));
  }
  if ((rc = reset_state(h, s))) return bail(rc);
  // the autotuners time the FP32 kernels: no problem in a BF16 phase meanwhile
  CUDA_TRY(cudaMemsetAsync(h->d_lowp, 0, sizeof(int32_t) * h->nprob, s));
  if ((rc = recount_live(h, s))) return bail(rc);
  if (o.autotune && !h->fp64 && (rc = autotune_recompute(h, s))) return bail(rc);
  if (!h->fp64) {
    if ((rc = upload_stream_tasks(h, s))) return bail(rc);
    if (o.flags & (TREE_OT_OPT_DENSE_TMA | TREE_OT_OPT_TEST_STALL)) {
      if (!apply_tma_available()) return bail(fail(TREE_OT_ERR_CUDA, "staged edge apply unavailable"));
      h->dense_tma = 1;
    } else if (!(o.flags & TREE_OT_OPT_DENSE_LDG) && o.autotune && (rc = autotune_dense(h, s))) {
      return bail(rc);
    }
  }
  if (h->lowp && (rc = reset_state(h, s))) return bail(rc);  // the BF16 phases back
  if ((rc = setup_forest(h, s))) return bail(rc);
  {
    cudaError_t ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return bail(cuda_fail(ce, "cudaStreamSynchronize(create)"));
  }
  *out = h;
  return TREE_OT_OK;
}

int tree_ot_destroy(tree_ot_handle* h) {
  if (!h) return TREE_OT_OK;
  if (h->d_setbuf) cudaFree(h->d_setbuf);
  if (h->graph) cudaGraphExecDestroy(h->graph);
  if (h->hstream) cudaStreamDestroy(h->hstream);
  for (cudaEvent_t e : h->prof_ev) cudaEventDestroy(e);
  for (void* p : h->owned) cudaFree(p);
  delete h;
  return TREE_OT_OK;
}

int tree_ot_reset(tree_ot_handle* h, void* cuda_stream) {
  g_err.clear();
  if (!h) return fail(TREE_OT_ERR_ARG, "handle is NULL");
  ++h->pot_version;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  RC_TRY(reset_state(h, s));
  h->h_done.clear();
  h->h_done_at.clear();
  h->last_status.clear();
  return TREE_OT_OK;
}

int tree_ot_half_steps(tree_ot_handle* h, void* cuda_stream, int64_t T) {
  g_err.clear();
  if (!h || T < 0) return fail(TREE_OT_ERR_ARG, "handle is NULL or T < 0");
  ++h->pot_version;
  return queue_half_steps(h, T, false, (cudaStream_t)cuda_stream);
}

int tree_ot_apply(tree_ot_handle* h, void* cuda_stream, int32_t colour) {
  g_err.clear();
  if (!h || (colour != 0 && colour != 1)) return fail(TREE_OT_ERR_ARG, "handle is NULL or colour not 0/1");
  return launch_apply(h, colour, (cudaStream_t)cuda_stream);
}

int tree_ot_node_update(tree_ot_handle* h, void* cuda_stream, int32_t colour) {
  g_err.clear();
  if (!h || (colour != 0 && colour != 1)) return fail(TREE_OT_ERR_ARG, "handle is NULL or colour not 0/1");
  if ((h->hs_host % 2) != colour) return fail(TREE_OT_ERR_STATE, "node_update colour does not follow the schedule");
  ++h->pot_version;
  RC_TRY(launch_update(h, colour, false, (cudaStream_t)cuda_stream));
  ++h->hs_host;
  return TREE_OT_OK;
}

int tree_ot_solve(tree_ot_handle* h, void* cuda_stream, tree_ot_result* results) {
  g_err.clear();
  if (!h) return fail(TREE_OT_ERR_ARG, "handle is NULL");
  ++h->pot_version;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const auto t0 = std::chrono::steady_clock::now();
  const int G = h->opt.check_every;
  h->h_done.assign(h->nprob, 0);
  h->h_done_at.assign(h->nprob, 0);
  int32_t err = 0;
  if (h->hs_host % 2) RC_TRY(queue_half_steps(h, 1, true, s));
  bool use_graph = h->opt.use_graph != 0;
  if (use_graph) RC_TRY(build_graph(h, G));
  // Certification: a problem retires on the FP32 stopping quantity of the
  // half-step kernels; the FP64-grade check of its returned iterate decides.
  // If the check exceeds tol, the problem resumes with a threshold below the
  // FP32 quantity it retired on, scaled by how far the check missed, up to
  // kCertifyRounds times and only while each round still lowers the check
  // (else the FP32 iterate has reached its accuracy floor; a recomputed-cost
  // problem then gets one more chance with exact squared distances).
  constexpr int kCertifyRounds = 8;
  std::vector<double> prev_got(h->nprob, INFINITY);
  std::vector<int32_t> resumed(h->nprob, 0);  // problems resumed by the last round
  for (int cert = 0;; ++cert) {
    while (h->hs_host < h->opt.max_half_steps) {
      const int64_t left = h->opt.max_half_steps - h->hs_host;
      if (use_graph && left >= G) {
        CUDA_TRY(cudaGraphLaunch(h->graph, s));
        h->hs_host += G;
        h->f_stale = !h->fp64;
      } else {
        RC_TRY(queue_half_steps(h, std::min<int64_t>(G, left), true, s));
      }
      CUDA_TRY(cudaMemcpyAsync(h->h_done.data(), h->d_done, sizeof(int32_t) * h->nprob, cudaMemcpyDeviceToHost, s));
      CUDA_TRY(cudaMemcpyAsync(&err, h->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      CUDA_TRY(cudaStreamSynchronize(s));
      if (err & 2) return fail(TREE_OT_ERR_TIMEOUT, "a bounded wait in the staged edge apply ran out");
      if (err) return fail(TREE_OT_ERR_NONFINITE, "a potential became non-finite (an infeasible or degenerate input)");
      bool all = true;
      for (int p = 0; p < h->nprob; ++p) all = all && h->h_done[p];
      if (all) break;
    }
    CUDA_TRY(cudaMemcpyAsync(h->h_done.data(), h->d_done, sizeof(int32_t) * h->nprob, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(
        cudaMemcpyAsync(h->h_done_at.data(), h->d_done_at, sizeof(int64_t) * h->nprob, cudaMemcpyDeviceToHost, s));
    h->h_lowp_span.assign(2 * h->nprob, 0);
    CUDA_TRY(cudaMemcpyAsync(h->h_lowp_span.data(), h->d_lowp_span, sizeof(int64_t) * 2 * h->nprob,
                             cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(&h->h_absorb_count, h->d_absorb_count, sizeof(unsigned long long),
                             cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    RC_TRY(run_check(h, s, cert == 0 ? nullptr : &resumed));
    if (cert >= kCertifyRounds || h->hs_host >= h->opt.max_half_steps) break;
    std::vector<tree_ot_result> chk(h->nprob);
    fill_results(h, chk.data());
    // the FP32 stopping quantity each problem retired on (ring slot of its last half-step)
    std::vector<double> ring_sum((size_t)kResidRing * h->nprob);
    std::vector<unsigned long long> ring_max((size_t)kResidRing * h->nprob);
    CUDA_TRY(cudaMemcpyAsync(ring_sum.data(), h->d_res_sum, sizeof(double) * ring_sum.size(), cudaMemcpyDeviceToHost,
                             s));
    CUDA_TRY(cudaMemcpyAsync(ring_max.data(), h->d_res_max, sizeof(unsigned long long) * ring_max.size(),
                             cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    auto retired_on = [&](int p) {
      const size_t slot = (size_t)((h->h_done_at[p] - 1) % kResidRing);
      if (h->opt.tol_kind == TREE_OT_TOL_MAX) {
        double v;
        std::memcpy(&v, &ring_max[slot * h->nprob + p], sizeof(double));
        return v;
      }
      return ring_sum[slot * h->nprob + p];
    };
    bool resume = false;
    std::fill(resumed.begin(), resumed.end(), 0);
    for (int p = 0; p < h->nprob; ++p) {
      if (!h->h_done[p]) continue;
      const double got = h->opt.tol_kind == TREE_OT_TOL_MAX ? chk[p].max_marginal_l1 : chk[p].residual_sum_l1;
      if (!(got > h->opt.tol)) continue;
      // no gain since the last round: the FP32 iterate's accuracy floor is above tol;
      // a recomputed-cost problem then continues with exact squared distances
      const bool to_exact = !(got < 0.99 * prev_got[p]) && h->probs[p].cost_kind == TREE_OT_COST_SQEUCLID &&
                            !h->h_exact[p];
      if (!(got < 0.99 * prev_got[p]) && !to_exact) continue;
      if (to_exact) h->h_exact[p] = 1;
      prev_got[p] = got;
      // next threshold: the FP32 quantity it retired on, scaled by how far the check missed
      const double crit = retired_on(p);
      const double scale = std::min(0.9, std::max(0.05, 0.8 * h->opt.tol / got));
      h->h_ptol[p] = std::min(h->h_ptol[p], (crit > 0.0 && std::isfinite(crit) ? crit : h->h_ptol[p]) * scale);
      h->h_done[p] = 0;
      // a resumed problem retires within a quarter of its first run (at least 64 half-steps),
      // whether or not its FP32 quantity gets below the new threshold
      h->h_deadline[p] = h->hs_host + std::max<int64_t>(64, h->h_done_at[p] / 4);
      resumed[p] = 1;
      resume = true;
      // the problem's residual ring restarts from zero
      static const double zeros[kResidRing] = {};
      CUDA_TRY(cudaMemcpy2DAsync(h->d_res_sum + p, sizeof(double) * h->nprob, zeros, sizeof(double),
                                 sizeof(double), kResidRing, cudaMemcpyHostToDevice, s));
      CUDA_TRY(cudaMemcpy2DAsync(h->d_res_max + p, sizeof(unsigned long long) * h->nprob, zeros, sizeof(double),
                                 sizeof(double), kResidRing, cudaMemcpyHostToDevice, s));
    }
    if (!resume) break;
    {
      const int32_t any = *std::max_element(h->h_exact.begin(), h->h_exact.end());
      CUDA_TRY(cudaMemcpyAsync(h->d_exact, h->h_exact.data(), sizeof(int32_t) * h->nprob, cudaMemcpyHostToDevice, s));
      if (any != h->any_exact) {
        h->any_exact = any;
        if (use_graph) {
          if (h->graph) cudaGraphExecDestroy(h->graph);
          h->graph = nullptr;
          RC_TRY(build_graph(h, G));
        }
      }
    }
    // A resumed problem must next update the colour it did not update last; half-steps
    // alternate colours for every problem at once, so those whose last colour comes
    // next sit out one half-step (then one more half-step restores the even count the
    // captured graph starts from).
    std::vector<int32_t> later(h->nprob, 0);
    bool any_later = false;
    for (int p = 0; p < h->nprob; ++p)
      if (resumed[p] && (h->h_done_at[p] - 1) % 2 == h->hs_host % 2) {
        later[p] = 1;
        h->h_done[p] = 1;
        any_later = true;
      }
    CUDA_TRY(cudaMemcpyAsync(h->d_ptol, h->h_ptol.data(), sizeof(double) * h->nprob, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(h->d_deadline, h->h_deadline.data(), sizeof(int64_t) * h->nprob, cudaMemcpyHostToDevice,
                             s));
    CUDA_TRY(cudaMemcpyAsync(h->d_done, h->h_done.data(), sizeof(int32_t) * h->nprob, cudaMemcpyHostToDevice, s));
    RC_TRY(recount_live(h, s));
    if (any_later) {
      RC_TRY(queue_half_steps(h, 1, true, s));
      CUDA_TRY(cudaMemcpyAsync(h->h_done.data(), h->d_done, sizeof(int32_t) * h->nprob, cudaMemcpyDeviceToHost, s));
      CUDA_TRY(cudaStreamSynchronize(s));
      for (int p = 0; p < h->nprob; ++p)
        if (later[p]) h->h_done[p] = 0;
      CUDA_TRY(cudaMemcpyAsync(h->d_done, h->h_done.data(), sizeof(int32_t) * h->nprob, cudaMemcpyHostToDevice, s));
      RC_TRY(recount_live(h, s));
      RC_TRY(queue_half_steps(h, 1, true, s));
    }
    CUDA_TRY(cudaStreamSynchronize(s));
  }
  // converged = retired and certified by the check
  std::vector<tree_ot_result> fin(h->nprob);
  fill_results(h, fin.data());
  h->last_status.assign(h->nprob, TREE_OT_OK);
  bool any_nc = false;
  for (int p = 0; p < h->nprob; ++p) {
    const double got = h->opt.tol_kind == TREE_OT_TOL_MAX ? fin[p].max_marginal_l1 : fin[p].residual_sum_l1;
    if (!h->h_done[p] || got > h->opt.tol) {
      h->last_status[p] = TREE_OT_NOT_CONVERGED;
      any_nc = true;
    }
  }
  h->last_wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (results) fill_results(h, results);
  return any_nc ? TREE_OT_NOT_CONVERGED : TREE_OT_OK;
}

int tree_ot_check(tree_ot_handle* h, void* cuda_stream, tree_ot_result* results) {
  g_err.clear();
  if (!h) return fail(TREE_OT_ERR_ARG, "handle is NULL");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (h->h_done.empty()) {
    h->h_done.assign(h->nprob, 0);
    h->h_done_at.assign(h->nprob, 0);
  }
  RC_TRY(run_check(h, s));
  if (results) fill_results(h, results);
  return TREE_OT_OK;
}

int tree_ot_marginals(tree_ot_handle* h, int32_t prob, int32_t node, double* out) {
  g_err.clear();
  if (!h || !out || prob < 0 || prob >= h->nprob || node < 0 || node >= h->prob_nodes[prob])
    return fail(TREE_OT_ERR_ARG, "bad handle, problem, node or output pointer");
  if (!h->have_check) return fail(TREE_OT_ERR_STATE, "call tree_ot_check or tree_ot_solve first");
  const NodeD& nd = h->nodes[h->prob_node_base[prob] + node];
  for (int32_t x = 0; x < nd.n; ++x) {
    double q = 0.0;
    for (int32_t i = 0; i < nd.deg; ++i) q += h->h_marg[h->dedges[h->node_dedges[nd.dedge_begin + i]].off + x];
    out[x] = q / nd.deg;
  }
  return TREE_OT_OK;
}

int tree_ot_residual_history(tree_ot_handle* h, void* cuda_stream, int32_t prob, int64_t first, int64_t count,
                             double* sum_out, double* max_out) {
  g_err.clear();
  if (!h || prob < 0 || prob >= h->nprob || count < 0 || (count > 0 && !sum_out && !max_out))
    return fail(TREE_OT_ERR_ARG, "bad handle, problem, count or output pointers");
  // the terms of iterate t are recorded by half-step t + 1 in ring slot t % kResidRing
  if (first < 0 || first + count > h->hs_host || first < h->hs_host - kResidRing)
    return fail(TREE_OT_ERR_ARG, "iterates " + std::to_string(first) + " .. " + std::to_string(first + count - 1) +
                                     " are not in the history (half-steps done: " + std::to_string(h->hs_host) +
                                     ", kept: " + std::to_string(kResidRing) + ")");
  if (count == 0) return TREE_OT_OK;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  std::vector<double> ring_sum(kResidRing);
  std::vector<unsigned long long> ring_max(kResidRing);
  CUDA_TRY(cudaMemcpy2DAsync(ring_sum.data(), sizeof(double), h->d_res_sum + prob, sizeof(double) * h->nprob,
                             sizeof(double), kResidRing, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpy2DAsync(ring_max.data(), sizeof(double), h->d_res_max + prob,
                             sizeof(unsigned long long) * h->nprob, sizeof(double), kResidRing,
                             cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  for (int64_t i = 0; i < count; ++i) {
    const size_t slot = (size_t)((first + i) % kResidRing);
    if (sum_out) sum_out[i] = ring_sum[slot];
    if (max_out) std::memcpy(&max_out[i], &ring_max[slot], sizeof(double));
  }
  return TREE_OT_OK;
}

int tree_ot_round(tree_ot_handle* h, void* cuda_stream, int32_t side, tree_ot_round_result* results) {
  g_err.clear();
  if (!h || side < -1 || side > 1) return fail(TREE_OT_ERR_ARG, "bad handle or side (-1, 0 or 1)");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // the iterate of every problem: a retired problem's potentials stopped at its retirement
  std::vector<int32_t> done(h->nprob, 0);
  std::vector<int64_t> done_at(h->nprob, 0);
  CUDA_TRY(cudaMemcpyAsync(done.data(), h->d_done, sizeof(int32_t) * h->nprob, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(done_at.data(), h->d_done_at, sizeof(int64_t) * h->nprob, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  std::vector<int32_t> pside(h->nprob);
  std::vector<int64_t> piter(h->nprob);
  for (int p = 0; p < h->nprob; ++p) {
    piter[p] = done[p] ? done_at[p] : h->hs_host;
    if (side < 0 && piter[p] < 1)
      return fail(TREE_OT_ERR_STATE, "problem " + std::to_string(p) +
                                         " has had no half-step: no colour class is known to be matched");
    // half-step t updated colour (t + 1) % 2, so colour t % 2 missed its marginals
    pside[p] = side >= 0 ? side : (int32_t)(piter[p] % 2);
  }
  // buffers on first use
  if (!h->d_rsum) {
    int rc = 0;
    if ((rc = h->alloc(&h->d_rsum, h->vec_len)) || (rc = h->alloc(&h->d_rtgt, h->vec_len)) ||
        (rc = h->alloc(&h->d_rxy, h->vec_len)) || (rc = h->alloc(&h->d_rs2, h->vec_len)) ||
        (rc = h->alloc(&h->d_rer, h->vec_len)) || (rc = h->alloc(&h->d_racc, (int64_t)kRoundAcc * h->edges.size())) ||
        (rc = h->alloc(&h->d_rnmass, (int64_t)h->nodes.size())) || (rc = h->alloc(&h->d_rside, h->nprob)))
      return rc;
    // mass of every fixed node's mu (targets are taken at unit mass)
    std::vector<double> nm(h->nodes.size(), 1.0);
    for (size_t j = 0; j < h->nodes.size(); ++j)
      if (h->nodes[j].fixed) {
        double m = 0.0;
        for (double v : h->mu[j]) m += v;
        nm[j] = m;
      }
    CUDA_TRY(cudaMemcpyAsync(h->d_rnmass, nm.data(), sizeof(double) * nm.size(), cudaMemcpyHostToDevice, s));
  }
  // tasks: 64 rows of every plan with its rows on the rounded side
  h->rtasks.clear();
  h->rt_begin.assign(h->edges.size(), 0);
  h->rt_count.assign(h->edges.size(), 0);
  for (int32_t e = 0; e < (int32_t)h->edges.size(); ++e) {
    for (int k = 0; k < 2; ++k) {
      const int32_t di = 2 * e + k;
      const DEdgeD& d = h->dedges[di];
      if (h->nodes[d.owner].colour != pside[d.prob]) continue;
      h->rt_begin[e] = (int32_t)h->rtasks.size();
      const int32_t n = h->nodes[d.owner].n;
      for (int32_t o = 0; o < n; o += 64) h->rtasks.push_back({di, o, std::min(64, n - o), 0});
      h->rt_count[e] = (int32_t)h->rtasks.size() - h->rt_begin[e];
    }
  }
  if ((int64_t)h->rtasks.size() > h->rtask_cap) {
    int rc = h->alloc(&h->d_rtasks, (int64_t)h->rtasks.size());
    if (rc) return rc;
    h->rtask_cap = (int64_t)h->rtasks.size();
  }
  CUDA_TRY(cudaMemcpyAsync(h->d_rtasks, h->rtasks.data(), sizeof(RoundTask) * h->rtasks.size(),
                           cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(h->d_rside, pside.data(), sizeof(int32_t) * h->nprob, cudaMemcpyHostToDevice, s));
  // the plans' operands, as for the check
  RC_TRY(sync_potentials(h, s));
  if (!h->fp64)
    CUDA_TRY(launch_operand(h->d_f, h->d_Z, h->d_logg, h->d_dedges, h->d_nodes, h->d_probs,
                            (int32_t)h->dedges.size(), 1.0, false, h->d_ah, h->d_al, s));
  CUDA_TRY(cudaMemsetAsync(h->d_rsum, 0, sizeof(double) * h->vec_len, s));
  CUDA_TRY(cudaMemsetAsync(h->d_rs2, 0, sizeof(double) * h->vec_len, s));
  CUDA_TRY(cudaMemsetAsync(h->d_racc, 0, sizeof(double) * kRoundAcc * h->edges.size(), s));
  const RoundArgs a = round_args(h);
  const int p0 = prof_mark(h, s);
  CUDA_TRY(launch_round(a, h->fp64, s));
  prof_span(h, TREE_OT_PROF_ROUND, p0, prof_mark(h, s));
  std::vector<double> acc((size_t)kRoundAcc * h->edges.size()), q(h->vec_len);
  CUDA_TRY(cudaMemcpyAsync(acc.data(), h->d_racc, sizeof(double) * acc.size(), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(q.data(), h->d_rsum, sizeof(double) * q.size(), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  h->round_version = h->pot_version;
  if (!results) return TREE_OT_OK;
  for (int p = 0; p < h->nprob; ++p) {
    tree_ot_round_result r{};
    r.side = pside[p];
    r.half_steps = piter[p];
    // stopping sum of the input plans from their own FP64 marginals (q of every directed edge)
    double rsum = 0.0;
    int32_t dmax = 1;
    const int32_t nb = h->prob_node_base[p], J = h->prob_nodes[p];
    for (int32_t j = nb; j < nb + J; ++j) {
      const NodeD& nd = h->nodes[j];
      dmax = std::max(dmax, nd.n);
      if (nd.fixed) {
        const DEdgeD& d = h->dedges[h->node_dedges[nd.dedge_begin]];
        for (int32_t x = 0; x < nd.n; ++x) rsum += std::fabs(q[d.off + x] - h->mu[j][x]);
      } else {
        for (int32_t x = 0; x < nd.n; ++x) {
          double qb = 0.0;
          for (int32_t i = 0; i < nd.deg; ++i) qb += q[h->dedges[h->node_dedges[nd.dedge_begin + i]].off + x];
          qb /= nd.deg;
          for (int32_t i = 0; i < nd.deg; ++i)
            rsum += std::fabs(q[h->dedges[h->node_dedges[nd.dedge_begin + i]].off + x] - qb);
        }
      }
    }
    double tc = 0.0, trc = 0.0, cinf = 0.0;
    for (int32_t e = h->prob_edge_base[p]; e < h->prob_edge_base[p] + J - 1; ++e) {
      const double* v = &acc[(size_t)kRoundAcc * e];
      tc += v[0];
      trc += v[1] + (v[3] > 0.0 ? v[2] / v[3] : 0.0);
      double cm;
      std::memcpy(&cm, &v[4], sizeof(double));
      cinf = std::max(cinf, cm);
    }
    r.residual_sum_l1 = rsum;
    r.transport_cost = tc;
    r.rounded_transport_cost = trc;
    r.c_inf = cinf;
    r.bound = 2.0 * h->probs[p].eps * (J - 1) * std::log((double)dmax) + 4.0 * cinf * rsum;
    results[p] = r;
  }
  return TREE_OT_OK;
}

int tree_ot_round_plan(tree_ot_handle* h, void* cuda_stream, int32_t prob, int32_t edge, double* plan_out,
                       int64_t ld) {
  g_err.clear();
  if (!h || !plan_out || prob < 0 || prob >= h->nprob || edge < 0 || edge >= h->prob_nodes[prob] - 1)
    return fail(TREE_OT_ERR_ARG, "bad handle, problem, edge or output pointer");
  const int32_t e = h->prob_edge_base[prob] + edge;
  if (ld < h->edges[e].nb) return fail(TREE_OT_ERR_ARG, "ld must be at least the column count n_b");
  if (h->round_version != h->pot_version || h->rt_count.empty())
    return fail(TREE_OT_ERR_STATE, "call tree_ot_round after the potentials last changed");
  RoundArgs a = round_args(h);
  a.tasks = h->d_rtasks + h->rt_begin[e];
  a.ntasks = h->rt_count[e];
  a.plan_out = plan_out;
  a.plan_ld = ld;
  CUDA_TRY(launch_round_plan(a, h->fp64, (cudaStream_t)cuda_stream));
  return TREE_OT_OK;
}

int tree_ot_get_potentials(tree_ot_handle* h, void* cuda_stream, int32_t prob, int32_t dedge, double* out) {
  g_err.clear();
  if (!h || !out || prob < 0 || prob >= h->nprob || dedge < 0 || dedge >= 2 * (h->prob_nodes[prob] - 1))
    return fail(TREE_OT_ERR_ARG, "bad handle, problem, directed edge or output pointer");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const DEdgeD& d = h->dedges[2 * h->prob_edge_base[prob] + dedge];
  const int32_t n = h->nodes[d.owner].n;
  double z = 0.0;
  RC_TRY(sync_potentials(h, s));
  CUDA_TRY(cudaMemcpyAsync(out, h->d_f + d.off, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(&z, h->d_Z + d.owner, sizeof(double), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  const double eps = h->probs[prob].eps;
  for (int32_t x = 0; x < n; ++x) out[x] -= eps * z;
  return TREE_OT_OK;
}

int tree_ot_set_potentials(tree_ot_handle* h, void* cuda_stream, int32_t prob, int32_t dedge, const double* in) {
  g_err.clear();
  if (!h || !in || prob < 0 || prob >= h->nprob || dedge < 0 || dedge >= 2 * (h->prob_nodes[prob] - 1))
    return fail(TREE_OT_ERR_ARG, "bad handle, problem, directed edge or input pointer");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int32_t di = 2 * h->prob_edge_base[prob] + dedge;
  const DEdgeD& d = h->dedges[di];
  const int32_t n = h->nodes[d.owner].n;
  for (int32_t x = 0; x < n; ++x)
    if (!std::isfinite(in[x])) return fail(TREE_OT_ERR_NONFINITE, "potential entries must be finite");
  ++h->pot_version;
  double z = 0.0;
  CUDA_TRY(cudaMemcpyAsync(&z, h->d_Z + d.owner, sizeof(double), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  std::vector<double> v(in, in + n);
  const double eps = h->probs[prob].eps;
  for (int32_t x = 0; x < n; ++x) v[x] += eps * z;
  RC_TRY(sync_potentials(h, s));
  CUDA_TRY(cudaMemcpyAsync(h->d_f + d.off, v.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
  CUDA_TRY(launch_operand(h->d_f, nullptr, h->d_logg, h->d_dedges + di, h->d_nodes, h->d_probs, 1, kLog2e, true,
                          h->d_hh, h->d_hl, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  h->have_check = false;
  return TREE_OT_OK;
}

namespace {
// Validates the (problem, directed edge) items of a batched potential call,
// uploads their global directed-edge indices into the handle's item buffer
// (grown as needed) and returns the device list and record array.
int stage_items(tree_ot_handle* h, cudaStream_t s, int32_t count, const int32_t* probs, const int32_t* dedges,
                int64_t ld, int32_t** d_dlist, DEdgeD** d_picked) {
  std::vector<int32_t> dlist(count);
  for (int32_t i = 0; i < count; ++i) {
    const int32_t p = probs[i], d = dedges[i];
    if (p < 0 || p >= h->nprob || d < 0 || d >= 2 * (h->prob_nodes[p] - 1))
      return fail(TREE_OT_ERR_ARG, "item " + std::to_string(i) + ": bad problem or directed edge");
    dlist[i] = 2 * h->prob_edge_base[p] + d;
    if (h->nodes[h->dedges[dlist[i]].owner].n > ld)
      return fail(TREE_OT_ERR_ARG, "item " + std::to_string(i) + ": row stride ld is smaller than n_owner");
  }
  if (count > h->setbuf_cap) {
    if (h->d_setbuf) {
      CUDA_TRY(cudaStreamSynchronize(s));
      cudaFree(h->d_setbuf);
      h->d_setbuf = nullptr;
      h->setbuf_cap = 0;
    }
    CUDA_TRY(cudaMalloc(&h->d_setbuf, align_up(sizeof(int32_t) * (size_t)count, 256) + sizeof(DEdgeD) * (size_t)count));
    h->setbuf_cap = count;
  }
  *d_dlist = (int32_t*)h->d_setbuf;
  *d_picked = (DEdgeD*)((char*)h->d_setbuf + align_up(sizeof(int32_t) * (size_t)h->setbuf_cap, 256));
  CUDA_TRY(cudaMemcpyAsync(*d_dlist, dlist.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice, s));
  // the pageable source is read before the call returns, so dlist may go out of scope
  return TREE_OT_OK;
}
}  // namespace

int tree_ot_get_potentials_batch(tree_ot_handle* h, void* cuda_stream, int32_t count, const int32_t* probs,
                                 const int32_t* dedges, float* values, int64_t ld, uint32_t flags) {
  g_err.clear();
  if (!h || count < 0 || (count > 0 && (!probs || !dedges || !values)))
    return fail(TREE_OT_ERR_ARG, "bad handle, count or pointer");
  if (count == 0) return TREE_OT_OK;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int32_t* d_dlist = nullptr;
  DEdgeD* d_picked = nullptr;
  RC_TRY(stage_items(h, s, count, probs, dedges, ld, &d_dlist, &d_picked));
  RC_TRY(sync_potentials(h, s));
  CUDA_TRY(launch_get_potentials(d_dlist, count, h->d_dedges, h->d_nodes, h->d_probs, h->d_Z, h->d_f, values, ld,
                                 (flags & TREE_OT_GET_CENTRED) != 0, s));
  return TREE_OT_OK;
}

int tree_ot_set_potentials_batch(tree_ot_handle* h, void* cuda_stream, int32_t count, const int32_t* probs,
                                 const int32_t* dedges, const float* values, int64_t ld) {
  g_err.clear();
  if (!h || count < 0 || (count > 0 && (!probs || !dedges || !values)))
    return fail(TREE_OT_ERR_ARG, "bad handle, count or pointer");
  if (count == 0) return TREE_OT_OK;
  ++h->pot_version;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int32_t* d_dlist = nullptr;
  DEdgeD* d_picked = nullptr;
  RC_TRY(stage_items(h, s, count, probs, dedges, ld, &d_dlist, &d_picked));
  CUDA_TRY(cudaMemsetAsync(h->d_scan, 0, sizeof(int32_t), s));
  CUDA_TRY(launch_set_potentials(values, ld, d_dlist, count, h->d_dedges, h->d_nodes, h->d_probs, h->d_Z, h->d_f,
                                 d_picked, h->d_scan, false, s));
  int32_t bad = 0;
  CUDA_TRY(cudaMemcpyAsync(&bad, h->d_scan, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (bad) return fail(TREE_OT_ERR_NONFINITE, "potential entries must be finite");
  RC_TRY(sync_potentials(h, s));
  CUDA_TRY(launch_set_potentials(values, ld, d_dlist, count, h->d_dedges, h->d_nodes, h->d_probs, h->d_Z, h->d_f,
                                 d_picked, h->d_scan, true, s));
  CUDA_TRY(launch_operand(h->d_f, nullptr, h->d_logg, d_picked, h->d_nodes, h->d_probs, count, kLog2e, true, h->d_hh,
                          h->d_hl, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  h->have_check = false;
  return TREE_OT_OK;
}

int tree_ot_profile(tree_ot_handle* h, int32_t enable) {
  g_err.clear();
  if (!h) return fail(TREE_OT_ERR_ARG, "handle is NULL");
  h->prof_on = enable != 0;
  h->prof_used = 0;
  h->prof_spans.clear();
  return TREE_OT_OK;
}

int tree_ot_profile_read(tree_ot_handle* h, double* ms, int64_t* launches, int32_t ncat) {
  g_err.clear();
  if (!h || ncat < 0 || (ncat > 0 && !ms && !launches)) return fail(TREE_OT_ERR_ARG, "bad handle or outputs");
  std::vector<double> t(TREE_OT_PROF_CATEGORIES, 0.0);
  std::vector<int64_t> n(TREE_OT_PROF_CATEGORIES, 0);
  if (h->prof_used > 0) CUDA_TRY(cudaEventSynchronize(h->prof_ev[h->prof_used - 1]));
  for (const auto& sp : h->prof_spans) {
    float v = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&v, h->prof_ev[sp.i0], h->prof_ev[sp.i1]));
    t[sp.cat] += v;
    n[sp.cat] += 1;
  }
  for (int32_t c = 0; c < ncat && c < TREE_OT_PROF_CATEGORIES; ++c) {
    if (ms) ms[c] = t[c];
    if (launches) launches[c] = n[c];
  }
  h->prof_used = 0;
  h->prof_spans.clear();
  return TREE_OT_OK;
}

int tree_ot_plan_stats(tree_ot_handle* h, int64_t* stats, int32_t nstats) {
  g_err.clear();
  if (!h || !stats || nstats < 0) return fail(TREE_OT_ERR_ARG, "bad handle or stats pointer");
  int64_t sk_form = 0;  // the shared-kernel product: 0 none, 1 mma.sync, 2 tcgen05 one CTA per tile, 3 CTA pairs
  for (const auto& g : h->sk)
    for (int c = 0; c < 2; ++c)
      if (g.args[c].ncols > 0)
        sk_form = std::max<int64_t>(sk_form, g.args[c].use_tc ? (g.args[c].tc_pair ? 3 : 2) : 1);
  const int64_t v[16] = {(int64_t)h->dedges.size(),
                        (int64_t)h->edges.size(),
                        h->elems,
                        h->matrix_bytes,
                        (int64_t)h->tasks[0].size(),
                        (int64_t)h->tasks[1].size(),
                        h->device_bytes,
                        (int64_t)h->chunks[0].size(),
                        (int64_t)h->chunks[1].size(),
                        (int64_t)h->rec_ob,
                        (int64_t)h->grid_mult,
                        (int64_t)h->rec_variant,
                        (int64_t)h->dense_tma,
                        (int64_t)h->persistent,
                        (int64_t)((h->node_defer[0] ? 1 : 0) | (h->node_defer[1] ? 2 : 0)),
                        sk_form};
  for (int32_t i = 0; i < nstats && i < 16; ++i) stats[i] = v[i];
  return TREE_OT_OK;
}

int tree_ot_edge_apply_noalloc(const float* cost, int64_t ld, int32_t n_rows, int32_t n_cols, const double* g,
                               double eps, double* m_out, void* cuda_stream) {
  g_err.clear();
  if (!cost || !g || !m_out) return fail(TREE_OT_ERR_ARG, "cost, g and m_out must be device pointers");
  if (n_rows < 1 || n_cols < 1 || ld < n_cols || (ld % 4) != 0 || ((uintptr_t)cost % 16) != 0)
    return fail(TREE_OT_ERR_ARG, "need n_rows, n_cols >= 1, ld >= n_cols, ld % 4 == 0 and a 16-byte aligned cost");
  if (!(eps > 0.0) || !std::isfinite(eps)) return fail(TREE_OT_ERR_EPS, "eps must be positive and finite");
  float* scratch = nullptr;
  int64_t cap = 0;
  CUDA_TRY(noalloc_scratch(&scratch, &cap));
  const int64_t need = noalloc_scratch_floats_needed(n_rows, n_cols);
  if (need > cap)
    return fail(TREE_OT_ERR_ARG, "tree_ot_edge_apply_noalloc: " + std::to_string(n_rows) + " x " +
                                     std::to_string(n_cols) + " needs " + std::to_string(need) +
                                     " scratch floats, more than the fixed " + std::to_string(cap));
  float shi, slo;
  split_positive(kLog2e / eps, &shi, &slo);
  CUDA_TRY(launch_edge_apply_noalloc(cost, ld, n_rows, n_cols, g, shi, slo, m_out, scratch,
                                     (cudaStream_t)cuda_stream));
  return TREE_OT_OK;
}

}  // extern "C"
