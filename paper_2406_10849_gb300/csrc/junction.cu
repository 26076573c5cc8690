// Coupled MOT on a modified junction tree (Sec. 4): the separator update of
// proposition prop:general_algo for general (nested) inclusion sequences,
// the plans of prop:local_reg_dual, the stopping quantity and the transport
// cost, all in log domain and FP64 on the device.
//
// Every step is one of a few tensor operations over variable subsets, and each
// is written as one generic "op": an output tensor over variables T, a set of
// reduced variables R, and up to kJtMaxIn inputs, each a tensor over a subset of
// T u R (broadcast along the variables it lacks, by stride 0) with a
// coefficient:
//     out[t] = log sum_{r in R} exp( sum_j alpha_j in_j[t, r] )      (R empty: the sum itself)
// The planner (host) turns one half-step of a colour into a few stages of such
// ops -- all separators of the colour in each stage, the ops of a stage
// independent -- and the op kernel runs a stage with one warp per output
// (lanes over the reduced index) or, without reduced variables, one lane per
// output.  With k_i the projection onto s n c_i of clique c_i's kernel, cost
// and its other separator's dual variable and factor m (s's own factor m_s
// left out of every k_i, so that mu_gamma cancels in v_{l+1}; the same reading
// as the FP64 oracle), the stages of a half-step are
//   k_i;  q_2 = (k_1 + k_2)/2;  Pq_i = P_{s n c_i} q_{i-1}, q_i = ((i-1) Pq_i + k_i)/i  (i = 3..l);
//   Pg = P_gamma q_l;  a_l = q_l - Pg (x) 1;  a_i = q_i + (a_{i+1} - Pq_{i+1}) (x) 1  (i = l-1..2);
//   u_1 = a_2 - k_1,  u_i = a_i - k_i;   and for l = 1:  u_1 = -(P_gamma k_1) (x) 1.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/tree_ot.h"
#include "internal.h"

namespace treeot {
namespace {

constexpr int kJtMaxDims = 8;  // output plus reduced variables of one op
constexpr int kJtMaxIn = 5;   // a log plan: the cost, and each of two separators' dual and factor m
constexpr int kJtWarps = 8;    // warps per CTA of the op kernels

struct JtIn {
  const double* p64;
  const float* p32;
  double alpha;
  int64_t stride[kJtMaxDims];  // per op dimension (output dims, then reduced dims); 0 where absent
};

struct JtOp {
  int32_t nt, nr, nin, pad;
  int32_t dim[kJtMaxDims];
  int64_t tcount, rcount;
  double* out;  // row-major over the output dims (the last fastest)
  JtIn in[kJtMaxIn];
};

// a sum over a tensor (the stopping quantity and the transport cost):
//   kind 0: sum |exp a - exp b|,  kind 1: sum exp a,  kind 2: sum exp(a) c
struct JtSum {
  const double* a;
  const double* b;
  const float* c;
  int64_t n;
  int32_t slot, kind;
};

__device__ __forceinline__ double jt_value(const JtOp& op, const int64_t* off) {
  double v = 0.0;
  for (int j = 0; j < op.nin; ++j) {
    const JtIn& in = op.in[j];
    v += in.alpha * (in.p32 ? (double)in.p32[off[j]] : in.p64[off[j]]);
  }
  return v;
}

__device__ __forceinline__ int jt_find(const int64_t* start, int32_t n, int64_t w) {
  int lo = 0, hi = n;  // start[0..n], start[0] = 0
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (start[mid] <= w) lo = mid; else hi = mid;
  }
  return lo;
}

// one stage of ops; start[o] = the first work unit of op o (a warp per output
// when the op reduces, a lane per output otherwise), start[nops] = the total
__global__ void __launch_bounds__(32 * kJtWarps) jt_op_kernel(const JtOp* ops, const int64_t* start, int32_t nops) {
  const int lane = threadIdx.x & 31;
  const int64_t w = (int64_t)blockIdx.x * kJtWarps + (threadIdx.x >> 5);
  if (w >= start[nops]) return;
  const JtOp& op = ops[jt_find(start, nops, w)];
  const int64_t unit = w - start[jt_find(start, nops, w)];
  int64_t t = unit;
  if (op.rcount == 1) {  // no reduction: one output per lane
    t = unit * 32 + lane;
    if (t >= op.tcount) return;
  }
  int64_t base[kJtMaxIn];
  for (int j = 0; j < kJtMaxIn; ++j) base[j] = 0;
  int64_t rem = t;
  for (int k = op.nt - 1; k >= 0; --k) {
    const int64_t x = rem % op.dim[k];
    rem /= op.dim[k];
    for (int j = 0; j < op.nin; ++j) base[j] += x * op.in[j].stride[k];
  }
  if (op.rcount == 1) {
    op.out[t] = jt_value(op, base);
    return;
  }
  double m = -INFINITY, s = 0.0;
  for (int64_t r = lane; r < op.rcount; r += 32) {
    int64_t off[kJtMaxIn];
    for (int j = 0; j < kJtMaxIn; ++j) off[j] = base[j];
    int64_t rr = r;
    for (int k = op.nr - 1; k >= 0; --k) {
      const int64_t x = rr % op.dim[op.nt + k];
      rr /= op.dim[op.nt + k];
      for (int j = 0; j < op.nin; ++j) off[j] += x * op.in[j].stride[op.nt + k];
    }
    const double v = jt_value(op, off);
    if (v > m) {
      s = s * exp(m - v) + 1.0;  // (m = -inf: s = 0)
      m = v;
    } else if (v > -INFINITY) {
      s += exp(v - m);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {  // merge the lanes' (max, sum) pairs
    const double m2 = __shfl_xor_sync(0xffffffffu, m, o), s2 = __shfl_xor_sync(0xffffffffu, s, o);
    const double M = fmax(m, m2);
    if (M > -INFINITY) {
      s = (m > -INFINITY ? s * exp(m - M) : 0.0) + (m2 > -INFINITY ? s2 * exp(m2 - M) : 0.0);
      m = M;
    }
  }
  if (lane == 0) op.out[t] = m > -INFINITY ? m + log(s) : -INFINITY;
}

// sums over tensors into slots; one CTA per (item, 8192-entry block)
__global__ void __launch_bounds__(256) jt_sum_kernel(const JtSum* items, const int64_t* start, int32_t nitems,
                                                     double* slots) {
  __shared__ double red[8];
  if ((int64_t)blockIdx.x >= start[nitems]) return;
  const int it = jt_find(start, nitems, blockIdx.x);
  const JtSum& q = items[it];
  const int64_t i0 = (blockIdx.x - start[it]) * 8192;
  const int64_t i1 = min(q.n, i0 + 8192);
  double acc = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += 256) {
    const double ea = exp(q.a[i]);
    acc += q.kind == 0 ? fabs(ea - exp(q.b[i])) : q.kind == 1 ? ea : (ea > 0.0 ? ea * (double)q.c[i] : 0.0);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    atomicAdd(&slots[q.slot], t);
  }
}

// per separator: r_s = sum of its |differences| + |total mass - 1| when unconstrained;
// out = (sum_s r_s, max_s r_s)
__global__ void jt_residual_finish_kernel(const double* slots, const int32_t* constrained, int32_t nsep, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double sum = 0.0, mx = 0.0;
  for (int s = 0; s < nsep; ++s) {
    const double r = slots[2 * s] + (constrained[s] ? 0.0 : fabs(slots[2 * s + 1] - 1.0));
    sum += r;
    mx = fmax(mx, r);
  }
  out[0] = sum;
  out[1] = mx;
}

__global__ void jt_exp_kernel(const double* a, double* out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = exp(a[i]);
}

}  // namespace
}  // namespace treeot

using namespace treeot;

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

namespace {

struct Tensor {
  std::vector<int32_t> vars;  // axis order
  int64_t off = 0;            // in the FP64 arena
  int64_t size = 1;
};

struct Stage {
  std::vector<JtOp> ops;  // host copy (pointers filled once the arena exists)
  JtOp* d_ops = nullptr;
  int64_t* d_start = nullptr;
  int64_t units = 0;
};

}  // namespace

struct tree_ot_jt_handle {
  int32_t nvars = 0, ncl = 0, nsep = 0;
  double eps = 0.0;
  std::vector<int32_t> vsize;
  std::vector<std::vector<int32_t>> cvars, svars, scl, sgamma;
  std::vector<std::vector<std::pair<int32_t, int32_t>>> clsep;  // per clique: (separator, position)
  std::vector<int32_t> colour;
  std::vector<std::vector<Tensor>> dual;  // [s][i] over s n c_i (separator order)
  std::vector<Tensor> logm;               // [s] over gamma (constrained separators)
  std::vector<Tensor> logplan;            // [c] over the clique's variables
  std::vector<int64_t> cost_off;          // [c] offset in the FP32 cost arena
  std::vector<int64_t> cost_size;
  int64_t arena_len = 0, cost_len = 0;
  double* d_arena = nullptr;
  float* d_cost = nullptr;
  double* d_slots = nullptr;   // 2 per separator
  int32_t* d_constrained = nullptr;
  double* d_res = nullptr;     // (sum, max)
  double* d_tmp = nullptr;     // plan read-back buffer
  int64_t tmp_len = 0;
  std::vector<Stage> stages[2];
  std::vector<Stage> res_stages;
  std::vector<JtSum> res_sums, tc_sums;
  JtSum* d_res_sums = nullptr;
  JtSum* d_tc_sums = nullptr;
  int64_t* d_res_start = nullptr;
  int64_t* d_tc_start = nullptr;
  int64_t res_blocks = 0, tc_blocks = 0;
  int64_t hs = 0;
  cudaGraphExec_t pair = nullptr;   // two half-steps (colour 0, then 1) captured once, replayed
  cudaStream_t pair_stream = nullptr;
  std::vector<void*> owned;
  ~tree_ot_jt_handle() {
    if (pair) cudaGraphExecDestroy(pair);
    for (void* p : owned) cudaFree(p);
  }
};

namespace {

int jt_fail(int code, const std::string& msg) {
  set_last_error(msg);
  return code;
}

int jt_cuda(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return TREE_OT_OK;
  return jt_fail(e == cudaErrorMemoryAllocation ? TREE_OT_ERR_OOM : TREE_OT_ERR_CUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}

#define JT_TRY(call)                              \
  do {                                            \
    const int rc_ = (call);                       \
    if (rc_ != TREE_OT_OK) return rc_;            \
  } while (0)

template <class T>
int jt_alloc(tree_ot_jt_handle* h, T** p, int64_t count) {
  *p = nullptr;
  const cudaError_t e = cudaMalloc((void**)p, sizeof(T) * (size_t)std::max<int64_t>(count, 1));
  if (e != cudaSuccess) return jt_cuda(e, "cudaMalloc");
  h->owned.push_back(*p);
  return TREE_OT_OK;
}

std::vector<int32_t> inter(const std::vector<int32_t>& a, const std::vector<int32_t>& b) {
  std::vector<int32_t> out;
  for (int32_t v : a)
    if (std::find(b.begin(), b.end(), v) != b.end()) out.push_back(v);
  return out;
}

bool subset(const std::vector<int32_t>& a, const std::vector<int32_t>& b) {
  for (int32_t v : a)
    if (std::find(b.begin(), b.end(), v) == b.end()) return false;
  return true;
}

Tensor new_tensor(tree_ot_jt_handle* h, const std::vector<int32_t>& vars) {
  Tensor t;
  t.vars = vars;
  for (int32_t v : vars) t.size *= h->vsize[v];
  t.off = h->arena_len;
  h->arena_len += t.size;
  return t;
}

// an input: a tensor in the FP64 arena or a clique's FP32 cost
struct Src {
  const std::vector<int32_t>* vars;
  int64_t off;
  bool cost;
  double alpha;
};
Src src(const Tensor& t, double alpha) { return Src{&t.vars, t.off, false, alpha}; }

// out over out.vars, reduced over `red`; op pointers are offsets until resolve()
JtOp make_op(const tree_ot_jt_handle* h, const Tensor& out, const std::vector<int32_t>& red,
             const std::vector<Src>& ins) {
  JtOp op{};
  std::vector<int32_t> dims = out.vars;
  dims.insert(dims.end(), red.begin(), red.end());
  // by construction: dims are a clique's variables (at most kJtMaxDims, checked at
  // create) and an op has at most kJtMaxIn inputs
  if ((int)dims.size() > kJtMaxDims || (int)ins.size() > kJtMaxIn) std::abort();
  op.nt = (int32_t)out.vars.size();
  op.nr = (int32_t)red.size();
  op.nin = (int32_t)ins.size();
  op.tcount = 1;
  op.rcount = 1;
  for (int k = 0; k < (int)dims.size(); ++k) {
    op.dim[k] = h->vsize[dims[k]];
    (k < op.nt ? op.tcount : op.rcount) *= op.dim[k];
  }
  op.out = reinterpret_cast<double*>((intptr_t)out.off);
  for (int j = 0; j < op.nin; ++j) {
    const Src& s = ins[j];
    JtIn& in = op.in[j];
    in.alpha = s.alpha;
    if (s.cost)
      in.p32 = reinterpret_cast<const float*>((intptr_t)(s.off + 1));  // +1: tells resolve() it is a cost
    else
      in.p64 = reinterpret_cast<const double*>((intptr_t)s.off);
    // row-major strides of the input's own axes
    const std::vector<int32_t>& iv = *s.vars;
    std::vector<int64_t> st(iv.size(), 1);
    for (int a = (int)iv.size() - 2; a >= 0; --a) st[a] = st[a + 1] * h->vsize[iv[a + 1]];
    for (int k = 0; k < (int)dims.size(); ++k) {
      in.stride[k] = 0;
      for (size_t a = 0; a < iv.size(); ++a)
        if (iv[a] == dims[k]) in.stride[k] = st[a];
    }
  }
  return op;
}

void resolve(const tree_ot_jt_handle* h, JtOp& op) {
  op.out = h->d_arena + (intptr_t)op.out;
  for (int j = 0; j < op.nin; ++j) {
    JtIn& in = op.in[j];
    if (in.p32) {
      in.p32 = h->d_cost + ((intptr_t)in.p32 - 1);
      in.p64 = nullptr;
    } else {
      in.p64 = h->d_arena + (intptr_t)in.p64;
    }
  }
}

int upload_stage(tree_ot_jt_handle* h, Stage& st, cudaStream_t s) {
  std::vector<int64_t> start(st.ops.size() + 1, 0);
  for (size_t o = 0; o < st.ops.size(); ++o) {
    resolve(h, st.ops[o]);
    const JtOp& op = st.ops[o];
    start[o + 1] = start[o] + (op.rcount == 1 ? (op.tcount + 31) / 32 : op.tcount);
  }
  st.units = start.back();
  JT_TRY(jt_alloc(h, &st.d_ops, (int64_t)st.ops.size()));
  JT_TRY(jt_alloc(h, &st.d_start, (int64_t)start.size()));
  JT_TRY(jt_cuda(cudaMemcpyAsync(st.d_ops, st.ops.data(), sizeof(JtOp) * st.ops.size(), cudaMemcpyHostToDevice, s),
                 "upload ops"));
  JT_TRY(jt_cuda(cudaMemcpyAsync(st.d_start, start.data(), sizeof(int64_t) * start.size(), cudaMemcpyHostToDevice, s),
                 "upload ops"));
  return TREE_OT_OK;
}

int run_stage(const Stage& st, cudaStream_t s) {
  if (st.ops.empty() || st.units == 0) return TREE_OT_OK;
  const int64_t blocks = (st.units + kJtWarps - 1) / kJtWarps;
  jt_op_kernel<<<(unsigned)blocks, 32 * kJtWarps, 0, s>>>(st.d_ops, st.d_start, (int32_t)st.ops.size());
  return jt_cuda(cudaGetLastError(), "junction-tree op launch");
}

int upload_sums(tree_ot_jt_handle* h, const std::vector<JtSum>& items, JtSum** d_items, int64_t** d_start,
                int64_t* blocks, cudaStream_t s) {
  std::vector<int64_t> start(items.size() + 1, 0);
  for (size_t i = 0; i < items.size(); ++i) start[i + 1] = start[i] + (items[i].n + 8191) / 8192;
  *blocks = start.back();
  JT_TRY(jt_alloc(h, d_items, (int64_t)items.size()));
  JT_TRY(jt_alloc(h, d_start, (int64_t)start.size()));
  if (!items.empty())
    JT_TRY(jt_cuda(cudaMemcpyAsync(*d_items, items.data(), sizeof(JtSum) * items.size(), cudaMemcpyHostToDevice, s),
                   "upload sums"));
  JT_TRY(jt_cuda(cudaMemcpyAsync(*d_start, start.data(), sizeof(int64_t) * start.size(), cudaMemcpyHostToDevice, s),
                 "upload sums"));
  return TREE_OT_OK;
}

// the stages of one colour's half-step (see the top of the file)
void plan_half_step(tree_ot_jt_handle* h, int colour, std::vector<Stage>& stages) {
  struct SepWork {
    int32_t s, l;
    std::vector<std::vector<int32_t>> sets;
    std::vector<int32_t> g;
    std::vector<Tensor> k, q, Pq, a;
    Tensor Pg;
  };
  std::vector<SepWork> work;
  int32_t lmax = 1;
  for (int32_t s = 0; s < h->nsep; ++s) {
    if (h->colour[s] != colour) continue;
    SepWork w;
    w.s = s;
    w.l = (int32_t)h->scl[s].size();
    for (int32_t c : h->scl[s]) w.sets.push_back(inter(h->svars[s], h->cvars[c]));
    w.g = h->sgamma[s];
    lmax = std::max(lmax, w.l);
    work.push_back(std::move(w));
  }
  // temporaries
  for (SepWork& w : work) {
    for (int i = 0; i < w.l; ++i) w.k.push_back(new_tensor(h, w.sets[i]));
    w.q.resize(w.l + 1);
    w.Pq.resize(w.l + 1);
    w.a.resize(w.l + 1);
    for (int i = 2; i <= w.l; ++i) {
      w.q[i] = new_tensor(h, w.sets[i - 1]);
      if (i >= 3) w.Pq[i] = new_tensor(h, w.sets[i - 1]);
      w.a[i] = new_tensor(h, w.sets[i - 1]);
    }
    w.Pg = new_tensor(h, w.g);
  }
  auto minus = [](const std::vector<int32_t>& a, const std::vector<int32_t>& b) {
    std::vector<int32_t> out;
    for (int32_t v : a)
      if (std::find(b.begin(), b.end(), v) == b.end()) out.push_back(v);
    return out;
  };
  // k_i: the clique's log kernel, its other separator's factor m and dual variable
  Stage sk;
  for (SepWork& w : work)
    for (int i = 0; i < w.l; ++i) {
      const int32_t c = h->scl[w.s][i];
      std::vector<Src> ins;
      ins.push_back(Src{&h->cvars[c], h->cost_off[c], true, -1.0 / h->eps});
      for (const auto& si : h->clsep[c]) {
        if (si.first == w.s && si.second == i) continue;
        ins.push_back(src(h->dual[si.first][si.second], 1.0));
        if (!h->sgamma[si.first].empty()) ins.push_back(src(h->logm[si.first], 1.0));
      }
      sk.ops.push_back(make_op(h, w.k[i], minus(h->cvars[c], w.sets[i]), ins));
    }
  stages.push_back(std::move(sk));
  // the geometric chain
  {
    Stage st;
    for (SepWork& w : work)
      if (w.l >= 2) st.ops.push_back(make_op(h, w.q[2], {}, {src(w.k[0], 0.5), src(w.k[1], 0.5)}));
    stages.push_back(std::move(st));
  }
  for (int i = 3; i <= lmax; ++i) {
    Stage sp, sq;
    for (SepWork& w : work) {
      if (w.l < i) continue;
      sp.ops.push_back(make_op(h, w.Pq[i], minus(w.sets[i - 2], w.sets[i - 1]), {src(w.q[i - 1], 1.0)}));
      sq.ops.push_back(make_op(h, w.q[i], {}, {src(w.Pq[i], (i - 1.0) / i), src(w.k[i - 1], 1.0 / i)}));
    }
    stages.push_back(std::move(sp));
    stages.push_back(std::move(sq));
  }
  // P_gamma of q_l (or of k_1 when l = 1)
  {
    Stage st;
    for (SepWork& w : work) {
      const Tensor& top = w.l >= 2 ? w.q[w.l] : w.k[0];
      st.ops.push_back(make_op(h, w.Pg, minus(top.vars, w.g), {src(top, 1.0)}));
    }
    stages.push_back(std::move(st));
  }
  // a_l, then down the chain
  {
    Stage st;
    for (SepWork& w : work)
      if (w.l >= 2) st.ops.push_back(make_op(h, w.a[w.l], {}, {src(w.q[w.l], 1.0), src(w.Pg, -1.0)}));
    stages.push_back(std::move(st));
  }
  for (int down = 1; down <= lmax - 2; ++down) {
    Stage st;
    for (SepWork& w : work) {
      const int i = w.l - down;
      if (i < 2) continue;
      st.ops.push_back(make_op(h, w.a[i], {}, {src(w.q[i], 1.0), src(w.a[i + 1], 1.0), src(w.Pq[i + 1], -1.0)}));
    }
    stages.push_back(std::move(st));
  }
  // the new dual variables
  {
    Stage st;
    for (SepWork& w : work) {
      std::vector<Tensor>& u = h->dual[w.s];
      if (w.l == 1) {
        st.ops.push_back(make_op(h, u[0], {}, {src(w.Pg, -1.0)}));
        continue;
      }
      st.ops.push_back(make_op(h, u[0], {}, {src(w.a[2], 1.0), src(w.k[0], -1.0)}));
      for (int i = 2; i <= w.l; ++i)
        st.ops.push_back(make_op(h, u[i - 1], {}, {src(w.a[i], 1.0), src(w.k[i - 1], -1.0)}));
    }
    stages.push_back(std::move(st));
  }
  std::vector<Stage> kept;
  for (Stage& st : stages)
    if (!st.ops.empty()) kept.push_back(std::move(st));
  stages = std::move(kept);
}

// log plans, their projections and the sums of the stopping quantity and transport cost
void plan_residual(tree_ot_jt_handle* h) {
  auto minus = [](const std::vector<int32_t>& a, const std::vector<int32_t>& b) {
    std::vector<int32_t> out;
    for (int32_t v : a)
      if (std::find(b.begin(), b.end(), v) == b.end()) out.push_back(v);
    return out;
  };
  Stage plans;
  for (int32_t c = 0; c < h->ncl; ++c) {
    h->logplan.push_back(new_tensor(h, h->cvars[c]));
    std::vector<Src> ins;
    ins.push_back(Src{&h->cvars[c], h->cost_off[c], true, -1.0 / h->eps});
    for (const auto& si : h->clsep[c]) {
      ins.push_back(src(h->dual[si.first][si.second], 1.0));
      if (!h->sgamma[si.first].empty()) ins.push_back(src(h->logm[si.first], 1.0));
    }
    plans.ops.push_back(make_op(h, h->logplan[c], {}, ins));
  }
  Stage proj, ref;
  for (int32_t s = 0; s < h->nsep; ++s) {
    const std::vector<int32_t>& cl = h->scl[s];
    std::vector<std::vector<int32_t>> sets;
    for (int32_t c : cl) sets.push_back(inter(h->svars[s], h->cvars[c]));
    std::vector<Tensor> P;
    for (size_t i = 0; i < cl.size(); ++i) {
      P.push_back(new_tensor(h, sets[i]));
      proj.ops.push_back(make_op(h, P[i], minus(h->cvars[cl[i]], sets[i]), {src(h->logplan[cl[i]], 1.0)}));
    }
    for (size_t i = 1; i < cl.size(); ++i) {
      Tensor r = new_tensor(h, sets[i]);
      ref.ops.push_back(make_op(h, r, minus(sets[0], sets[i]), {src(P[0], 1.0)}));
      h->res_sums.push_back(JtSum{reinterpret_cast<const double*>((intptr_t)P[i].off),
                                  reinterpret_cast<const double*>((intptr_t)r.off), nullptr, P[i].size, 2 * s, 0});
    }
    if (h->sgamma[s].empty()) {
      h->res_sums.push_back(
          JtSum{reinterpret_cast<const double*>((intptr_t)P[0].off), nullptr, nullptr, P[0].size, 2 * s + 1, 1});
    } else {
      Tensor pg = new_tensor(h, h->sgamma[s]);
      ref.ops.push_back(make_op(h, pg, minus(sets[0], h->sgamma[s]), {src(P[0], 1.0)}));
      h->res_sums.push_back(JtSum{reinterpret_cast<const double*>((intptr_t)pg.off),
                                  reinterpret_cast<const double*>((intptr_t)h->logm[s].off), nullptr, pg.size, 2 * s,
                                  0});
    }
  }
  for (int32_t c = 0; c < h->ncl; ++c)
    h->tc_sums.push_back(JtSum{reinterpret_cast<const double*>((intptr_t)h->logplan[c].off), nullptr,
                               reinterpret_cast<const float*>((intptr_t)h->cost_off[c]), h->logplan[c].size, 0, 2});
  h->res_stages.push_back(std::move(plans));
  h->res_stages.push_back(std::move(proj));
  h->res_stages.push_back(std::move(ref));
}

void resolve_sums(const tree_ot_jt_handle* h, std::vector<JtSum>& v) {
  for (JtSum& q : v) {
    q.a = h->d_arena + (intptr_t)q.a;
    if (q.b) q.b = h->d_arena + (intptr_t)q.b;
    if (q.kind == 2) q.c = h->d_cost + (intptr_t)q.c;
  }
}

// structure checks of def:jt_general and ass:inclusion; the two-colouring
int validate_jt(const tree_ot_jt_problem* p, tree_ot_jt_handle* h) {
  if (!p || p->num_vars < 1 || p->num_cliques < 1 || p->num_seps < 1 || !p->var_size || !p->clique_var_begin ||
      !p->clique_vars || !p->clique_cost || !p->sep_var_begin || !p->sep_vars || !p->sep_clique_begin ||
      !p->sep_cliques || !p->sep_gamma_begin)
    return jt_fail(TREE_OT_ERR_ARG, "junction tree: missing arrays or empty structure");
  if (!(p->eps > 0.0) || !std::isfinite(p->eps)) return jt_fail(TREE_OT_ERR_EPS, "eps must be positive and finite");
  h->nvars = p->num_vars;
  h->ncl = p->num_cliques;
  h->nsep = p->num_seps;
  h->eps = p->eps;
  h->vsize.assign(p->var_size, p->var_size + p->num_vars);
  for (int32_t v : h->vsize)
    if (v < 1) return jt_fail(TREE_OT_ERR_ARG, "support sizes must be >= 1");
  auto take = [&](const int32_t* begin, const int32_t* items, int32_t n, std::vector<std::vector<int32_t>>& out,
                  int32_t lim, const char* what) -> int {
    out.resize(n);
    for (int32_t i = 0; i < n; ++i) {
      if (begin[i + 1] < begin[i]) return jt_fail(TREE_OT_ERR_ARG, std::string(what) + ": offsets decrease");
      out[i].assign(items + begin[i], items + begin[i + 1]);
      for (int32_t x : out[i])
        if (x < 0 || x >= lim) return jt_fail(TREE_OT_ERR_ARG, std::string(what) + ": index out of range");
      std::vector<int32_t> srt = out[i];
      std::sort(srt.begin(), srt.end());
      if (std::adjacent_find(srt.begin(), srt.end()) != srt.end())
        return jt_fail(TREE_OT_ERR_ARG, std::string(what) + ": repeated index");
    }
    return TREE_OT_OK;
  };
  JT_TRY(take(p->clique_var_begin, p->clique_vars, h->ncl, h->cvars, h->nvars, "clique variables"));
  JT_TRY(take(p->sep_var_begin, p->sep_vars, h->nsep, h->svars, h->nvars, "separator variables"));
  JT_TRY(take(p->sep_clique_begin, p->sep_cliques, h->nsep, h->scl, h->ncl, "separator cliques"));
  JT_TRY(take(p->sep_gamma_begin, p->sep_gamma, h->nsep, h->sgamma, h->nvars, "constraint variables"));
  for (int32_t c = 0; c < h->ncl; ++c) {
    if (h->cvars[c].empty() || (int)h->cvars[c].size() > kJtMaxDims)
      return jt_fail(TREE_OT_ERR_ARG, "a clique needs 1 to 8 variables");
    if (!p->clique_cost[c]) return jt_fail(TREE_OT_ERR_ARG, "a clique's cost is NULL");
  }
  h->clsep.assign(h->ncl, {});
  for (int32_t s = 0; s < h->nsep; ++s) {
    if (h->scl[s].empty()) return jt_fail(TREE_OT_ERR_NOT_TREE, "a separator has no clique");
    for (size_t i = 0; i < h->scl[s].size(); ++i) h->clsep[h->scl[s][i]].push_back({s, (int32_t)i});
    std::vector<std::vector<int32_t>> sets;
    for (int32_t c : h->scl[s]) sets.push_back(inter(h->svars[s], h->cvars[c]));
    if (sets.size() > 1 && !(subset(sets[0], sets[1]) && subset(sets[1], sets[0])))
      return jt_fail(TREE_OT_ERR_NOT_TREE, "the first two intersections of a separator must be equal (ass:inclusion)");
    for (size_t i = 2; i < sets.size(); ++i)
      if (!subset(sets[i], sets[i - 1]))
        return jt_fail(TREE_OT_ERR_NOT_TREE, "a separator's intersections must be nested (ass:inclusion)");
    if (!subset(h->sgamma[s], sets.back()))
      return jt_fail(TREE_OT_ERR_NOT_TREE, "a constraint must lie in the separator's smallest intersection");
    if (!h->sgamma[s].empty() && (!p->sep_mu || !p->sep_mu[s]))
      return jt_fail(TREE_OT_ERR_ARG, "a constrained separator needs its marginal");
  }
  for (int32_t c = 0; c < h->ncl; ++c)
    if (h->clsep[c].size() != 2)
      return jt_fail(TREE_OT_ERR_NOT_TREE, "every clique must join exactly two separators (def:jt_general)");
  // two-colouring through the cliques, separator 0 first
  std::vector<std::vector<int32_t>> nb(h->nsep);
  for (int32_t c = 0; c < h->ncl; ++c) {
    const int32_t a = h->clsep[c][0].first, b = h->clsep[c][1].first;
    nb[a].push_back(b);
    nb[b].push_back(a);
  }
  h->colour.assign(h->nsep, -1);
  h->colour[0] = 0;
  std::deque<int32_t> dq{0};
  while (!dq.empty()) {
    const int32_t v = dq.front();
    dq.pop_front();
    for (int32_t w : nb[v]) {
      if (h->colour[w] < 0) {
        h->colour[w] = 1 - h->colour[v];
        dq.push_back(w);
      } else if (h->colour[w] == h->colour[v]) {
        return jt_fail(TREE_OT_ERR_NOT_TREE, "the separators do not two-colour through the cliques");
      }
    }
  }
  for (int32_t col : h->colour)
    if (col < 0) return jt_fail(TREE_OT_ERR_NOT_TREE, "the junction tree is not connected");
  return TREE_OT_OK;
}

}  // namespace

extern "C" {

int tree_ot_jt_create(const tree_ot_jt_problem* p, void* cuda_stream, tree_ot_jt_handle** out) {
  set_last_error("");
  if (!out) return jt_fail(TREE_OT_ERR_ARG, "out is NULL");
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  auto* h = new tree_ot_jt_handle();
  auto bail = [&](int rc) {
    delete h;
    return rc;
  };
  int rc = validate_jt(p, h);
  if (rc) return bail(rc);
  // costs (FP32, finite or +inf) and marginals (probability tensors)
  std::vector<float> cost;
  for (int32_t c = 0; c < h->ncl; ++c) {
    int64_t n = 1;
    for (int32_t v : h->cvars[c]) n *= h->vsize[v];
    h->cost_off.push_back((int64_t)cost.size());
    h->cost_size.push_back(n);
    for (int64_t i = 0; i < n; ++i) {
      const float x = p->clique_cost[c][i];
      if (std::isnan(x) || x == -INFINITY) return bail(jt_fail(TREE_OT_ERR_NONFINITE, "a cost is NaN or -inf"));
      cost.push_back(x);
    }
  }
  h->cost_len = (int64_t)cost.size();
  for (int32_t sp = 0; sp < h->nsep; ++sp) {
    h->dual.emplace_back();
    for (int32_t c : h->scl[sp]) h->dual[sp].push_back(new_tensor(h, inter(h->svars[sp], h->cvars[c])));
  }
  std::vector<std::pair<int64_t, std::vector<double>>> logm_init;
  h->logm.resize(h->nsep);
  for (int32_t sp = 0; sp < h->nsep; ++sp) {
    if (h->sgamma[sp].empty()) continue;
    h->logm[sp] = new_tensor(h, h->sgamma[sp]);
    std::vector<double> lm((size_t)h->logm[sp].size);
    double tot = 0.0;
    for (int64_t i = 0; i < h->logm[sp].size; ++i) {
      const double m = p->sep_mu[sp][i];
      if (!(m >= 0.0) || !std::isfinite(m)) return bail(jt_fail(TREE_OT_ERR_MARGINAL, "a marginal entry is negative"));
      tot += m;
      lm[(size_t)i] = m > 0.0 ? std::log(m) : -INFINITY;
    }
    if (std::fabs(tot - 1.0) > 1e-9) return bail(jt_fail(TREE_OT_ERR_MARGINAL, "a marginal does not sum to 1"));
    logm_init.push_back({h->logm[sp].off, std::move(lm)});
  }
  for (int c = 0; c < 2; ++c) plan_half_step(h, c, h->stages[c]);
  plan_residual(h);
  int64_t maxplan = 1;
  for (int32_t c = 0; c < h->ncl; ++c) maxplan = std::max(maxplan, h->cost_size[c]);
  h->tmp_len = maxplan;
  if ((rc = jt_alloc(h, &h->d_arena, h->arena_len)) || (rc = jt_alloc(h, &h->d_cost, h->cost_len)) ||
      (rc = jt_alloc(h, &h->d_slots, 2 * (int64_t)h->nsep + 1)) || (rc = jt_alloc(h, &h->d_constrained, h->nsep)) ||
      (rc = jt_alloc(h, &h->d_res, 2)) || (rc = jt_alloc(h, &h->d_tmp, h->tmp_len)))
    return bail(rc);
  if ((rc = jt_cuda(cudaMemsetAsync(h->d_arena, 0, sizeof(double) * (size_t)h->arena_len, s), "memset")) ||
      (rc = jt_cuda(cudaMemcpyAsync(h->d_cost, cost.data(), sizeof(float) * cost.size(), cudaMemcpyHostToDevice, s),
                    "upload costs")))
    return bail(rc);
  for (auto& lm : logm_init)
    if ((rc = jt_cuda(cudaMemcpyAsync(h->d_arena + lm.first, lm.second.data(), sizeof(double) * lm.second.size(),
                                      cudaMemcpyHostToDevice, s),
                      "upload marginals")))
      return bail(rc);
  std::vector<int32_t> cons(h->nsep);
  for (int32_t sp = 0; sp < h->nsep; ++sp) cons[sp] = h->sgamma[sp].empty() ? 0 : 1;
  if ((rc = jt_cuda(cudaMemcpyAsync(h->d_constrained, cons.data(), sizeof(int32_t) * cons.size(),
                                    cudaMemcpyHostToDevice, s),
                    "upload flags")))
    return bail(rc);
  for (int c = 0; c < 2; ++c)
    for (Stage& st : h->stages[c])
      if ((rc = upload_stage(h, st, s))) return bail(rc);
  for (Stage& st : h->res_stages)
    if ((rc = upload_stage(h, st, s))) return bail(rc);
  resolve_sums(h, h->res_sums);
  resolve_sums(h, h->tc_sums);
  if ((rc = upload_sums(h, h->res_sums, &h->d_res_sums, &h->d_res_start, &h->res_blocks, s)) ||
      (rc = upload_sums(h, h->tc_sums, &h->d_tc_sums, &h->d_tc_start, &h->tc_blocks, s)))
    return bail(rc);
  if ((rc = jt_cuda(cudaStreamSynchronize(s), "cudaStreamSynchronize(create)"))) return bail(rc);
  *out = h;
  return TREE_OT_OK;
}

int tree_ot_jt_destroy(tree_ot_jt_handle* h) {
  delete h;
  return TREE_OT_OK;
}

int tree_ot_jt_reset(tree_ot_jt_handle* h, void* cuda_stream) {
  set_last_error("");
  if (!h) return jt_fail(TREE_OT_ERR_ARG, "handle is NULL");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  for (auto& ds : h->dual)
    for (const Tensor& t : ds)
      JT_TRY(jt_cuda(cudaMemsetAsync(h->d_arena + t.off, 0, sizeof(double) * (size_t)t.size, s), "memset"));
  h->hs = 0;
  return TREE_OT_OK;
}

namespace {
int run_half_step(tree_ot_jt_handle* h, cudaStream_t s) {
  for (const Stage& st : h->stages[h->hs % 2]) JT_TRY(run_stage(st, s));
  ++h->hs;
  return TREE_OT_OK;
}

// a half-step is a few dozen small launches: pairs of half-steps replay one
// captured CUDA graph (captured on first use, per stream)
int pair_graph(tree_ot_jt_handle* h, cudaStream_t s) {
  if (h->pair && h->pair_stream == s) return TREE_OT_OK;
  if (h->pair) {
    cudaGraphExecDestroy(h->pair);
    h->pair = nullptr;
  }
  cudaStream_t cap = nullptr;
  JT_TRY(jt_cuda(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "cudaStreamCreate"));
  cudaGraph_t g = nullptr;
  int rc = jt_cuda(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
  if (!rc) {
    const int64_t hs0 = h->hs;
    h->hs = 0;
    for (int c = 0; c < 2 && !rc; ++c) rc = run_half_step(h, cap);
    h->hs = hs0;
    const int rc2 = jt_cuda(cudaStreamEndCapture(cap, &g), "cudaStreamEndCapture");
    if (!rc) rc = rc2;
  }
  if (!rc) rc = jt_cuda(cudaGraphInstantiate(&h->pair, g, 0), "cudaGraphInstantiate");
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cap);
  if (!rc) h->pair_stream = s;
  return rc;
}
}  // namespace

int tree_ot_jt_half_steps(tree_ot_jt_handle* h, void* cuda_stream, int64_t T) {
  set_last_error("");
  if (!h || T < 0) return jt_fail(TREE_OT_ERR_ARG, "handle is NULL or T < 0");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (T > 0 && h->hs % 2) {  // pairs start with colour 0
    JT_TRY(run_half_step(h, s));
    --T;
  }
  if (T >= 2) {
    JT_TRY(pair_graph(h, s));
    for (; T >= 2; T -= 2) {
      JT_TRY(jt_cuda(cudaGraphLaunch(h->pair, s), "cudaGraphLaunch"));
      h->hs += 2;
    }
  }
  if (T > 0) JT_TRY(run_half_step(h, s));
  return TREE_OT_OK;
}

int tree_ot_jt_residual(tree_ot_jt_handle* h, void* cuda_stream, double* sum, double* max) {
  set_last_error("");
  if (!h || !sum || !max) return jt_fail(TREE_OT_ERR_ARG, "NULL argument");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  for (const Stage& st : h->res_stages) JT_TRY(run_stage(st, s));
  JT_TRY(jt_cuda(cudaMemsetAsync(h->d_slots, 0, sizeof(double) * (2 * (size_t)h->nsep + 1), s), "memset"));
  if (h->res_blocks > 0)
    jt_sum_kernel<<<(unsigned)h->res_blocks, 256, 0, s>>>(h->d_res_sums, h->d_res_start, (int32_t)h->res_sums.size(),
                                                           h->d_slots);
  jt_residual_finish_kernel<<<1, 32, 0, s>>>(h->d_slots, h->d_constrained, h->nsep, h->d_res);
  JT_TRY(jt_cuda(cudaGetLastError(), "residual launch"));
  double r[2];
  JT_TRY(jt_cuda(cudaMemcpyAsync(r, h->d_res, sizeof(r), cudaMemcpyDeviceToHost, s), "read residual"));
  JT_TRY(jt_cuda(cudaStreamSynchronize(s), "cudaStreamSynchronize(residual)"));
  *sum = r[0];
  *max = r[1];
  return TREE_OT_OK;
}

int tree_ot_jt_solve(tree_ot_jt_handle* h, void* cuda_stream, double tol, int32_t tol_kind, int64_t max_half_steps,
                     int32_t check_every, int64_t* half_steps, double* residual_out) {
  set_last_error("");
  if (!h || !(tol > 0.0) || (tol_kind != TREE_OT_TOL_SUM && tol_kind != TREE_OT_TOL_MAX) || max_half_steps < 0 ||
      check_every < 1)
    return jt_fail(TREE_OT_ERR_ARG, "bad handle, tol, tol_kind, max_half_steps or check_every");
  int64_t done = 0;
  double rs = 0.0, rm = 0.0;
  JT_TRY(tree_ot_jt_residual(h, cuda_stream, &rs, &rm));
  while ((tol_kind == TREE_OT_TOL_SUM ? rs : rm) >= tol && done < max_half_steps) {
    const int64_t k = std::min<int64_t>(check_every, max_half_steps - done);
    JT_TRY(tree_ot_jt_half_steps(h, cuda_stream, k));
    done += k;
    JT_TRY(tree_ot_jt_residual(h, cuda_stream, &rs, &rm));
  }
  if (half_steps) *half_steps = done;
  if (residual_out) *residual_out = tol_kind == TREE_OT_TOL_SUM ? rs : rm;
  return (tol_kind == TREE_OT_TOL_SUM ? rs : rm) < tol ? TREE_OT_OK : TREE_OT_NOT_CONVERGED;
}

int tree_ot_jt_plan(tree_ot_jt_handle* h, void* cuda_stream, int32_t clique, double* plan_out) {
  set_last_error("");
  if (!h || !plan_out || clique < 0 || clique >= h->ncl) return jt_fail(TREE_OT_ERR_ARG, "bad handle or clique");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  JT_TRY(run_stage(h->res_stages[0], s));  // every clique's log plan
  const Tensor& t = h->logplan[clique];
  const int blocks = (int)std::min<int64_t>((t.size + 255) / 256, 4096);
  jt_exp_kernel<<<blocks, 256, 0, s>>>(h->d_arena + t.off, h->d_tmp, t.size);
  JT_TRY(jt_cuda(cudaGetLastError(), "plan launch"));
  JT_TRY(jt_cuda(cudaMemcpyAsync(plan_out, h->d_tmp, sizeof(double) * (size_t)t.size, cudaMemcpyDeviceToHost, s),
                 "read plan"));
  return jt_cuda(cudaStreamSynchronize(s), "cudaStreamSynchronize(plan)");
}

int tree_ot_jt_transport_cost(tree_ot_jt_handle* h, void* cuda_stream, double* tc) {
  set_last_error("");
  if (!h || !tc) return jt_fail(TREE_OT_ERR_ARG, "NULL argument");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  JT_TRY(run_stage(h->res_stages[0], s));
  JT_TRY(jt_cuda(cudaMemsetAsync(h->d_slots, 0, sizeof(double), s), "memset"));
  if (h->tc_blocks > 0)
    jt_sum_kernel<<<(unsigned)h->tc_blocks, 256, 0, s>>>(h->d_tc_sums, h->d_tc_start, (int32_t)h->tc_sums.size(),
                                                          h->d_slots);
  JT_TRY(jt_cuda(cudaGetLastError(), "transport cost launch"));
  JT_TRY(jt_cuda(cudaMemcpyAsync(tc, h->d_slots, sizeof(double), cudaMemcpyDeviceToHost, s), "read cost"));
  return jt_cuda(cudaStreamSynchronize(s), "cudaStreamSynchronize(cost)");
}

int tree_ot_jt_get_dual(tree_ot_jt_handle* h, void* cuda_stream, int32_t sep, int32_t pos, double* log_u) {
  set_last_error("");
  if (!h || !log_u || sep < 0 || sep >= h->nsep || pos < 0 || pos >= (int32_t)h->scl[sep].size())
    return jt_fail(TREE_OT_ERR_ARG, "bad handle, separator or position");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const Tensor& t = h->dual[sep][pos];
  JT_TRY(jt_cuda(cudaMemcpyAsync(log_u, h->d_arena + t.off, sizeof(double) * (size_t)t.size, cudaMemcpyDeviceToHost, s),
                 "read dual"));
  return jt_cuda(cudaStreamSynchronize(s), "cudaStreamSynchronize(dual)");
}

int tree_ot_jt_colour(tree_ot_jt_handle* h, int32_t* colour_out) {
  set_last_error("");
  if (!h || !colour_out) return jt_fail(TREE_OT_ERR_ARG, "NULL argument");
  for (int32_t sp = 0; sp < h->nsep; ++sp) colour_out[sp] = h->colour[sp];
  return TREE_OT_OK;
}

}  // extern "C"
