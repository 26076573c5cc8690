// Node update of one half-step (the block-update theorem thm:tree_dual_var, in log form),
// fused with the stopping terms of the Bipartite Iterative Scaling algorithm.
//
// One CTA handles a chunk of up to kNodeChunk support points of one node j of
// the active colour.  For each owned directed edge (j,k) it merges the apply
// kernel's partial log-sum-exps into the message m_(j,k)(x) (subtracting the
// neighbour's normaliser Z_k), then
//   fixed j:  f_(j,k) = -eps m_(j,k)                               (u = 1./(K u'))
//   free  j:  s(x) = mean_k m_(j,k)(x);  f'_(j,k) = eps (s - m_(j,k));
//             Z_j = LSE_x s(x);  rho_j = -|N(j)| Z_j              (f = f' - eps Z_j)
// Before overwriting, it evaluates the stopping terms of the iterate the
// previous half-step produced (only this colour's terms are non-zero there):
//   fixed j:  sum_x |q(x) - mu_j(x)|,        q = mu_j exp(f/eps + m)  (= B 1)
//   free  j:  sum_x |q_k(x) - qbar(x)|,      q_k = exp(f_(j,k)/eps + m_(j,k))
// Chunks of a node, nodes of a problem and CTAs of the launch meet through
// arrival counters (the last arrival finishes the reduction; nobody waits):
// the last chunk of a node merges Z_j and the node's stopping terms, the last
// node of a problem records the stopping quantity and (when asked) retires the
// problem, the last CTA of the launch advances the half-step counter.
#include <cmath>

#include "internal.h"
#include "ptx.cuh"

namespace treeot {
namespace {

// merge the apply's (frame, sum) pieces of one output; empty pieces (sum 0) carry no frame
__device__ __forceinline__ double merge32(const float2* part, int nsplit, int64_t stride) {
  float Rm = -INFINITY;
  for (int p = 0; p < nsplit; ++p) {
    const float2 v = part[p * stride];
    if (v.y > 0.f) Rm = fmaxf(Rm, v.x);
  }
  if (Rm == -INFINITY) return -INFINITY;
  float S = 0.f;
  for (int p = 0; p < nsplit; ++p) {
    const float2 v = part[p * stride];
    if (v.y > 0.f) S += (v.x == Rm) ? v.y : v.y * ex2(v.x - Rm);
  }
  if (!isfinite(S) || !(S > 0.f)) return (S > 0.f) ? INFINITY : -INFINITY;
  int e;
  const float mant = frexpf(S, &e);  // S = mant * 2^e, mant in [0.5, 1)
  return ((double)Rm + (double)e) * kLn2 + (double)logf(mant);
}

__device__ __forceinline__ double merge64(const double2* part, int nsplit, int64_t stride) {
  double M = -INFINITY;
  for (int p = 0; p < nsplit; ++p) M = fmax(M, part[p * stride].x);
  if (!(M > -INFINITY)) return -INFINITY;
  double S = 0.0;
  for (int p = 0; p < nsplit; ++p) {
    const double2 v = part[p * stride];
    S += v.y * exp(v.x - M);
  }
  return M + log(S);
}

// exp of a double argument, evaluated at the precision of the path
template <bool F64>
__device__ __forceinline__ double expx(double a) {
  if (F64) return exp(a);
  return (double)ex2((float)(a * kLog2e));
}

// two-float split of an apply operand: hi on the 2^-10 grid, lo the (small) rest
__device__ __forceinline__ void split2(double v, float& hi, float& lo) {
  if (!isfinite(v)) {
    hi = (float)v;
    lo = 0.f;
    return;
  }
  hi = (float)(rint(v * kGrid) / kGrid);
  lo = (float)(v - (double)hi);
}

// block-wide sum / max of a double (kNodeThreads threads); result valid in all threads
__device__ double block_sum(double v, double* red) {
  v = warp_sum_d(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double r = 0.0;
#pragma unroll
  for (int i = 0; i < kNodeThreads / 32; ++i) r += red[i];
  return r;
}

__device__ double block_max(double v, double* red) {
  v = warp_max_d(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double r = -INFINITY;
#pragma unroll
  for (int i = 0; i < kNodeThreads / 32; ++i) r = fmax(r, red[i]);
  return r;
}

// frame of a message for the next apply: log2 of it on the 2^-10 grid (0 when not finite)
__device__ __forceinline__ float frame_grid(double m) {
  return isfinite(m) ? (float)(rint(m * (kLog2e * kGrid)) * (1.0 / kGrid)) : 0.f;
}

template <bool F64>
__device__ __forceinline__ double merged(const NodeArgs& A, const DEdgeD& d, int n_owner, int x) {
  if (F64) return merge64(A.part64 + d.part_off + x, d.nsplit, n_owner);
  return merge32(A.part32 + d.part_off + x, d.nsplit, n_owner);
}

template <bool F64>
__device__ void fixed_chunk(const NodeArgs& A, const NodeD& nd, const NodeChunk& c, const ProbD& P, double* red) {
  const DEdgeD d = A.dedges[A.node_dedges[nd.dedge_begin]];
  const double Zn = A.Z[d.nbr];
  double r = 0.0;
  bool bad = false;
  // low-precision phase: flag the edge when the operand leaves its absorbed base
  const bool track = A.absorbed && A.lowp[nd.prob] == 1;
  bool drift = false;
  for (int xi = threadIdx.x; xi < c.cnt; xi += kNodeThreads) {
    const int x = c.x0 + xi;
    const double mr = merged<F64>(A, d, nd.n, x);
    A.m[d.off + x] = mr;
    A.fr[d.off + x] = frame_grid(mr);
    const double mi = mr - Zn;
    const double fo = A.f[d.off + x];
    const double lg = A.logg[nd.node_off + x];
    const double mu = A.mu[nd.node_off + x];
    const double q = (mu > 0.0) ? mu * expx<F64>(fo * P.inv_eps + mi) : 0.0;
    r += fabs(q - mu);
    const double fn = -P.eps * mi;
    A.f[d.off + x] = fn;
    float hi, lo;
    if (lg == -INFINITY) {
      hi = -INFINITY;
      lo = 0.f;
    } else {
      split2((lg - mi) * kLog2e, hi, lo);
      if (!isfinite(mi)) bad = true;
    }
    A.hh[d.off + x] = hi;
    A.hl[d.off + x] = lo;
    if (track && hi > -INFINITY && fabsf((hi - A.bh[d.off + x]) + (lo - A.bl[d.off + x])) > A.tau) drift = true;
  }
  if (bad) atomicOr(A.err, 1);
  if (__syncthreads_or(drift) && threadIdx.x == 0) atomicOr(&A.drift[d.edge], 1);
  r = block_sum(r, red);
  if (threadIdx.x == 0) atomicAdd(&A.resid_acc[A.node_dedges[nd.dedge_begin]], r);
}

template <bool F64>
__device__ void free_chunk(const NodeArgs& A, const NodeD& nd, const NodeChunk& c, const ProbD& P, double* red,
                           double* s_s, double* s_q, int node_id) {
  const int deg = nd.deg;
  const double Zold = A.Z[node_id];
  const bool track = A.absorbed && A.lowp[nd.prob] == 1;
  const double inv_deg = 1.0 / (double)deg;
  bool bad = false;
  double smax = -INFINITY;
  for (int xi = threadIdx.x; xi < c.cnt; xi += kNodeThreads) {
    const int x = c.x0 + xi;
    double ssum = 0.0, qsum = 0.0;
    for (int i = 0; i < deg; ++i) {
      const DEdgeD d = A.dedges[A.node_dedges[nd.dedge_begin + i]];
      const double mr = merged<F64>(A, d, nd.n, x);
      A.m[d.off + x] = mr;
      A.fr[d.off + x] = frame_grid(mr);
      const double mi = mr - A.Z[d.nbr];
      const double fo = A.f[d.off + x];
      qsum += expx<F64>((fo * P.inv_eps - Zold) + mi);
      ssum += mi;
    }
    const double s = ssum * inv_deg;
    if (!isfinite(s)) bad = true;
    s_s[xi] = s;
    s_q[xi] = qsum * inv_deg;
    smax = fmax(smax, s);
  }
  smax = block_max(smax, red);
  double se = 0.0;
  for (int xi = threadIdx.x; xi < c.cnt; xi += kNodeThreads) se += expx<F64>(s_s[xi] - smax);
  se = block_sum(se, red);
  if (threadIdx.x == 0) A.zpart[nd.chunk_base + c.chunk] = make_double2(smax, se);
  for (int i = 0; i < deg; ++i) {
    const int di = A.node_dedges[nd.dedge_begin + i];
    const DEdgeD d = A.dedges[di];
    const double Zk = A.Z[d.nbr];
    double r = 0.0;
    bool drift = false;
    for (int xi = threadIdx.x; xi < c.cnt; xi += kNodeThreads) {
      const int x = c.x0 + xi;
      const double mi = A.m[d.off + x] - Zk;
      const double fo = A.f[d.off + x];
      const double q = expx<F64>((fo * P.inv_eps - Zold) + mi);
      r += fabs(q - s_q[xi]);
      const double g = s_s[xi] - mi;  // f'/eps
      A.f[d.off + x] = P.eps * g;
      float hi, lo;
      split2(g * kLog2e, hi, lo);
      A.hh[d.off + x] = hi;
      A.hl[d.off + x] = lo;
      if (track && fabsf((hi - A.bh[d.off + x]) + (lo - A.bl[d.off + x])) > A.tau) drift = true;
    }
    if (__syncthreads_or(drift) && threadIdx.x == 0) atomicOr(&A.drift[d.edge], 1);
    r = block_sum(r, red);
    if (threadIdx.x == 0) atomicAdd(&A.resid_acc[di], r);
  }
  if (bad) atomicOr(A.err, 1);
}

template <bool F64>
__global__ void __launch_bounds__(kNodeThreads) node_update_kernel(NodeArgs A) {
  __shared__ double red[kNodeThreads / 32];
  __shared__ double s_s[kNodeChunk];
  __shared__ double s_q[kNodeChunk];
  const NodeChunk c = A.chunks[blockIdx.x];
  const NodeD nd = A.nodes[c.node];
  const int p = nd.prob;
  const ProbD P = A.probs[p];
  const int64_t t_now = *((volatile const int64_t*)A.hs);
  const int slot = (int)(t_now % kResidRing);
  const bool skip = A.done[p] != 0;
  if (!skip) {
    if (nd.fixed)
      fixed_chunk<F64>(A, nd, c, P, red);
    else
      free_chunk<F64>(A, nd, c, P, red, s_s, s_q, c.node);
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  __threadfence();
  if (!skip && atomicAdd(&A.node_arrive[c.node], 1) == nd.nchunks - 1) {
    // last chunk of this node: finish Z_j and the node's stopping terms
    __threadfence();
    if (!nd.fixed) {
      double M = -INFINITY;
      for (int k = 0; k < nd.nchunks; ++k) M = fmax(M, A.zpart[nd.chunk_base + k].x);
      double S = 0.0;
      for (int k = 0; k < nd.nchunks; ++k) {
        const double2 z = A.zpart[nd.chunk_base + k];
        S += z.y * exp(z.x - M);
      }
      const double Zn = M + log(S);
      A.Z[c.node] = Zn;
      A.rho[c.node] = -(double)nd.deg * Zn;
    }
    double nsum = 0.0, nmax = 0.0;
    for (int i = 0; i < nd.deg; ++i) {
      const int di = A.node_dedges[nd.dedge_begin + i];
      // read the chunks' accumulated term and clear it for the next launch
      const double r = __longlong_as_double(
          (long long)atomicExch((unsigned long long*)&A.resid_acc[di], 0ull));
      A.resid_dedge[di] = r;
      nsum += r;
      nmax = fmax(nmax, r);
    }
    A.node_arrive[c.node] = 0;
    atomicAdd(&A.res_sum[slot * A.nprob + p], nsum);
    atomicMax(&A.res_max[slot * A.nprob + p], (unsigned long long)__double_as_longlong(nmax));
    __threadfence();
    if (atomicAdd(&A.node_count[p], 1) == P.nodes_in_colour[A.colour] - 1) {
      // last node of this problem in this launch: the stopping quantity of iterate t_now is complete
      __threadfence();
      const double rs = *((volatile double*)&A.res_sum[slot * A.nprob + p]);
      const double rm = __longlong_as_double(
          (long long)*((volatile unsigned long long*)&A.res_max[slot * A.nprob + p]));
      const double crit = A.tol_kind == 1 ? rm : rs;
      const int lp = A.absorbed ? A.lowp[p] : 0;
      if (lp == 2 && t_now + 1 >= A.lowp_start) {
        // enter the low-precision phase: absorb every edge of the problem next
        A.lowp[p] = 1;
        A.lowp_span[2 * p] = t_now + 1;
        for (int k = 0; k < P.edge_count; ++k) A.drift[P.edge_begin + k] = 1;
      } else if (lp == 1) {
        // the absorbed kernel's accuracy is enough until the stopping quantity
        // reaches refine_tol; from then on the FP32 kernel refines
        if (crit < A.refine_tol) {
          A.lowp[p] = 0;
          A.lowp_span[2 * p + 1] = t_now + 1;
        }
      } else if (A.retire && (crit < A.ptol[p] || t_now + 1 >= A.deadline[p])) {
        A.done[p] = 1;
        A.done_at[p] = t_now + 1;
      }
      A.node_count[p] = 0;
      const int nslot = (int)((t_now + 1) % kResidRing);
      A.res_sum[nslot * A.nprob + p] = 0.0;
      A.res_max[nslot * A.nprob + p] = 0ull;
    }
  }
  __threadfence();
  if (atomicAdd(A.launch_count, 1) == (int)gridDim.x - 1) {
    *A.launch_count = 0;
    __threadfence();
    atomicAdd((unsigned long long*)A.hs, 1ull);
  }
}

}  // namespace

cudaError_t launch_node_update(const NodeArgs& a, bool fp64, cudaStream_t s) {
  if (a.nchunks <= 0) return cudaSuccess;
  if (fp64)
    node_update_kernel<true><<<a.nchunks, kNodeThreads, 0, s>>>(a);
  else
    node_update_kernel<false><<<a.nchunks, kNodeThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace treeot
