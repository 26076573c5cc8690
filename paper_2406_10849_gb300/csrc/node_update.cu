// Node update of one half-step (the block-update theorem thm:tree_dual_var, in log form),
// fused with the stopping terms of the Bipartite Iterative Scaling algorithm.
//
// One CTA handles a chunk of the support points of one node j of the active
// colour, sized so that it holds at most kNodePairs (owned directed edge,
// point) pairs; every pair's intermediate values stay in shared memory.  For
// each owned directed edge (j,k) it merges the apply kernel's partial
// log-sum-exps into the message m_(j,k)(x) (subtracting the neighbour's
// normaliser Z_k), then
//   fixed j:  f_(j,k) = -eps m_(j,k)                               (u = 1./(K u'))
//   free  j:  s(x) = mean_k m_(j,k)(x);  f'_(j,k) = eps (s - m_(j,k));
//             Z_j = LSE_x s(x);  rho_j = -|N(j)| Z_j              (f = f' - eps Z_j)
// A free node takes three passes: over the pairs (merge, frames, the previous
// iterate's q_k), over the points (s, mean q, the chunk's part of Z_j) and over
// the pairs again (potentials, the next apply's operand, stopping terms); a
// fixed leaf takes one.  Pairs are independent, so a CTA keeps many loads in
// flight instead of walking each point's edges in turn.
// Before overwriting, it evaluates the stopping terms of the iterate the
// previous half-step produced (only this colour's terms are non-zero there):
//   fixed j:  sum_x |q(x) - mu_j(x)|,        q = mu_j exp(f/eps + m)  (= B 1)
//   free  j:  sum_x |q_k(x) - qbar(x)|,      q_k = exp(f_(j,k)/eps + m_(j,k))
// Chunks of a node, nodes of a problem and CTAs of the launch meet through
// arrival counters (the last arrival finishes the reduction; nobody waits):
// the last chunk of a node merges Z_j and the node's stopping terms, the last
// node of a problem records the stopping quantity and (when asked) retires the
// problem, the last CTA of the launch advances the half-step counter.
#include <algorithm>
#include <cmath>

#include "internal.h"
#include "node_chunk.cuh"
#include "ptx.cuh"

namespace treeot {
namespace {

// the last CTA of a launch that counts (count_launch) advances the half-step counter
__device__ __forceinline__ void node_launch_done(const NodeArgs& A) {
  if (threadIdx.x != 0 || !A.count_launch) return;
  __threadfence();
  if (atomicAdd(A.launch_count, 1) == (int)gridDim.x - 1) {
    *A.launch_count = 0;
    __threadfence();
    atomicAdd((unsigned long long*)A.hs, 1ull);
  }
}

template <bool F64>
__global__ void __launch_bounds__(kNodeThreads) node_update_kernel(NodeArgs A) {
  extern __shared__ __align__(16) unsigned char node_sm[];
  __shared__ double red[kNodeThreads / 32];
  const NodeChunk c = A.chunks[blockIdx.x];
  const int64_t t_now = *((volatile const int64_t*)A.hs);
  node_chunk_item<F64, false>(A, c, t_now, node_sm, red);
  node_launch_done(A);
}

// FP32 handles with shared-kernel groups: the same, plus the point-major form
// of free nodes in the phase; three CTAs per SM (it would take ~100 registers;
// capped at 80 it spills a little and still runs faster than at two)
__global__ void __launch_bounds__(kNodeThreads, 3) node_update_sk_kernel(NodeArgs A) {
  extern __shared__ __align__(16) unsigned char node_sm[];
  __shared__ double red[kNodeThreads / 32];
  const NodeChunk c = A.chunks[blockIdx.x];
  const int64_t t_now = *((volatile const int64_t*)A.hs);
  node_chunk_item<false, false, true>(A, c, t_now, node_sm, red);
  node_launch_done(A);
}

// chunks of fixed leaves only: without the free-node path the FP32 form fits in
// 64 registers, so four CTAs share an SM instead of three
template <bool F64>
__global__ void __launch_bounds__(kNodeThreads, 4) node_update_fixed_kernel(NodeArgs A) {
  extern __shared__ __align__(16) unsigned char node_sm[];
  __shared__ double red[kNodeThreads / 32];
  if constexpr (!F64) {
    if (A.fixed && A.defer) {  // launch-uniform: host-resolved chunk records
      // a grid of resident CTAs walks the records; each CTA copies the next
      // record into shared memory while it works on the current one
      constexpr int kWords = sizeof(FixedChunkD) / 4;
      static_assert(sizeof(FixedChunkD) % 4 == 0 && kWords <= kNodeThreads, "record copied as words");
      __shared__ __align__(8) FixedChunkD s_rec[2];
      const int tid = threadIdx.x;
      if (tid < kWords && (int)blockIdx.x < A.nchunks)
        reinterpret_cast<int*>(&s_rec[0])[tid] = reinterpret_cast<const int*>(&A.fixed[blockIdx.x])[tid];
      __syncthreads();
      int buf = 0;
      for (int c = blockIdx.x; c < A.nchunks; c += gridDim.x, buf ^= 1) {  // block-uniform
        const int cn = c + (int)gridDim.x;
        int nxt = 0;
        if (tid < kWords && cn < A.nchunks) nxt = reinterpret_cast<const int*>(&A.fixed[cn])[tid];
        fixed_chunk_fast(A, s_rec[buf], red);
        if (tid < kWords) reinterpret_cast<int*>(&s_rec[buf ^ 1])[tid] = nxt;
        __syncthreads();  // the next record is in place; this chunk's shared values are free
      }
      return;
    }
  }
  const NodeChunk c = A.chunks[blockIdx.x];
  const int64_t t_now = *((volatile const int64_t*)A.hs);
  node_chunk_item<F64, true>(A, c, t_now, node_sm, red);
  node_launch_done(A);
}

// Deferred bookkeeping of one colour's node update, one warp per problem: each
// owned directed edge's stopping term (summed into resid_acc by the chunks),
// Z_j of the free nodes from their chunks' pieces, the problem's stopping
// quantity of iterate t_now, phase control and retirement; the last CTA
// advances the half-step counter.  The same arithmetic as the last-arrival
// path of node_chunk_item, run after the chunks' launch instead of on their
// way out: a chunk then leaves with no fence and no atomic it waits for.
constexpr int kFinishWarps = 8;
__global__ void __launch_bounds__(32 * kFinishWarps) node_finish_kernel(NodeArgs A, FinishList L) {
  const int lane = threadIdx.x & 31;
  const int p = blockIdx.x * kFinishWarps + (threadIdx.x >> 5);
  const int64_t t_now = *((volatile const int64_t*)A.hs);
  if (p < A.nprob && A.done[p] == 0) {
    const ProbD P = A.probs[p];
    if (P.nodes_in_colour[A.colour] > 0) {
      double nsum = 0.0, nmax = 0.0;
      for (int i = L.dbeg[p] + lane; i < L.dbeg[p + 1]; i += 32) {
        const int di = L.dedges[i];
        const double r = A.resid_acc[di];
        A.resid_acc[di] = 0.0;  // for the next launch
        A.resid_dedge[di] = r;
        nsum += r;
        nmax = fmax(nmax, r);
      }
      for (int i = L.nbeg[p]; i < L.nbeg[p + 1]; ++i) {  // warp-uniform
        const int node = L.nodes[i];
        finish_free_node_warp(A, node, A.nodes[node], lane);
      }
      nsum = warp_sum_d(nsum);
      nmax = warp_max_d(nmax);
      if (lane == 0) {
        const int slot = (int)(t_now % kResidRing);
        A.res_sum[slot * A.nprob + p] = nsum;
        A.res_max[slot * A.nprob + p] = (unsigned long long)__double_as_longlong(nmax);
        problem_after_update(A, p, P, t_now, nsum, nmax);
      }
    }
  }
  __syncthreads();
  node_launch_done(A);
}

// stored potentials of an FP32 handle from the operand the node update keeps:
// f' = eps ln2 (hh + hl) on a free owner, eps ln2 ((hh + hl) - log2 mu) on a
// fixed one (points with mu = 0 keep the f the update wrote).  One CTA per
// directed edge at a time; the two-floats are summed exactly in FP64.
__global__ void __launch_bounds__(256) materialise_f_kernel(const DEdgeD* dedges, int32_t ndedges, const NodeD* nodes,
                                                            const ProbD* probs, const float4* lgf, const float* hh,
                                                            const float* hl, double* f) {
  for (int di = blockIdx.x; di < ndedges; di += gridDim.x) {
    const DEdgeD d = dedges[di];
    const NodeD nd = nodes[d.owner];
    const double eps_ln2 = probs[d.prob].eps * kLn2;
    for (int x = threadIdx.x; x < nd.n; x += blockDim.x) {
      const double h = (double)hh[d.off + x] + (double)hl[d.off + x];
      if (nd.fixed) {
        const float4 lg = lgf[nd.node_off + x];
        if (lg.x == -INFINITY) continue;
        f[d.off + x] = eps_ln2 * (h - ((double)lg.x + (double)lg.y));
      } else {
        f[d.off + x] = eps_ln2 * h;
      }
    }
  }
}

__global__ void count_live_kernel(const int32_t* done, const int32_t* lowp, int32_t nprob, int32_t* out) {
  int n = 0;
  for (int p = threadIdx.x; p < nprob; p += blockDim.x) n += (done[p] == 0 && (!lowp || lowp[p] != 1)) ? 1 : 0;
  n = __reduce_add_sync(0xffffffffu, n);
  __shared__ int part[8];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = n;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    *out = t;
  }
}

}  // namespace

cudaError_t launch_count_live(const int32_t* done, const int32_t* lowp, int32_t nprob, int32_t* out, cudaStream_t s) {
  count_live_kernel<<<1, 256, 0, s>>>(done, lowp, nprob, out);
  return cudaGetLastError();
}

cudaError_t launch_node_update(const NodeArgs& a, bool fp64, bool fixed_only, cudaStream_t s) {
  if (a.nchunks <= 0) return cudaSuccess;
  const void* fn = fp64 ? (fixed_only ? reinterpret_cast<const void*>(node_update_fixed_kernel<true>)
                                      : reinterpret_cast<const void*>(node_update_kernel<true>))
                        : (fixed_only ? reinterpret_cast<const void*>(node_update_fixed_kernel<false>)
                           : a.sk_ref ? reinterpret_cast<const void*>(node_update_sk_kernel)
                                      : reinterpret_cast<const void*>(node_update_kernel<false>));
  // more than the default 48 KB of dynamic shared memory only for nodes of very
  // high degree; the attribute is per device and cheap to set again
  if (a.smem > 48u * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)a.smem);
    if (e != cudaSuccess) return e;
  }
  void* args[] = {const_cast<NodeArgs*>(&a)};
  if (!fp64 && fixed_only && a.fixed && a.defer) {
    // host-resolved records of fixed leaves: four resident CTAs per SM walk them
    // (no dynamic shared memory on that path)
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
    const int grid = std::min(a.nchunks, 4 * sms);
    return cudaLaunchKernel(fn, dim3(grid), dim3(kNodeThreads), args, 0, s);
  }
  return cudaLaunchKernel(fn, dim3(a.nchunks), dim3(kNodeThreads), args, a.smem, s);
}

cudaError_t launch_node_finish(const NodeArgs& a, const FinishList& l, cudaStream_t s) {
  if (a.nprob <= 0) return cudaSuccess;
  const int grid = (a.nprob + kFinishWarps - 1) / kFinishWarps;
  node_finish_kernel<<<grid, 32 * kFinishWarps, 0, s>>>(a, l);
  return cudaGetLastError();
}

cudaError_t launch_materialise_f(const DEdgeD* dedges, int32_t ndedges, const NodeD* nodes, const ProbD* probs,
                                 const float4* lgf, const float* hh, const float* hl, double* f, cudaStream_t s) {
  if (ndedges <= 0) return cudaSuccess;
  materialise_f_kernel<<<std::min(ndedges, 4096), 256, 0, s>>>(dedges, ndedges, nodes, probs, lgf, hh, hl, f);
  return cudaGetLastError();
}

}  // namespace treeot
