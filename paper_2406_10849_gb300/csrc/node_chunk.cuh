// Device functions of the node update (block updates of theorem thm:tree_dual_var
// in log form, fused with the stopping terms), shared by the per-half-step
// node-update kernel and the persistent forest kernel.  The algorithm is
// described at the top of node_update.cu.
#pragma once
#include <algorithm>
#include <cmath>

#include "grid.cuh"
#include "internal.h"
#include "ptx.cuh"

namespace treeot {
namespace {


// Two paths.  FP64 handles merge FP64 partials and work in double throughout
// (chunk_update64).  FP32 handles (chunk_update32) work in log2 units on
// two-float values with no FP64 arithmetic per pair or per block reduction
// (the stored potential is formed from the operand when it is read, by
// materialise_f_kernel): GB300 executes FP64 arithmetic and float <-> double
// conversions at a small fraction of its FP32 rate.


// frame of a message for the next apply: log2 of it on the 2^-10 grid (0 when not finite)
__device__ __forceinline__ float frame64(double m) {
  return isfinite(m) ? (float)(rint(m * (kLog2e * kGrid)) * (1.0 / kGrid)) : 0.f;
}

// two-float split of an apply operand v (log2 units): hi on the 2^-10 grid, lo
// the (small) rest.  hi comes from v rounded to FP32: any grid point within
// 2^-10 of v will do.
__device__ __forceinline__ void split2(double v, float& hi, float& lo) {
  if (!isfinite(v)) {
    hi = (float)v;
    lo = 0.f;
    return;
  }
  hi = quant((float)v);
  lo = (float)(v - (double)hi);
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

// FP32 block reductions for the FP32 path (FP64 adds run at a small fraction
// of the FP32 rate on GB300).  block_max_f: result in every thread.
__device__ float block_max_f(float v, float* red) {
  v = warp_max(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  float r = red[0];
#pragma unroll
  for (int i = 1; i < kNodeThreads / 32; ++i) r = fmaxf(r, red[i]);
  return r;
}

// plain sum, valid in thread 0 (the stopping terms)
__device__ float block_sum_f0(float v, float* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  float r = 0.f;
  if (threadIdx.x == 0)
#pragma unroll
    for (int i = 0; i < kNodeThreads / 32; ++i) r += red[i];
  return r;
}

// (hi, lo) + (hi, lo) with the rounding error of the hi sum kept (TwoSum)
__device__ __forceinline__ float2 add_f2(float2 a, float2 b) {
  const float s = a.x + b.x;
  const float bb = s - a.x;
  const float err = (a.x - (s - bb)) + (b.x - bb);
  return make_float2(s, (a.y + b.y) + err);
}

// compensated sum as (hi, lo), valid in thread 0 (the normaliser's partial
// sums: a few units of 2^-40 relative for non-negative terms)
__device__ float2 block_sum2_f0(float v, float2* red) {
  float2 a = make_float2(v, 0.f);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    a = add_f2(a, make_float2(__shfl_xor_sync(0xffffffffu, a.x, o), __shfl_xor_sync(0xffffffffu, a.y, o)));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = a;
  __syncthreads();
  float2 r = make_float2(0.f, 0.f);
  if (threadIdx.x == 0)
#pragma unroll
    for (int i = 0; i < kNodeThreads / 32; ++i) r = add_f2(r, red[i]);
  return r;
}

// merged message of pair (edge d, point x) minus Z_k (FP64 partials); writes its frame
__device__ __forceinline__ double merge_pair64(const NodeArgs& A, const DEdgeD& d, int n_owner, int x, double Zk) {
  const double mr = merge64(A.part64 + d.part_off + x, d.nsplit, n_owner);
  A.fr[d.off + x] = frame64(mr);
  return mr - Zk;
}

// walks the pairs q = tid, tid + T, ... of a chunk of cnt points: (edge i, point xi)
struct PairWalk {
  int i, xi, di, dx;
  __device__ PairWalk(int cnt) {
    i = (int)threadIdx.x / cnt;
    xi = (int)threadIdx.x - i * cnt;
    di = kNodeThreads / cnt;
    dx = kNodeThreads - di * cnt;
  }
  __device__ void next(int cnt) {
    i += di;
    xi += dx;
    if (xi >= cnt) {
      xi -= cnt;
      ++i;
    }
  }
};

// FP64 handles: three passes over the chunk's pairs / points in double
__device__ void chunk_update64(const NodeArgs& A, const NodeD& nd, const NodeChunk& c, const ProbD& P, double* red,
                               unsigned char* sm, int node_id) {
  using Q = double;
  const int deg = nd.deg, cnt = c.cnt, np = deg * cnt;
  const NodeSmem L = node_smem_layout(deg, cnt, true);
  DEdgeD* s_de = reinterpret_cast<DEdgeD*>(sm + L.de);
  double* s_zn = reinterpret_cast<double*>(sm + L.zn);
  int* s_di = reinterpret_cast<int*>(sm + L.di);
  int* s_dr = reinterpret_cast<int*>(sm + L.dr);
  Q* s_r = reinterpret_cast<Q*>(sm + L.r);
  double* s_mi = reinterpret_cast<double*>(sm + L.mi);
  Q* s_q = reinterpret_cast<Q*>(sm + L.q);
  double* s_s = reinterpret_cast<double*>(sm + L.s);
  Q* s_qb = reinterpret_cast<Q*>(sm + L.qb);
  const int tid = threadIdx.x, lane = tid & 31;
  for (int i = tid; i < deg; i += kNodeThreads) {
    const int di = A.node_dedges[nd.dedge_begin + i];
    const DEdgeD d = A.dedges[di];
    s_de[i] = d;
    s_zn[i] = A.Z[d.nbr];
    s_di[i] = di;
    s_dr[i] = 0;
    s_r[i] = Q(0);
  }
  __syncthreads();
  // low-precision phase: flag an edge when its operand leaves the absorbed base
  const bool track = A.absorbed && A.lowp[nd.prob] == 1;
  bool bad = false;

  if (nd.fixed) {  // a leaf: one edge, one pass
    const DEdgeD& d = s_de[0];
    Q r = Q(0);
    bool drift = false;
    for (int xi = tid; xi < cnt; xi += kNodeThreads) {
      const int x = c.x0 + xi;
      const double mi = merge_pair64(A, d, nd.n, x, s_zn[0]);
      const double fo = A.f[d.off + x];
      const double lg = A.logg[nd.node_off + x];
      const double mu = A.mu[nd.node_off + x];
      // stopping term mu |exp(f/eps + m) - 1| of the previous iterate
      if (mu > 0.0) r += fabs(mu * exp(fo * P.inv_eps + mi) - mu);
      A.f[d.off + x] = -P.eps * mi;
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
    if (__syncthreads_or(drift) && tid == 0) atomicOr(&A.drift[d.edge], 1);
    const double rs = block_sum((double)r, red);
    if (tid == 0) atomicAdd(&A.resid_acc[s_di[0]], rs);
    if (__syncthreads_or(bad) && tid == 0) atomicOr(A.err, 1);
    return;
  }

  const double Zold = A.Z[node_id];
  // pass 1, pairs: message - Z_k, its frame, and q_k(x) = exp(f_(j,k)/eps + m_(j,k) - Z_j)
  {
    PairWalk w(cnt);
    for (int q = tid; q < np; q += kNodeThreads, w.next(cnt)) {
      const DEdgeD& d = s_de[w.i];
      const int x = c.x0 + w.xi;
      const double mi = merge_pair64(A, d, nd.n, x, s_zn[w.i]);
      s_mi[q] = mi;
      const double fo = A.f[d.off + x];
      s_q[q] = exp((fo * P.inv_eps - Zold) + mi);
    }
  }
  __syncthreads();
  // pass 2, points: s(x), mean q, and the chunk's (max, sum of exp) of s
  const double inv_deg = 1.0 / (double)deg;
  double smax = -INFINITY;
  for (int xi = tid; xi < cnt; xi += kNodeThreads) {
    double ssum = 0.0;
    Q qsum = Q(0);
    for (int i = 0; i < deg; ++i) {
      ssum += s_mi[i * cnt + xi];
      qsum += s_q[i * cnt + xi];
    }
    const double s = ssum * inv_deg;
    if (!isfinite(s)) bad = true;
    s_s[xi] = s;
    s_qb[xi] = qsum * (Q)inv_deg;
    smax = fmax(smax, s);
  }
  smax = block_max(smax, red);  // its barriers also publish s_s and s_qb
  Q se = Q(0);
  for (int xi = tid; xi < cnt; xi += kNodeThreads) se += exp(s_s[xi] - smax);
  const double sse = block_sum(se, red);
  if (tid == 0) A.zpart[nd.chunk_base + c.chunk] = make_double2(smax, sse);
  // pass 3, pairs: f'_(j,k)/eps = s - m, the next apply's operand, |q_k - mean q|
  {
    PairWalk w(cnt);
    for (int q0 = 0; q0 < np; q0 += kNodeThreads) {  // warp-uniform trip count
      const int q = q0 + tid;
      const bool on = q < np;
      const int i = on ? w.i : -1;
      Q r = Q(0);
      if (on) {
        const DEdgeD& d = s_de[i];
        const int x = c.x0 + w.xi;
        const double mi = s_mi[q];
        r = s_q[q] > s_qb[w.xi] ? s_q[q] - s_qb[w.xi] : s_qb[w.xi] - s_q[q];
        const double g = s_s[w.xi] - mi;
        A.f[d.off + x] = P.eps * g;
        float hi, lo;
        split2(g * kLog2e, hi, lo);
        A.hh[d.off + x] = hi;
        A.hl[d.off + x] = lo;
        if (track && fabsf((hi - A.bh[d.off + x]) + (lo - A.bl[d.off + x])) > A.tau) s_dr[i] = 1;
        w.next(cnt);
      }
      // per-edge sums: one shared-memory atomic per warp when the warp's pairs share an edge
      const int i0 = __shfl_sync(0xffffffffu, i, 0);
      if (__all_sync(0xffffffffu, i == i0)) {
        r = warp_sum_d(r);
        if (lane == 0 && i0 >= 0) atomicAdd(&s_r[i0], r);
      } else if (on) {
        atomicAdd(&s_r[i], r);
      }
    }
  }
  __syncthreads();
  for (int i = tid; i < deg; i += kNodeThreads) {
    atomicAdd(&A.resid_acc[s_di[i]], (double)s_r[i]);
    if (s_dr[i]) atomicOr(&A.drift[s_de[i].edge], 1);
  }
  if (__syncthreads_or(bad) && tid == 0) atomicOr(A.err, 1);
}

// ---------------------------------------------------------------------------
// FP32 handles: the same three passes in log2 units on two-float values (hi on
// the 2^-10 grid, so sums and differences of hi parts are exact; lo small).
// Messages come from the merge as t + l (t = frame + exponent, exact), the
// normalisers Z as two-floats formed once per CTA, and the previous iterate's
// exponent f/eps from the operand (hh + hl) the previous update wrote.  The
// stored potentials f are not written here: the operand holds them exactly
// (f = eps ln2 (hh + hl), minus eps log mu on a fixed node), and
// materialise_f_kernel forms them in FP64 when they are read.  Only points of
// a fixed node with mu = 0, whose operand is -inf, keep f written per update.
// ---------------------------------------------------------------------------

// a value in log2 units as a two-float: hi on the grid, lo the rest
__device__ __forceinline__ float2 split_l2(double v) {
  if (!isfinite(v)) return make_float2((float)v, 0.f);
  const float hi = quant((float)v);
  return make_float2(hi, (float)(v - (double)hi));
}

// the first two partials of a pair (frame, sum), loaded ahead of the merge so
// that a thread keeps several pairs' loads in flight
struct Part2 {
  float2 a, b;
};
// The one piece of a problem in the shared-kernel phase, in two steps so that a
// thread's loads stay batched: load_sk_raw reads (R(x), S) -- the group's row
// frame and the product's sum -- and resolve_sk makes the piece (R(x) + M_j, S),
// or takes the exact fix-up's (frame, sum) where the product listed the output
// (S < 0); S = 0 is an empty column (no message).
__device__ __forceinline__ Part2 load_sk_raw(const SkEdgeS& e, int x) {
  Part2 v;
  v.a = make_float2(e.rf[x], e.s[x]);
  v.b = make_float2(0.f, 0.f);
  return v;
}
__device__ __forceinline__ void resolve_sk(Part2& v, float cm, const float2* part, int x) {
  const float S = v.a.y;
  v.a = S > 0.f ? make_float2(v.a.x + cm, S) : S == 0.f ? make_float2(0.f, 0.f) : part[x];
}

__device__ __forceinline__ Part2 load_part2(const float2* part, int nsplit, int64_t stride) {
  Part2 v;
  v.a = part[0];
  v.b = nsplit > 1 ? part[stride] : make_float2(0.f, 0.f);
  return v;
}

// the merged message in log2 units, m log2(e) = t + l with t on the grid
// (pieces 0 and 1 from v, the rest read from part)
__device__ __forceinline__ float2 merge32_l2(const Part2& v01, const float2* part, int nsplit, int64_t stride) {
  float Rm = -INFINITY;
  if (v01.a.y > 0.f) Rm = v01.a.x;
  if (v01.b.y > 0.f) Rm = fmaxf(Rm, v01.b.x);
  for (int p = 2; p < nsplit; ++p) {
    const float2 v = part[p * stride];
    if (v.y > 0.f) Rm = fmaxf(Rm, v.x);
  }
  if (Rm == -INFINITY) return make_float2(-INFINITY, 0.f);
  float S = 0.f;
  for (int p = 0; p < nsplit; ++p) {
    const float2 v = p == 0 ? v01.a : p == 1 ? v01.b : part[p * stride];
    if (v.y > 0.f) S += (v.x == Rm) ? v.y : v.y * ex2(v.x - Rm);
  }
  if (!isfinite(S) || !(S > 0.f)) return make_float2((S > 0.f) ? INFINITY : -INFINITY, 0.f);
  int e;
  const float mant = frexpf(S, &e);  // S = mant * 2^e, mant in [0.5, 1)
  const float ef = (float)e;
  const float t = Rm + ef;  // TwoSum: err is what t lost
  const float bb = t - Rm;
  const float err = (Rm - (t - bb)) + (ef - bb);
  return make_float2(t, log2f(mant) + err);
}

// (hi, lo) of hi + lo with the grid part of lo moved into hi
__device__ __forceinline__ float2 regrid(float hi, float lo) {
  const float q = quant(lo);
  return make_float2(hi + q, lo - q);
}

// One fixed leaf's chunk (FP32 path), from whichever source resolved its data:
// merge the partials (or the shared-kernel product's sum) into the message,
// the frame for the next apply, the stopping term of the previous iterate, the
// potential's operand, drift from an absorbed base; then the chunk's sums.
struct FixedView {
  int64_t d_off, part_off, node_off;
  int32_t n, x0, cnt, ns, edge, di;
  float2 zk;     // the neighbour's normaliser Z_k log2(e), two-float
  double eps_ln2;
  bool one_piece, track;
  SkEdgeS sk;
};

template <int kItF>
__device__ __forceinline__ void fixed_leaf_pass(const NodeArgs& A, const FixedView& v, double* red) {
  const int tid = threadIdx.x;
  float r = 0.f;
  bool drift = false, bad = false;
  for (int xb = 0; xb < v.cnt; xb += kItF * kNodeThreads) {
    Part2 pv[kItF];
    float4 lg[kItF];
    float oh[kItF], ol[kItF];
#pragma unroll
    for (int k = 0; k < kItF; ++k) {
      const int x = v.x0 + min(xb + tid + k * kNodeThreads, v.cnt - 1);  // past the end: reload the last point
      pv[k] = v.one_piece ? load_sk_raw(v.sk, x) : load_part2(A.part32 + v.part_off + x, v.ns, v.n);
      lg[k] = A.lgf[v.node_off + x];  // log2 mu (hi, lo), mu
      oh[k] = A.hh[v.d_off + x];
      ol[k] = A.hl[v.d_off + x];
    }
#pragma unroll
    for (int k = 0; k < kItF; ++k) {
      const int xi = xb + tid + k * kNodeThreads;
      if (xi >= v.cnt) break;
      const int x = v.x0 + xi;
      if (v.one_piece) resolve_sk(pv[k], v.sk.cm, A.part32 + v.part_off, x);
      const float2 mm = merge32_l2(pv[k], A.part32 + v.part_off + x, v.ns, v.n);
      A.fr[v.d_off + x] = isfinite(mm.x) ? quant(mm.x + mm.y) : 0.f;
      const float mh = mm.x - v.zk.x, ml = mm.y - v.zk.y;  // (m - Z_k) log2(e)
      // stopping term mu |exp(f/eps + m) - 1| of the previous iterate; f/eps log2(e) = h - log2 mu
      if (lg[k].z > 0.f) r += lg[k].z * fabsf(ex2(((oh[k] - lg[k].x) + mh) + ((ol[k] - lg[k].y) + ml)) - 1.f);
      float2 h2;
      if (lg[k].x == -INFINITY) {
        A.f[v.d_off + x] = -v.eps_ln2 * ((double)mh + (double)ml);  // mu = 0: the operand cannot carry f
        h2 = make_float2(-INFINITY, 0.f);
      } else {
        h2 = regrid(lg[k].x - mh, lg[k].y - ml);
        if (!isfinite(mh)) bad = true;
      }
      A.hh[v.d_off + x] = h2.x;
      A.hl[v.d_off + x] = h2.y;
      if (v.track && h2.x > -INFINITY && fabsf((h2.x - A.bh[v.d_off + x]) + (h2.y - A.bl[v.d_off + x])) > A.tau)
        drift = true;
    }
  }
  if (__syncthreads_or(drift) && tid == 0) atomicOr(&A.drift[v.edge], 1);
  const float rs = block_sum_f0(r, reinterpret_cast<float*>(red));
  if (tid == 0) atomicAdd(&A.resid_acc[v.di], (double)rs);
  if (__syncthreads_or(bad) && tid == 0) atomicOr(A.err, 1);
}

// A fixed leaf's chunk of a shared-kernel column (at most kSkLeafPts points per
// thread) while its problem is in the BF16 phase, the common case there: every
// load the chunk makes -- the problem's flags, the neighbour's normaliser, the
// column maximum and, for every point, the product's sum, the group's row frame,
// log2 mu and the previous operand -- leaves at once, before the flags are known
// (they only decide whether the values are used), so the chunk waits for memory
// twice (its record, then everything else) instead of once per dependent step.
// Returns false, having written nothing, when the problem is not in the phase.
// The same arithmetic as fixed_leaf_pass with one piece.
constexpr int kSkLeafPts = 4;
__device__ __forceinline__ bool fixed_sk_chunk(const NodeArgs& A, const FixedChunkD& fc, double* red) {
  const int tid = threadIdx.x;
  const int done = A.done[fc.prob];
  const int lp = A.absorbed ? A.lowp[fc.prob] : 0;
  const double zn = A.Z[fc.nbr];
  const float cm = *fc.sk.cm;
  float rfv[kSkLeafPts], sv[kSkLeafPts], oh[kSkLeafPts], ol[kSkLeafPts];
  float4 lg[kSkLeafPts];
#pragma unroll
  for (int k = 0; k < kSkLeafPts; ++k) {
    const int x = fc.x0 + min(tid + k * kNodeThreads, fc.cnt - 1);  // past the end: reload the last point
    rfv[k] = fc.sk.rf[x];
    sv[k] = fc.sk.s[x];
    lg[k] = A.lgf[fc.node_off + x];
    oh[k] = A.hh[fc.d_off + x];
    ol[k] = A.hl[fc.d_off + x];
  }
  if (done != 0) return true;  // block-uniform: retired, nothing to do
  if (lp != 1) return false;   // block-uniform: not in the phase
  const float2 zk = split_l2(zn * kLog2e);
  float r = 0.f;
  bool bad = false;
#pragma unroll
  for (int k = 0; k < kSkLeafPts; ++k) {
    const int xi = tid + k * kNodeThreads;
    if (xi >= fc.cnt) break;
    const int x = fc.x0 + xi;
    Part2 pv;
    pv.a = make_float2(rfv[k], sv[k]);
    pv.b = make_float2(0.f, 0.f);
    resolve_sk(pv, cm, A.part32 + fc.part_off, x);
    const float2 mm = merge32_l2(pv, A.part32 + fc.part_off + x, 1, fc.n);
    A.fr[fc.d_off + x] = isfinite(mm.x) ? quant(mm.x + mm.y) : 0.f;
    const float mh = mm.x - zk.x, ml = mm.y - zk.y;  // (m - Z_k) log2(e)
    // stopping term mu |exp(f/eps + m) - 1| of the previous iterate; f/eps log2(e) = h - log2 mu
    if (lg[k].z > 0.f) r += lg[k].z * fabsf(ex2(((oh[k] - lg[k].x) + mh) + ((ol[k] - lg[k].y) + ml)) - 1.f);
    float2 h2;
    if (lg[k].x == -INFINITY) {
      A.f[fc.d_off + x] = -fc.eps_ln2 * ((double)mh + (double)ml);  // mu = 0: the operand cannot carry f
      h2 = make_float2(-INFINITY, 0.f);
    } else {
      h2 = regrid(lg[k].x - mh, lg[k].y - ml);
      if (!isfinite(mh)) bad = true;
    }
    A.hh[fc.d_off + x] = h2.x;
    A.hl[fc.d_off + x] = h2.y;
  }
  // the chunk's stopping sum and error flag in one barrier
  float* red_f = reinterpret_cast<float*>(red);
  int* red_b = reinterpret_cast<int*>(red_f + kNodeThreads / 32);
  r = warp_sum(r);
  const bool wbad = __any_sync(0xffffffffu, bad);
  const int lane = tid & 31, w = tid >> 5;
  if (lane == 0) {
    red_f[w] = r;
    red_b[w] = wbad ? 1 : 0;
  }
  __syncthreads();
  if (tid == 0) {
    float rs = 0.f;
    int anyb = 0;
#pragma unroll
    for (int i = 0; i < kNodeThreads / 32; ++i) {
      rs += red_f[i];
      anyb |= red_b[i];
    }
    atomicAdd(&A.resid_acc[fc.di], (double)rs);
    if (anyb) atomicOr(A.err, 1);
  }
  return true;
}

// A fixed leaf's chunk from its host-resolved record (the fixed-leaf kernel, FP32,
// deferred bookkeeping): one load of the record, then the problem's flags, the
// neighbour's normaliser and the column maximum, then the pass -- instead of the
// chunk -> node -> owned edge -> edge record -> normaliser chain of the general path.
__device__ __forceinline__ void fixed_chunk_fast(const NodeArgs& A, const FixedChunkD& fc, double* red) {
  if (fc.cost_kind != 0 && fc.sk.s != nullptr && fc.cnt <= kSkLeafPts * kNodeThreads &&
      fixed_sk_chunk(A, fc, red))  // (record-static test: block-uniform)
    return;
  if (A.done[fc.prob] != 0) return;  // block-uniform
  const int lp = A.absorbed ? A.lowp[fc.prob] : 0;
  FixedView v;
  v.d_off = fc.d_off;
  v.part_off = fc.part_off;
  v.node_off = fc.node_off;
  v.n = fc.n;
  v.x0 = fc.x0;
  v.cnt = fc.cnt;
  v.edge = fc.edge;
  v.di = fc.di;
  v.zk = split_l2(A.Z[fc.nbr] * kLog2e);
  v.eps_ln2 = fc.eps_ln2;
  v.one_piece = lp == 1 && fc.cost_kind != 0 && fc.sk.s != nullptr;
  v.track = lp == 1 && fc.cost_kind == 0;
  v.ns = v.one_piece ? 1 : fc.nsplit;
  if (v.one_piece) v.sk = SkEdgeS{fc.sk.s, fc.sk.rf, *fc.sk.cm, 0.f};
  fixed_leaf_pass<2>(A, v, red);
}

// Point-major form of the free-node update (FP32, degree DEG <= kNodePmDeg,
// taken in the shared-kernel phase, where each message is one sum): a thread
// takes a point and all of its DEG edges -- loads every edge's sum and previous
// operand at once, then merges the messages, the previous iterate's q_k,
// s = mean_k (m - Z_k) and mean q, and writes the frames, the operands and the
// stopping terms -- with no per-pair arrays in shared memory.  The same
// arithmetic, in the same order per point, as the three passes of the
// pair-major form below; then the chunk's part of Z_j.  (With several partial
// pieces per message, as outside the phase, it gained little and its registers
// would weigh on every other handle's node update.)
template <int DEG, bool ONE>
__device__ __forceinline__ void free_points32(const NodeArgs& A, const NodeD& nd, const NodeChunk& c, double* red,
                                              const DEdgeD* s_de, const float2* s_zk, int* s_dr, float* s_r,
                                              const SkEdgeS* s_sk, float2* s_s, bool track, float2 zo, bool& bad) {
  constexpr bool one_piece = ONE;  // the shared-kernel phase: one sum per output
  const int tid = threadIdx.x, lane = tid & 31, cnt = c.cnt;
  const float fdeg = (float)DEG, inv_deg = 1.f / fdeg;
  float r[DEG];
#pragma unroll
  for (int k = 0; k < DEG; ++k) r[k] = 0.f;
  float smax = -INFINITY;
  for (int xi = tid; xi < cnt; xi += kNodeThreads) {
    const int x = c.x0 + xi;
    Part2 pv[DEG];
    float oh[DEG], ol[DEG];
#pragma unroll
    for (int k = 0; k < DEG; ++k) {
      const DEdgeD& d = s_de[k];
      pv[k] = one_piece ? load_sk_raw(s_sk[k], x) : load_part2(A.part32 + d.part_off + x, d.nsplit, nd.n);
      oh[k] = A.hh[d.off + x];  // f/eps log2(e) of the previous iterate
      ol[k] = A.hl[d.off + x];
    }
    float2 m[DEG];
    float q[DEG];
    float sh = 0.f, sl = 0.f, qsum = 0.f;
#pragma unroll
    for (int k = 0; k < DEG; ++k) {
      const DEdgeD& d = s_de[k];
      if (one_piece) resolve_sk(pv[k], s_sk[k].cm, A.part32 + d.part_off, x);
      const float2 mm = merge32_l2(pv[k], A.part32 + d.part_off + x, one_piece ? 1 : d.nsplit, nd.n);
      A.fr[d.off + x] = isfinite(mm.x) ? quant(mm.x + mm.y) : 0.f;
      const float2 zk = s_zk[k];
      const float mh = mm.x - zk.x, ml = mm.y - zk.y;
      m[k] = make_float2(mh, ml);
      q[k] = ex2(((oh[k] + mh) - zo.x) + ((ol[k] + ml) - zo.y));
      const float t = sh + mh;  // TwoSum of the hi parts, in edge order
      const float bb = t - sh;
      sl += ((sh - (t - bb)) + (mh - bb)) + ml;
      sh = t;
      qsum += q[k];
    }
    const float sm_h = quant(sh * inv_deg);
    const float sm_l = (fmaf(-sm_h, fdeg, sh) + sl) * inv_deg;
    if (!isfinite(sm_h)) bad = true;
    s_s[xi] = make_float2(sm_h, sm_l);
    const float qb = qsum * inv_deg;
    smax = fmaxf(smax, sm_h + sm_l);
    // g = s - (m - Z_k) (f'/eps in log2, the operand), |q_k - mean q|
#pragma unroll
    for (int k = 0; k < DEG; ++k) {
      const DEdgeD& d = s_de[k];
      r[k] += fabsf(q[k] - qb);
      const float2 g = regrid(sm_h - m[k].x, sm_l - m[k].y);
      A.hh[d.off + x] = g.x;
      A.hl[d.off + x] = g.y;
      if (track && fabsf((g.x - A.bh[d.off + x]) + (g.y - A.bl[d.off + x])) > A.tau) s_dr[k] = 1;
    }
  }
#pragma unroll
  for (int k = 0; k < DEG; ++k) {
    const float v = warp_sum(r[k]);
    if (lane == 0) atomicAdd(&s_r[k], v);
  }
  smax = block_max_f(smax, reinterpret_cast<float*>(red));  // its barriers also publish s_s
  const float sq = isfinite(smax) ? quant(smax) : 0.f;
  float se = 0.f;
  for (int xi = tid; xi < cnt; xi += kNodeThreads) se += ex2((s_s[xi].x - sq) + s_s[xi].y);
  const float2 sse = block_sum2_f0(se, reinterpret_cast<float2*>(red));
  if (tid == 0) A.zpart[nd.chunk_base + c.chunk] = make_double2((double)sq * kLn2, (double)sse.x + (double)sse.y);
}

// PM: the kernel carries the point-major form for the shared-kernel phase
// (handles with shared-kernel groups; it needs more registers than the rest)
template <bool FIXED_ONLY, bool PM = false>
__device__ void chunk_update32(const NodeArgs& A, const NodeD& nd, const NodeChunk& c, const ProbD& P, double* red,
                               unsigned char* sm, int node_id) {
  const int deg = nd.deg, cnt = c.cnt, np = deg * cnt;
  const NodeSmem L = node_smem_layout(deg, cnt, false);
  DEdgeD* s_de = reinterpret_cast<DEdgeD*>(sm + L.de);
  float2* s_zk = reinterpret_cast<float2*>(sm + L.zn);  // Z_k log2(e) as two-floats
  int* s_di = reinterpret_cast<int*>(sm + L.di);
  int* s_dr = reinterpret_cast<int*>(sm + L.dr);
  float* s_r = reinterpret_cast<float*>(sm + L.r);
  float2* s_mi = reinterpret_cast<float2*>(sm + L.mi);  // (m - Z_k) log2(e)
  float* s_q = reinterpret_cast<float*>(sm + L.q);
  float2* s_s = reinterpret_cast<float2*>(sm + L.s);    // s log2(e)
  float* s_qb = reinterpret_cast<float*>(sm + L.qb);
  SkEdgeS* s_sk = reinterpret_cast<SkEdgeS*>(sm + L.sk);
  const int tid = threadIdx.x, lane = tid & 31;
  // the shared-kernel phase leaves one sum per output (its product's, or the
  // fix-up's piece); drift from an absorbed base is tracked on stored-cost
  // problems, the only ones absorbed
  const int lp = A.absorbed ? A.lowp[nd.prob] : 0;
  const bool track = lp == 1 && P.cost_kind == 0;
  const bool one_piece = lp == 1 && P.cost_kind != 0 && A.sk_ref;
  for (int i = tid; i < deg; i += kNodeThreads) {
    const int di = A.node_dedges[nd.dedge_begin + i];
    const DEdgeD d = A.dedges[di];
    s_de[i] = d;
    s_zk[i] = split_l2(A.Z[d.nbr] * kLog2e);
    s_di[i] = di;
    s_dr[i] = 0;
    s_r[i] = 0.f;
    if (one_piece) {
      const SkRefD r = A.sk_ref[di];
      s_sk[i] = SkEdgeS{r.s, r.rf, *r.cm, 0.f};
    }
  }
  __syncthreads();
  bool bad = false;
  // a thread loads a batch of kIt pairs before it stores anything
  constexpr int kIt = 4;

  if (FIXED_ONLY || nd.fixed) {  // a leaf: one edge, one pass
    const DEdgeD& d = s_de[0];
    FixedView v;
    v.d_off = d.off;
    v.part_off = d.part_off;
    v.node_off = nd.node_off;
    v.n = nd.n;
    v.x0 = c.x0;
    v.cnt = cnt;
    v.ns = one_piece ? 1 : d.nsplit;
    v.edge = d.edge;
    v.di = s_di[0];
    v.zk = s_zk[0];
    v.eps_ln2 = P.eps * kLn2;
    v.one_piece = one_piece;
    v.track = track;
    if (one_piece) v.sk = s_sk[0];
    // the fixed-leaf kernel batches two pairs per thread (fewer live registers, more CTAs per SM)
    fixed_leaf_pass<FIXED_ONLY ? 2 : kIt>(A, v, red);
    return;
  }

  const float2 zo = split_l2(A.Z[node_id] * kLog2e);
  if (PM && !FIXED_ONLY && deg <= kNodePmDeg && one_piece) {
    float2* s_pm = reinterpret_cast<float2*>(sm + L.mi);  // s per point, where the per-pair arrays start
#define TREEOT_PM(D)                                                                                          \
  case D:                                                                                                     \
    free_points32<D, true>(A, nd, c, red, s_de, s_zk, s_dr, s_r, s_sk, s_pm, track, zo, bad);                 \
    break;
    switch (deg) {
      TREEOT_PM(1)
      TREEOT_PM(2)
      TREEOT_PM(3)
      TREEOT_PM(4)
      TREEOT_PM(5)
      TREEOT_PM(6)
      TREEOT_PM(7)
      TREEOT_PM(8)
      default:
        break;
    }
#undef TREEOT_PM
    __syncthreads();
    for (int i = tid; i < deg; i += kNodeThreads) {
      atomicAdd(&A.resid_acc[s_di[i]], (double)s_r[i]);
      if (s_dr[i]) atomicOr(&A.drift[s_de[i].edge], 1);
    }
    if (__syncthreads_or(bad) && tid == 0) atomicOr(A.err, 1);
    return;
  }
  // pass 1, pairs: (m - Z_k) log2(e), its frame, and q_k = exp(f_(j,k)/eps + m_(j,k) - Z_j)
  {
    PairWalk w(cnt);
    for (int qb = 0; qb < np; qb += kIt * kNodeThreads) {
      Part2 pv[kIt];
      float oh[kIt], ol[kIt];
      int pi[kIt], px[kIt];
#pragma unroll
      for (int k = 0; k < kIt; ++k) {
        const bool on = qb + tid + k * kNodeThreads < np;
        pi[k] = on ? w.i : 0;  // past the end: reload pair (0, 0)
        px[k] = on ? w.xi : 0;
        if (on) w.next(cnt);
        const DEdgeD& d = s_de[pi[k]];
        const int x = c.x0 + px[k];
        pv[k] = one_piece ? load_sk_raw(s_sk[pi[k]], x) : load_part2(A.part32 + d.part_off + x, d.nsplit, nd.n);
        oh[k] = A.hh[d.off + x];  // f/eps log2(e) of the previous iterate
        ol[k] = A.hl[d.off + x];
      }
#pragma unroll
      for (int k = 0; k < kIt; ++k) {
        const int q = qb + tid + k * kNodeThreads;
        if (q >= np) break;
        const DEdgeD& d = s_de[pi[k]];
        const int x = c.x0 + px[k];
        if (one_piece) resolve_sk(pv[k], s_sk[pi[k]].cm, A.part32 + d.part_off, x);
        const float2 mm = merge32_l2(pv[k], A.part32 + d.part_off + x, one_piece ? 1 : d.nsplit, nd.n);
        A.fr[d.off + x] = isfinite(mm.x) ? quant(mm.x + mm.y) : 0.f;
        const float2 zk = s_zk[pi[k]];
        const float mh = mm.x - zk.x, ml = mm.y - zk.y;
        s_mi[q] = make_float2(mh, ml);
        s_q[q] = ex2(((oh[k] + mh) - zo.x) + ((ol[k] + ml) - zo.y));
      }
    }
  }
  __syncthreads();
  // pass 2, points: s = mean_k (m - Z_k), mean q, and the chunk's part of Z_j
  const float fdeg = (float)deg, inv_deg = 1.f / fdeg;
  float smax = -INFINITY;
  for (int xi = tid; xi < cnt; xi += kNodeThreads) {
    float sh = 0.f, sl = 0.f, qsum = 0.f;
    for (int i = 0; i < deg; ++i) {
      const float2 v = s_mi[i * cnt + xi];
      const float t = sh + v.x;  // TwoSum of the hi parts
      const float bb = t - sh;
      sl += ((sh - (t - bb)) + (v.x - bb)) + v.y;
      sh = t;
      qsum += s_q[i * cnt + xi];
    }
    const float mh = quant(sh * inv_deg);
    const float ml = (fmaf(-mh, fdeg, sh) + sl) * inv_deg;
    if (!isfinite(mh)) bad = true;
    s_s[xi] = make_float2(mh, ml);
    s_qb[xi] = qsum * inv_deg;
    smax = fmaxf(smax, mh + ml);
  }
  smax = block_max_f(smax, reinterpret_cast<float*>(red));  // its barriers also publish s_s and s_qb
  const float sq = isfinite(smax) ? quant(smax) : 0.f;
  float se = 0.f;
  for (int xi = tid; xi < cnt; xi += kNodeThreads) se += ex2((s_s[xi].x - sq) + s_s[xi].y);
  const float2 sse = block_sum2_f0(se, reinterpret_cast<float2*>(red));
  if (tid == 0) A.zpart[nd.chunk_base + c.chunk] = make_double2((double)sq * kLn2, (double)sse.x + (double)sse.y);
  // pass 3, pairs: g = s - (m - Z_k) (f'/eps in log2, the operand; f' = eps ln2 g), |q_k - mean q|
  {
    PairWalk w(cnt);
    for (int q0 = 0; q0 < np; q0 += kNodeThreads) {  // warp-uniform trip count
      const int q = q0 + tid;
      const bool on = q < np;
      const int i = on ? w.i : -1;
      float r = 0.f;
      if (on) {
        const DEdgeD& d = s_de[i];
        const int x = c.x0 + w.xi;
        const float2 mi = s_mi[q], sv = s_s[w.xi];
        r = fabsf(s_q[q] - s_qb[w.xi]);
        const float2 g = regrid(sv.x - mi.x, sv.y - mi.y);
        A.hh[d.off + x] = g.x;
        A.hl[d.off + x] = g.y;
        if (track && fabsf((g.x - A.bh[d.off + x]) + (g.y - A.bl[d.off + x])) > A.tau) s_dr[i] = 1;
        w.next(cnt);
      }
      const int i0 = __shfl_sync(0xffffffffu, i, 0);
      if (__all_sync(0xffffffffu, i == i0)) {
        r = warp_sum(r);
        if (lane == 0 && i0 >= 0) atomicAdd(&s_r[i0], r);
      } else if (on) {
        atomicAdd(&s_r[i], r);
      }
    }
  }
  __syncthreads();
  for (int i = tid; i < deg; i += kNodeThreads) {
    atomicAdd(&A.resid_acc[s_di[i]], (double)s_r[i]);
    if (s_dr[i]) atomicOr(&A.drift[s_de[i].edge], 1);
  }
  if (__syncthreads_or(bad) && tid == 0) atomicOr(A.err, 1);
}

// Z_j of a free node from its chunks' (max, sum) pieces of s, and rho_j
__device__ __forceinline__ void finish_free_node(const NodeArgs& A, int node, const NodeD& nd) {
  double M = -INFINITY;
  for (int k = 0; k < nd.nchunks; ++k) M = fmax(M, A.zpart[nd.chunk_base + k].x);
  double S = 0.0;
  for (int k = 0; k < nd.nchunks; ++k) {
    const double2 z = A.zpart[nd.chunk_base + k];
    S += z.y * exp(z.x - M);
  }
  const double Zn = M + log(S);
  A.Z[node] = Zn;
  A.rho[node] = -(double)nd.deg * Zn;
}

// The same, by a whole warp (every lane gets the result): the exponentials of
// the chunks in parallel lanes, then the sum in chunk order by every lane, so
// the result is bit-identical to finish_free_node's (FP64 transcendental work
// by one lane at a time is slow on this GPU).
__device__ __forceinline__ void finish_free_node_warp(const NodeArgs& A, int node, const NodeD& nd, int lane) {
  double M = -INFINITY;
  for (int k = lane; k < nd.nchunks; k += 32) M = fmax(M, A.zpart[nd.chunk_base + k].x);
  M = warp_max_d(M);
  double S = 0.0;
  for (int k0 = 0; k0 < nd.nchunks; k0 += 32) {
    double zy = 0.0, ex = 0.0;
    if (k0 + lane < nd.nchunks) {
      const double2 z = A.zpart[nd.chunk_base + k0 + lane];
      zy = z.y;
      ex = exp(z.x - M);
    }
    const int m = min(32, nd.nchunks - k0);
    for (int i = 0; i < m; ++i) S += __shfl_sync(0xffffffffu, zy, i) * __shfl_sync(0xffffffffu, ex, i);
  }
  if (lane == 0) {
    const double Zn = M + log(S);
    A.Z[node] = Zn;
    A.rho[node] = -(double)nd.deg * Zn;
  }
}

// The stopping quantity of iterate t_now of problem p is complete (rs: the
// sum of its terms, rm: the largest): phase control and retirement, then the
// counters of the next launch.
__device__ __forceinline__ void problem_after_update(const NodeArgs& A, int p, const ProbD& P, int64_t t_now,
                                                     double rs, double rm) {
  const double crit = A.tol_kind == 1 ? rm : rs;
  const int lp = A.absorbed ? A.lowp[p] : 0;
  if (lp == 2 && t_now + 1 >= A.lowp_start) {
    // enter the low-precision phase: absorb every edge of the problem next
    A.lowp[p] = 1;
    if (A.fp32_live) atomicSub(A.fp32_live, 1);  // the FP32 applies skip it from now on
    A.lowp_span[2 * p] = t_now + 1;
    A.lowp_best[p] = INFINITY;
    A.lowp_best_t[p] = t_now + 1;
    for (int k = 0; k < P.edge_count; ++k) A.drift[P.edge_begin + k] = 1;
  } else if (lp == 1) {
    // the phase's accuracy is enough until the stopping quantity reaches
    // refine_tol; from then on (or once the phase stops improving) the FP32
    // kernel refines.  refine_tol = 0 keeps a problem in the phase.
    if (crit < A.refine_tol || !(crit == crit)) {
      A.lowp[p] = 0;
      A.lowp_span[2 * p + 1] = t_now + 1;
      if (A.fp32_live) atomicAdd(A.fp32_live, 1);  // back to the FP32 applies
    } else if (crit < 0.9 * A.lowp_best[p]) {
      A.lowp_best[p] = crit;
      A.lowp_best_t[p] = t_now;
    } else if (A.refine_tol > 0.0 && t_now - A.lowp_best_t[p] > kLowpStall) {
      A.lowp[p] = 0;
      A.lowp_span[2 * p + 1] = t_now + 1;
      if (A.fp32_live) atomicAdd(A.fp32_live, 1);
    }
  } else if (A.retire && (crit < A.ptol[p] || t_now + 1 >= A.deadline[p])) {
    A.done[p] = 1;
    A.done_at[p] = t_now + 1;
    if (A.fp32_live) atomicSub(A.fp32_live, 1);  // retired: no FP32 apply any more
  }
  A.node_count[p] = 0;
  const int nslot = (int)((t_now + 1) % kResidRing);
  A.res_sum[nslot * A.nprob + p] = 0.0;
  A.res_max[nslot * A.nprob + p] = 0ull;
}

// One node-update item: chunk c of a node of the active colour at half-step
// t_now (the number of half-steps done before it).  Unless the launch defers
// it to node_finish_kernel, thread 0 also does the chunk's arrival
// bookkeeping: the last chunk of a node merges Z_j and the node's stopping
// terms; the last node of a problem records the stopping quantity of iterate
// t_now and (when asked) retires the problem.
template <bool F64, bool FIXED_ONLY = false, bool PM = false>
__device__ __forceinline__ void node_chunk_item(const NodeArgs& A, const NodeChunk c, int64_t t_now,
                                                unsigned char* node_sm, double* red) {
  const NodeD nd = A.nodes[c.node];
  const int p = nd.prob;
  const ProbD P = A.probs[p];
  const int slot = (int)(t_now % kResidRing);
  const bool skip = A.done[p] != 0;
  if (!skip) {
    if constexpr (F64)
      chunk_update64(A, nd, c, P, red, node_sm, c.node);
    else
      chunk_update32<FIXED_ONLY, PM>(A, nd, c, P, red, node_sm, c.node);
  }
  if (A.defer) return;  // launch-uniform: the chunk's terms are in resid_acc and zpart
  __syncthreads();
  if (threadIdx.x != 0) return;
  __threadfence();
  if (!skip && atomicAdd(&A.node_arrive[c.node], 1) == nd.nchunks - 1) {
    // last chunk of this node: finish Z_j and the node's stopping terms
    __threadfence();
    if (!nd.fixed) finish_free_node(A, c.node, nd);
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
      problem_after_update(A, p, P, t_now, rs, rm);
    }
  }
}

}  // namespace
}  // namespace treeot
