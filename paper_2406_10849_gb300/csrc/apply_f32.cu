// Edge apply, FP32 per-element arithmetic: one persistent launch computes the
// partial log-sum-exp messages of every directed edge owned by the active colour
// (the K_(j,k)(u_(k,j) gamma_k) of the block-update theorem, in log form), in
// base 2:
//
//   m2_(j,k)(x) = log2 sum_y 2^( h_(k,j)(y) - s * C(x,y) ),
//   h_(k,j)(y)  = (f_(k,j)(y)/eps + log gamma_k(y)) * log2(e),    s = log2(e)/eps.
//
// Exactness of the per-element argument.  h arrives as two floats, hh on a
// 2^-10 grid plus a small remainder hl; every frame R (a per-output shift close
// to the running maximum) is kept on the same grid.  hh - R is then exact, the
// product C*s is formed inside an FMA (s itself as s_hi + s_lo), and only the
// small final argument t = (hh - R) - C*s + hl is ever rounded.  Terms near the
// maximum therefore carry ~1e-7 relative error however large f/eps and C/eps are.
//
// Frames.  A frame starts at the output's previous message.  A chunk whose
// maximum lies above the frame, or (when nothing has been accumulated yet) far
// below it, moves the frame to the quantised chunk maximum and the chunk's terms
// are recomputed from the new frame.  Results are (frame, sum) pairs per
// reduction split; the node update merges them, ignoring empty pieces.
//
// Task kinds: ROW (stored matrix, reduce along a contiguous row: one warp per
// row with a warp-uniform frame, lanes across 1024 columns), COL (stored matrix,
// reduce down columns: a warp owns 128 columns, 8 warps split the rows and merge
// through shared memory) -- both in apply_dense_kernel, where each term is formed
// once (maximum and sum together) and only re-formed when a frame moves -- and RECOMP
// (squared-Euclidean cost recomputed from coordinates: each thread owns 4
// outputs, reduction points staged in shared memory) in apply_recomp_kernel<D>.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <mutex>

#include "internal.h"
#include "ptx.cuh"
#include "recomp_task.cuh"

namespace treeot {

namespace {

// ROW task: rows o0..o0+ocount of the stored matrix against 1024 columns; one
// warp per row, the task's operand staged in shared memory.  Every term is
// formed once (maximum and sum relative to the row's frame in one pass); only
// when the maximum leaves the frame's window (early half-steps) is the row
// summed again from the moved frame, so results equal those of a separate
// maximum pass.
__device__ void row_task(const ApplyArgs& A, const Task& t, float* sm) {
  const DEdgeD d = A.dedges[t.dedge];
  const EdgeD e = A.edges[d.edge];
  const ProbD P = A.probs[d.prob];
  // owner = row node: rows of C; owner = column node (pad = 1): rows of the transpose
  const float* Cm = t.pad ? e.CT : e.C;
  const int64_t ldm = t.pad ? e.ldt : e.ld;
  const int n_owner = t.pad ? e.nb : e.na;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int nvec = (t.rcount + 3) >> 2;
  const uint32_t row_bytes = 16u * (uint32_t)nvec;  // within the row: the stride is padded to 4 floats
  float4 c[8];
  auto load = [&](int r) {
    const int x = t.o0 + r;
    const float4* row = reinterpret_cast<const float4*>(Cm + (int64_t)x * ldm + t.r0);
    // the warp's next row heads for L2 while this one is in flight
    if (lane == 0 && r + kApplyThreads / 32 < t.ocount)
      prefetch_l2(Cm + (int64_t)(x + kApplyThreads / 32) * ldm + t.r0, row_bytes);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int v = lane + 32 * i;
      c[i] = v < nvec ? ldg_stream(row + v) : make_float4(kInf, kInf, kInf, kInf);
    }
  };
  if (warp < t.ocount) load(warp);  // the first row is in flight while the operand is staged
  float* sh = sm;
  float* sl = sm + kRowCols;
  for (int i = tid; i < kRowCols; i += kApplyThreads) {
    const bool v = i < t.rcount;
    sh[i] = v ? A.hh[d.rev_off + t.r0 + i] : 0.f;
    sl[i] = v ? A.hl[d.rev_off + t.r0 + i] : 0.f;
  }
  __syncthreads();
  const float4* sh4 = reinterpret_cast<const float4*>(sh);
  const float4* sl4 = reinterpret_cast<const float4*>(sl);
  const float2 nhi = make_float2(-P.s2, -P.s2), nlo = make_float2(-P.s2_lo, -P.s2_lo);
  for (int r = warp; r < t.ocount; r += kApplyThreads / 32) {
    const int x = t.o0 + r;
    if (r != warp) load(r);
    float R = A.fr[d.off + x];  // warp-uniform, on the grid
    float cm = -kInf, acc = 0.f;
    {
      const float2 negR = make_float2(-R, -R);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int v = lane + 32 * i;
        float2 t01, t23;
        terms4(c[i], sh4[v], sl4[v], negR, nhi, nlo, t01, t23);
        cm = max3f(cm, t01.x, t01.y);
        cm = max3f(cm, t23.x, t23.y);
        acc += (ex2(t01.x) + ex2(t01.y)) + (ex2(t23.x) + ex2(t23.y));
      }
    }
    const float cw = warp_max(cm);
    if ((cw > 0.5f || cw < -kWindow) && cw > -kInf) {  // warp-uniform: move onto the grid, sum again
      R += quant(cw);
      acc = 0.f;
      const float2 negR = make_float2(-R, -R);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int v = lane + 32 * i;
        float2 t01, t23;
        terms4(c[i], sh4[v], sl4[v], negR, nhi, nlo, t01, t23);
        acc += (ex2(t01.x) + ex2(t01.y)) + (ex2(t23.x) + ex2(t23.y));
      }
    }
    acc = warp_sum(acc);
    if (lane == 0) A.part32[d.part_off + (int64_t)t.split * n_owner + x] = make_float2(R, acc);
  }
  __syncthreads();
}


// COL task: 128 columns (4 per lane) of the stored matrix against up to 512
// rows, split over the 8 warps.  Per chunk of 8 rows every term is formed once
// (maximum and sum together); a column whose maximum leaves its frame's window
// has the chunk summed again from the moved frame (results equal those of a
// separate maximum pass).
__device__ void col_task(const ApplyArgs& A, const Task& t, float* sm) {
  const DEdgeD d = A.dedges[t.dedge];
  const EdgeD e = A.edges[d.edge];
  const ProbD P = A.probs[d.prob];
  const int n_owner = e.nb;
  float* sh = sm;
  float* sl = sm + kColRows;
  float2* comb = reinterpret_cast<float2*>(sm + 2 * kColRows);  // [8][kColCols]
  const int tid = threadIdx.x;
  for (int i = tid; i < kColRows; i += kApplyThreads) {
    const bool v = i < t.rcount;
    sh[i] = v ? A.hh[d.rev_off + t.r0 + i] : 0.f;
    sl[i] = v ? A.hl[d.rev_off + t.r0 + i] : 0.f;
  }
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5;
  const int rpw = (t.rcount + 7) / 8;
  const int rr0 = warp * rpw;
  const int rr1 = min(rr0 + rpw, t.rcount);
  const int c0 = 4 * lane;  // first of this lane's 4 columns (task-relative)
  const bool lane_on = c0 < t.ocount;
  float R[4], acc[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    R[k] = (lane_on && c0 + k < t.ocount) ? A.fr[d.off + t.o0 + c0 + k] : 0.f;
    acc[k] = 0.f;
  }
  const float2 nhi = make_float2(-P.s2, -P.s2), nlo = make_float2(-P.s2_lo, -P.s2_lo);
  const float* base = e.C + t.o0 + c0;
  const uint32_t chunk_bytes = 16u * (uint32_t)((t.ocount + 3) >> 2);  // the task's columns of one row
  for (int rr = rr0; rr < rr1; rr += 8) {
    // the warp's next 8 rows head for L2 while these are in flight
    if (lane < 8 && rr + 8 + lane < rr1)
      prefetch_l2(e.C + (int64_t)(t.r0 + rr + 8 + lane) * e.ld + t.o0, chunk_bytes);
    float4 c[8];
    float hh[8], hl[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int xr = rr + i;
      const bool ok = xr < rr1;
      c[i] = (lane_on && ok) ? ldg_stream(reinterpret_cast<const float4*>(base + (int64_t)(t.r0 + xr) * e.ld))
                             : make_float4(kInf, kInf, kInf, kInf);
      hh[i] = ok ? sh[xr] : 0.f;
      hl[i] = ok ? sl[xr] : 0.f;
    }
    float cm[4] = {-kInf, -kInf, -kInf, -kInf};
    float2 a01 = make_float2(0.f, 0.f), a23 = make_float2(0.f, 0.f);
    {
      const float2 nR01 = make_float2(-R[0], -R[1]);
      const float2 nR23 = make_float2(-R[2], -R[3]);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float2 h2 = make_float2(hh[i], hh[i]), l2 = make_float2(hl[i], hl[i]);
        float2 t01 = fma2(make_float2(c[i].x, c[i].y), nhi, add2(h2, nR01));
        float2 t23 = fma2(make_float2(c[i].z, c[i].w), nhi, add2(h2, nR23));
        t01 = add2(fma2(make_float2(c[i].x, c[i].y), nlo, t01), l2);
        t23 = add2(fma2(make_float2(c[i].z, c[i].w), nlo, t23), l2);
        cm[0] = fmaxf(cm[0], t01.x);
        cm[1] = fmaxf(cm[1], t01.y);
        cm[2] = fmaxf(cm[2], t23.x);
        cm[3] = fmaxf(cm[3], t23.y);
        a01 = add2(a01, make_float2(ex2(t01.x), ex2(t01.y)));
        a23 = add2(a23, make_float2(ex2(t23.x), ex2(t23.y)));
      }
    }
    float part[4] = {a01.x, a01.y, a23.x, a23.y};
    bool moved[4];
    bool any = false;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      moved[k] = (cm[k] > 0.5f || (acc[k] == 0.f && cm[k] < -kWindow)) && cm[k] > -kInf;
      any = any || moved[k];
    }
    if (any) {  // rare after the first half-steps: re-sum the chunk for the moved columns
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (!moved[k]) continue;
        const float Rn = R[k] + quant(cm[k]);
        acc[k] = acc[k] == 0.f ? 0.f : acc[k] * ex2(R[k] - Rn);
        R[k] = Rn;
        float sk = 0.f;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float ck = k == 0 ? c[i].x : k == 1 ? c[i].y : k == 2 ? c[i].z : c[i].w;
          sk += ex2(arg1(hh[i], Rn, ck, P.s2, P.s2_lo, hl[i]));
        }
        part[k] = sk;
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[k] += part[k];
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) comb[warp * kColCols + c0 + k] = make_float2(R[k], acc[k]);
  __syncthreads();
  for (int c = tid; c < t.ocount; c += kApplyThreads)
    A.part32[d.part_off + (int64_t)t.split * n_owner + t.o0 + c] = merge_pieces(comb + c, 8, kColCols);
  __syncthreads();
}

__global__ void __launch_bounds__(kApplyThreads, 2) apply_dense_kernel(ApplyArgs A) {
  __shared__ __align__(16) float sm[2 * kColRows + 2 * 8 * kColCols];  // 12 KB
  // every problem retired or in a BF16 phase: nothing to apply (the same for every CTA)
  if (A.fp32_live && *((volatile const int32_t*)A.fp32_live) <= 0) return;
  for (int ti = blockIdx.x; ti < A.ntasks; ti += gridDim.x) {
    const Task t = A.tasks[ti];
    const int prob = A.dedges[t.dedge].prob;
    if (A.done[prob] || A.lowp[prob] == 1) continue;  // retired, or in the absorbed BF16 phase
    if (t.kind == TASK_ROW)
      row_task(A, t, sm);
    else
      col_task(A, t, sm);
  }
}

// Tasks come from a work queue (an atomic counter; tasks are sorted by cost on
// the host), so uneven edges of a batch of trees balance across the CTAs.  The
// last CTA to leave resets the counter for the next launch.
// EXACT: some problems run the exact-distance variant (A.exact); instantiated
// separately so the plain kernel keeps its register budget.
template <int D, int MINB, bool EXACT>
__global__ void __launch_bounds__(kApplyThreads, MINB) apply_recomp_kernel(ApplyArgs A) {
  __shared__ __align__(16) float sm[16 * kApplyThreads + 2 * 4 * kApplyThreads];  // 24 KB
  __shared__ int s_ti;
  // every problem retired or in a BF16 phase: nothing to apply (the same for every CTA; the
  // work queue is then untouched and stays reset)
  if (A.fp32_live && *((volatile const int32_t*)A.fp32_live) <= 0) return;
  for (;;) {
    if (threadIdx.x == 0) s_ti = atomicAdd(&A.queue[0], 1);
    __syncthreads();
    const int ti = s_ti;
    __syncthreads();
    if (ti >= A.ntasks) break;
    const Task t = A.tasks[ti];
    const int prob = A.dedges[t.dedge].prob;
    if (A.done[prob] || A.lowp[prob] == 1) continue;  // retired, or in a BF16 phase
    if (EXACT && A.exact[prob])  // block-uniform: refined past the plain recomputation's floor
      recomp_task_exact<D>(A, t, sm);
    else
      recomp_task<D>(A, t, sm);
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&A.queue[1], 1) == (int)gridDim.x - 1) {
      A.queue[0] = 0;
      A.queue[1] = 0;
      __threadfence();
    }
  }
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the stored-cost row apply (see
// tree_ot_edge_apply_noalloc in include/tree_ot.h).  Its scratch (the two-float
// operand and the per-split partial sums) lives in one file-scope device array
// instead of memory the caller or the library allocates.
// ---------------------------------------------------------------------------

constexpr int64_t kNoAllocScratchFloats = int64_t(1) << 20;  // 4 MiB per device
static __device__ __align__(256) float g_noalloc_scratch[kNoAllocScratchFloats];

// h(y) = g(y) * log2(e) as a two-float (hi on the 2^-10 grid); y < n_cols
__global__ void noalloc_operand_kernel(const double* g, int32_t n_cols, float* hh, float* hl) {
  for (int y = blockIdx.x * blockDim.x + threadIdx.x; y < n_cols; y += gridDim.x * blockDim.x) {
    const double v = g[y] * 1.4426950408889634074;
    if (!isfinite(v)) {
      hh[y] = (float)v;
      hl[y] = 0.f;
    } else {
      const float hi = (float)(rint(v * 1024.0) / 1024.0);
      hh[y] = hi;
      hl[y] = (float)(v - (double)hi);
    }
  }
}

// one CTA per (64-row block, 1024-column split); a warp per row, frame found
// by a max pass over the register-resident costs, then the sum pass
__global__ void __launch_bounds__(kApplyThreads) noalloc_row_kernel(const float* C, int64_t ld, int32_t n_rows,
                                                                    int32_t n_cols, const float* hh_g,
                                                                    const float* hl_g, float shi, float slo,
                                                                    int32_t nsplit, float2* part) {
  __shared__ __align__(16) float sh[kRowCols];
  __shared__ __align__(16) float sl[kRowCols];
  const int split = blockIdx.x % nsplit;
  const int o0 = (blockIdx.x / nsplit) * (8 * kRowRowsPerWarp);
  const int r0 = split * kRowCols;
  const int rcount = min(kRowCols, n_cols - r0);
  const int ocount = min(8 * kRowRowsPerWarp, n_rows - o0);
  for (int i = threadIdx.x; i < kRowCols; i += kApplyThreads) {
    const bool v = i < rcount;
    sh[i] = v ? hh_g[r0 + i] : 0.f;
    sl[i] = v ? hl_g[r0 + i] : 0.f;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float4* sh4 = reinterpret_cast<const float4*>(sh);
  const float4* sl4 = reinterpret_cast<const float4*>(sl);
  const float2 nhi = make_float2(-shi, -shi), nlo = make_float2(-slo, -slo);
  const int nvec = (rcount + 3) >> 2;
  for (int r = warp; r < ocount; r += kApplyThreads / 32) {
    const int x = o0 + r;
    const float* rowp = C + (int64_t)x * ld + r0;
    float4 c[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int v = lane + 32 * i;
      if (v < nvec) {
        c[i] = ldg_stream(reinterpret_cast<const float4*>(rowp) + v);
        // columns past n_cols belong to the caller's row padding: no term
        const int y = 4 * v;
        if (y + 0 >= rcount) c[i].x = kInf;
        if (y + 1 >= rcount) c[i].y = kInf;
        if (y + 2 >= rcount) c[i].z = kInf;
        if (y + 3 >= rcount) c[i].w = kInf;
      } else {
        c[i] = make_float4(kInf, kInf, kInf, kInf);
      }
    }
    float R = 0.f;
    float cm = -kInf;
    for (int pass = 0; pass < 2; ++pass) {
      const float2 negR = make_float2(-R, -R);
      float acc = 0.f;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int v = lane + 32 * i;
        const float4 H = sh4[v];
        const float4 L = sl4[v];
        float2 t01 = fma2(make_float2(c[i].x, c[i].y), nhi, add2(make_float2(H.x, H.y), negR));
        float2 t23 = fma2(make_float2(c[i].z, c[i].w), nhi, add2(make_float2(H.z, H.w), negR));
        t01 = add2(fma2(make_float2(c[i].x, c[i].y), nlo, t01), make_float2(L.x, L.y));
        t23 = add2(fma2(make_float2(c[i].z, c[i].w), nlo, t23), make_float2(L.z, L.w));
        if (pass == 0) {
          cm = max3f(cm, t01.x, t01.y);
          cm = max3f(cm, t23.x, t23.y);
        } else {
          acc += (ex2(t01.x) + ex2(t01.y)) + (ex2(t23.x) + ex2(t23.y));
        }
      }
      if (pass == 0) {
        const float cw = warp_max(cm);
        if (cw > -kInf) R = quant(cw);
      } else {
        acc = warp_sum(acc);
        if (lane == 0) part[(int64_t)split * n_rows + x] = make_float2(R, acc);
      }
    }
  }
}

// m_out[x] = ln 2 * (R + log2 sum_s S_s 2^(R_s - R)) over the non-empty pieces
// (natural log).  The pieces are merged and the logarithm taken in FP64 (one
// double log per row), so the output adds no rounding beyond the pieces' own.
__global__ void noalloc_merge_kernel(const float2* part, int32_t n_rows, int32_t nsplit, double* m_out) {
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < n_rows; x += gridDim.x * blockDim.x) {
    float Rm = -kInf;
    for (int s = 0; s < nsplit; ++s) {
      const float2 v = part[(int64_t)s * n_rows + x];
      if (v.y > 0.f) Rm = fmaxf(Rm, v.x);
    }
    if (Rm == -kInf) {
      m_out[x] = -INFINITY;
      continue;
    }
    double S = 0.0;
    for (int s = 0; s < nsplit; ++s) {
      const float2 v = part[(int64_t)s * n_rows + x];
      if (v.y > 0.f) S += (double)v.y * exp2((double)v.x - (double)Rm);  // frames on the 2^-10 grid: exact
    }
    m_out[x] = (double)Rm * 0.69314718055994530942 + log(S);
  }
}

}  // namespace

template <int D, int MINB>
int occ_recomp() {
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, apply_recomp_kernel<D, MINB, false>, kApplyThreads, 0);
  return n > 0 ? n : 1;
}

int apply_ctas_per_sm(int slot, int variant) {
  int n = 0;
  if (slot == 0) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, apply_dense_kernel, kApplyThreads, 0);
    return n > 0 ? n : 1;
  }
  if (variant == 0) return slot == 1 ? occ_recomp<1, 2>() : slot == 2 ? occ_recomp<2, 2>() : occ_recomp<3, 2>();
  return slot == 1 ? occ_recomp<1, 3>() : slot == 2 ? occ_recomp<2, 3>() : occ_recomp<3, 3>();
}

cudaError_t launch_apply_f32(const ApplyArgs& a, int slot, int variant, int grid, cudaStream_t s) {
  if (a.ntasks <= 0) return cudaSuccess;
  if (slot == 0) {
    apply_dense_kernel<<<grid, kApplyThreads, 0, s>>>(a);
  } else if (a.any_exact) {
    // rare (after certification): the 2-CTA register budget, whatever the tuned variant
    if (slot == 1) apply_recomp_kernel<1, 2, true><<<grid, kApplyThreads, 0, s>>>(a);
    if (slot == 2) apply_recomp_kernel<2, 2, true><<<grid, kApplyThreads, 0, s>>>(a);
    if (slot == 3) apply_recomp_kernel<3, 2, true><<<grid, kApplyThreads, 0, s>>>(a);
  } else if (variant == 0) {
    if (slot == 1) apply_recomp_kernel<1, 2, false><<<grid, kApplyThreads, 0, s>>>(a);
    if (slot == 2) apply_recomp_kernel<2, 2, false><<<grid, kApplyThreads, 0, s>>>(a);
    if (slot == 3) apply_recomp_kernel<3, 2, false><<<grid, kApplyThreads, 0, s>>>(a);
  } else {
    if (slot == 1) apply_recomp_kernel<1, 3, false><<<grid, kApplyThreads, 0, s>>>(a);
    if (slot == 2) apply_recomp_kernel<2, 3, false><<<grid, kApplyThreads, 0, s>>>(a);
    if (slot == 3) apply_recomp_kernel<3, 3, false><<<grid, kApplyThreads, 0, s>>>(a);
  }
  return cudaGetLastError();
}

// ---- allocation-free entry point: host side ---------------------------------

namespace {
constexpr int kNoAllocMaxDevices = 64;
float* g_noalloc_dev_ptr[kNoAllocMaxDevices] = {};
std::mutex g_noalloc_mu;
}  // namespace

// Device address of the scratch array for the current device; resolved once per
// device (this lookup is the only set-up the entry point performs).
cudaError_t noalloc_scratch(float** out, int64_t* capacity_floats) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_dev_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_dev_ptr[dev] = static_cast<float*>(p);
  }
  *out = g_noalloc_dev_ptr[dev];
  *capacity_floats = kNoAllocScratchFloats;
  return cudaSuccess;
}

int64_t noalloc_scratch_floats_needed(int32_t n_rows, int32_t n_cols) {
  const int64_t nsplit = (n_cols + kRowCols - 1) / kRowCols;
  const int64_t op = 2 * ((int64_t)(n_cols + 63) / 64 * 64);
  return op + 2 * nsplit * (int64_t)n_rows;
}

cudaError_t launch_edge_apply_noalloc(const float* C, int64_t ld, int32_t n_rows, int32_t n_cols, const double* g,
                                      float shi, float slo, double* m_out, float* scratch, cudaStream_t s) {
  const int32_t nsplit = (n_cols + kRowCols - 1) / kRowCols;
  const int64_t op_len = (int64_t)(n_cols + 63) / 64 * 64;
  float* hh = scratch;
  float* hl = scratch + op_len;
  float2* part = reinterpret_cast<float2*>(scratch + 2 * op_len);  // 2*op_len is a multiple of 128 floats
  const int ob = (n_rows + 8 * kRowRowsPerWarp - 1) / (8 * kRowRowsPerWarp);
  noalloc_operand_kernel<<<std::min<int64_t>(1024, (n_cols + 255) / 256), 256, 0, s>>>(g, n_cols, hh, hl);
  noalloc_row_kernel<<<ob * nsplit, kApplyThreads, 0, s>>>(C, ld, n_rows, n_cols, hh, hl, shi, slo, nsplit, part);
  noalloc_merge_kernel<<<std::min<int64_t>(1024, (n_rows + 255) / 256), 256, 0, s>>>(part, n_rows, nsplit, m_out);
  return cudaGetLastError();
}

}  // namespace treeot
