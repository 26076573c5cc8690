// Absorbed low-precision edge apply for stored costs (BF16 Gibbs kernel with
// FP32 accumulation), the absorption step that builds it, and flag clearing.
//
// Absorption (per edge e = (a,b), rows a, columns b).  With the apply operands
// A(x) = h_(a,b)(x), B(y) = h_(b,a)(y) (base 2, two-float, see apply_f32.cu)
// taken as the edge's bases, the kernel stores
//     Kt(x,y) = 2^( A(x) + B(y) - s C(x,y) - rho(x) ),   rho(x) = max_y (...)
// rounded to BF16 (so every row has maximum 1 and BF16's FP32 exponent range
// covers the rest).  Afterwards the messages of the block updates are GEMVs:
//     row node a:    m2(x) = rho(x) - A(x) + log2 sum_y Kt(x,y) 2^(h_(b,a)(y) - B(y))
//     column node b: m2(y) = -B(y) + log2 sum_x Kt(x,y) 2^(h_(a,b)(x) - A(x) + rho(x))
// The frame of each output (rho - A_hi, or -B_hi) sits on the 2^-10 grid and
// the low parts enter the sum as a factor, so the node update's merge is the
// one of the log-sum-exp kernel.  Only the BF16 rounding of Kt (relative 2^-9
// per entry) limits accuracy, which is why problems switch to the FP32 kernel
// below a stopping-quantity threshold.
#include <cuda_bf16.h>

#include <algorithm>
#include <cfloat>
#include <cmath>

#include "internal.h"
#include "ptx.cuh"

namespace treeot {
namespace {

#define kInf (__int_as_float(0x7f800000))
constexpr int kBfRowsPerIter = 4;  // ROW: rows per warp iteration (16 loads of 16 B in flight per lane)
constexpr int kBfColChunk = 8;     // COL: rows per chunk (8 loads of 16 B in flight per lane)

__device__ __forceinline__ float quantf(float v) { return rintf(v * 1024.f) * (1.f / 1024.f); }

__device__ __forceinline__ float bf_lo(uint32_t u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf_hi(uint32_t u) { return __uint_as_float(u & 0xffff0000u); }

// ---------------------------------------------------------------------------
// absorption: one CTA per (edge, 64-row block); acts only on flagged edges of
// problems in the low-precision phase
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) absorb_kernel(AbsorbArgs A) {
  for (int ti = blockIdx.x; ti < A.ntasks; ti += gridDim.x) {
    const Task t = A.tasks[ti];  // dedge = 2e (row side), o0/ocount = rows
    const DEdgeD da = A.dedges[t.dedge];
    if (A.lowp[da.prob] != 1 || !A.drift[da.edge]) continue;
    const DEdgeD db = A.dedges[t.dedge + 1];
    const EdgeD e = A.edges[da.edge];
    const ProbD P = A.probs[da.prob];
    const float shi = P.s2, slo = P.s2_lo;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // column bases: the whole column operand, copied once per edge
    if (t.o0 == 0) {
      if (threadIdx.x == 0) atomicAdd(A.count, 1ull);
      for (int y = threadIdx.x; y < e.nb; y += blockDim.x) {
        A.bh[db.off + y] = A.hh[db.off + y];
        A.bl[db.off + y] = A.hl[db.off + y];
      }
    }
    for (int r = warp; r < t.ocount; r += 8) {
      const int x = t.o0 + r;
      const float ah = A.hh[da.off + x], al = A.hl[da.off + x];
      const float* Crow = e.C + (int64_t)x * e.ld;
      __nv_bfloat16* Krow = reinterpret_cast<__nv_bfloat16*>(e.K) + (int64_t)x * e.ldk;
      // pass 1: row maximum of A + B - sC (exact grid sums, small final rounding)
      float mx = -kInf;
      if (ah > -kInf) {
        for (int y = lane; y < e.nb; y += 32) {
          const float c = Crow[y];
          float v = fmaf(-c, shi, ah + A.hh[db.off + y]);
          v = fmaf(-c, slo, v) + (al + A.hl[db.off + y]);
          mx = fmaxf(mx, v);
        }
      }
      mx = warp_max(mx);
      const float rho = mx > -kInf ? quantf(mx) : 0.f;
      // pass 2: Kt = 2^(value - rho) in BF16; padding columns are zero
      for (int y = lane; y < e.ldk; y += 32) {
        float k = 0.f;
        if (y < e.nb && ah > -kInf) {
          const float c = Crow[y];
          float v = fmaf(-c, shi, (ah - rho) + A.hh[db.off + y]);
          v = fmaf(-c, slo, v) + (al + A.hl[db.off + y]);
          k = ex2(v);
        }
        Krow[y] = __float2bfloat16_rn(k);
      }
      if (lane == 0) {
        A.arho[da.off + x] = rho;
        A.bh[da.off + x] = ah;
        A.bl[da.off + x] = al;
      }
    }
  }
}

__global__ void clear_flags_kernel(int32_t* drift, int32_t nedges) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nedges; i += gridDim.x * blockDim.x) drift[i] = 0;
}

// ---------------------------------------------------------------------------
// absorbed apply
// ---------------------------------------------------------------------------
__device__ void bf_row_task(const ApplyArgs& A, const Task& t, float* sm) {
  const DEdgeD d = A.dedges[t.dedge];  // owner = row node a
  const EdgeD e = A.edges[d.edge];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nvec = (t.rcount + 7) >> 3;  // uint4 = 8 BF16 entries
  constexpr int W = kApplyThreads / 32;
  // kBfRowsPerIter rows per warp iteration: 4 x kBfRowsPerIter 16-byte loads in flight per lane
  uint4 k[kBfRowsPerIter][4];
  auto load = [&](int r) {
#pragma unroll
    for (int q = 0; q < kBfRowsPerIter; ++q) {
      const int rq = r + q * W;
      const bool has = rq < t.ocount;
      const uint4* row = reinterpret_cast<const uint4*>(e.K + (int64_t)(t.o0 + (has ? rq : r)) * e.ldk + t.r0);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int v = lane + 32 * i;
        k[q][i] = (v < nvec && has) ? ldg_stream_u4(row + v) : make_uint4(0u, 0u, 0u, 0u);
      }
    }
  };
  // the first rows are in flight while the task's weights are formed
  if (warp < t.ocount) load(warp);
  float* wv = sm;  // [kRowCols] weights of the reduction columns
  for (int i = threadIdx.x; i < kRowCols; i += kApplyThreads) {
    float w = 0.f;
    if (i < t.rcount) {
      const int64_t o = d.rev_off + t.r0 + i;
      const float hh = A.hh[o];
      if (hh > -kInf) w = ex2((hh - A.bh[o]) + (A.hl[o] - A.bl[o]));  // mu = 0 entries weigh nothing
    }
    wv[i] = w;
  }
  __syncthreads();
  for (int r = warp; r < t.ocount; r += kBfRowsPerIter * W) {
    if (r != warp) load(r);
    float acc[kBfRowsPerIter];
#pragma unroll
    for (int q = 0; q < kBfRowsPerIter; ++q) acc[q] = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int y0 = 8 * (lane + 32 * i);
      const float4 w0 = *reinterpret_cast<const float4*>(wv + y0);
      const float4 w1 = *reinterpret_cast<const float4*>(wv + y0 + 4);
#pragma unroll
      for (int q = 0; q < kBfRowsPerIter; ++q) {
        acc[q] = fmaf(bf_lo(k[q][i].x), w0.x, acc[q]);
        acc[q] = fmaf(bf_hi(k[q][i].x), w0.y, acc[q]);
        acc[q] = fmaf(bf_lo(k[q][i].y), w0.z, acc[q]);
        acc[q] = fmaf(bf_hi(k[q][i].y), w0.w, acc[q]);
        acc[q] = fmaf(bf_lo(k[q][i].z), w1.x, acc[q]);
        acc[q] = fmaf(bf_hi(k[q][i].z), w1.y, acc[q]);
        acc[q] = fmaf(bf_lo(k[q][i].w), w1.z, acc[q]);
        acc[q] = fmaf(bf_hi(k[q][i].w), w1.w, acc[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < kBfRowsPerIter; ++q) {
      const float sq = warp_sum(acc[q]);
      const int rq = r + q * W;
      if (lane == 0 && rq < t.ocount) {
        const int x = t.o0 + rq;
        A.part32[d.part_off + (int64_t)t.split * e.na + x] =
            make_float2(A.arho[d.off + x] - A.bh[d.off + x], sq * ex2(-A.bl[d.off + x]));
      }
    }
  }
  __syncthreads();
}

__device__ void bf_col_task(const ApplyArgs& A, const Task& t, float* sm) {
  const DEdgeD d = A.dedges[t.dedge];  // owner = column node b
  const EdgeD e = A.edges[d.edge];
  float* wv = sm;                    // [kRowCols] weights of the reduction rows (<= kRowCols per split)
  float* comb = sm + kRowCols;       // [8][kBfCols] per-warp column sums
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rpw = (t.rcount + 7) / 8;
  const int rr0 = warp * rpw;
  const int rr1 = min(rr0 + rpw, t.rcount);
  const int c0 = 8 * lane;
  const bool on = c0 < t.ocount;
  const uint16_t* base = e.K + t.o0 + c0;
  uint4 k[kBfColChunk];  // kBfColChunk 16-byte loads in flight per lane
  auto load = [&](int rr) {
#pragma unroll
    for (int i = 0; i < kBfColChunk; ++i) {
      const int xr = rr + i;
      k[i] = (on && xr < rr1) ? ldg_stream_u4(reinterpret_cast<const uint4*>(base + (int64_t)(t.r0 + xr) * e.ldk))
                              : make_uint4(0u, 0u, 0u, 0u);
    }
  };
  load(rr0);  // the first rows are in flight while the task's weights are formed
  for (int i = threadIdx.x; i < t.rcount; i += kApplyThreads) {
    float w = 0.f;
    if (i < t.rcount) {
      const int64_t o = d.rev_off + t.r0 + i;  // row-side vectors (owner a)
      const float hh = A.hh[o];
      if (hh > -kInf) w = ex2((hh - A.bh[o]) + (A.hl[o] - A.bl[o]) + A.arho[o]);
    }
    wv[i] = w;
  }
  __syncthreads();
  float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int rr = rr0; rr < rr1; rr += kBfColChunk) {
    if (rr != rr0) load(rr);
#pragma unroll
    for (int i = 0; i < kBfColChunk; ++i) {
      const float w = (rr + i < rr1) ? wv[rr + i] : 0.f;
      acc[0] = fmaf(bf_lo(k[i].x), w, acc[0]);
      acc[1] = fmaf(bf_hi(k[i].x), w, acc[1]);
      acc[2] = fmaf(bf_lo(k[i].y), w, acc[2]);
      acc[3] = fmaf(bf_hi(k[i].y), w, acc[3]);
      acc[4] = fmaf(bf_lo(k[i].z), w, acc[4]);
      acc[5] = fmaf(bf_hi(k[i].z), w, acc[5]);
      acc[6] = fmaf(bf_lo(k[i].w), w, acc[6]);
      acc[7] = fmaf(bf_hi(k[i].w), w, acc[7]);
    }
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) comb[warp * kBfCols + c0 + j] = acc[j];
  __syncthreads();
  for (int c = threadIdx.x; c < t.ocount; c += kApplyThreads) {
    float S = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) S += comb[w * kBfCols + c];
    const int y = t.o0 + c;
    const float R = -A.bh[d.off + y];
    A.part32[d.part_off + (int64_t)t.split * e.nb + y] = make_float2(R, S * ex2(-A.bl[d.off + y]));
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kApplyThreads, 2) apply_bf16_kernel(ApplyArgs A) {
  __shared__ __align__(16) float sm[kRowCols + 8 * kBfCols];  // 12 KB
  for (int ti = blockIdx.x; ti < A.ntasks; ti += gridDim.x) {
    const Task t = A.tasks[ti];
    const int prob = A.dedges[t.dedge].prob;
    if (A.done[prob] || A.lowp[prob] != 1) continue;
    if (t.kind == TASK_ROW)
      bf_row_task(A, t, sm);
    else
      bf_col_task(A, t, sm);
  }
}

}  // namespace

int apply_bf16_ctas_per_sm() {
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, apply_bf16_kernel, kApplyThreads, 0);
  return n > 0 ? n : 1;
}

cudaError_t launch_apply_bf16(const ApplyArgs& a, int grid, cudaStream_t s) {
  if (a.ntasks <= 0) return cudaSuccess;
  apply_bf16_kernel<<<grid, kApplyThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_absorb(const AbsorbArgs& a, int grid, cudaStream_t s) {
  if (a.ntasks <= 0) return cudaSuccess;
  absorb_kernel<<<grid, 256, 0, s>>>(a);
  clear_flags_kernel<<<std::max(1, std::min(1024, (a.nedges + 255) / 256)), 256, 0, s>>>(a.drift, a.nedges);
  return cudaGetLastError();
}

}  // namespace treeot
