// Edge apply, FP32 per-element arithmetic: one persistent launch computes the
// partial log-sum-exp messages of every directed edge owned by the active colour
// (Theorem 1's K_(j,k)(u_(k,j) gamma_k), in log form), in base 2:
//
//   m2_(j,k)(x) = log2 sum_y 2^( h_(k,j)(y) - s * C(x,y) ),
//   h_(k,j)(y)  = (f_(k,j)(y)/eps + log gamma_k(y)) * log2(e)   (two floats: hi + lo)
//   s           = log2(e) / eps.
//
// Each thread keeps, per output x, a frame R (an FP32 value close to the row's
// maximum, seeded from the previous message of that row) and a sum of
// 2^(t - R).  The per-element argument t = (hh - R) + hl - s*C stays small for
// the terms that matter, so FP32 rounding of large potentials never enters.
// A chunk whose maximum exceeds the frame (or lies far below it) moves the
// frame.  Results are written as (frame, sum) pairs per reduction split and
// merged by the node-update kernel in FP64.
//
// Task kinds: ROW (stored matrix, reduce along a contiguous row: one warp per
// row, lanes across 1024 columns), COL (stored matrix, reduce down columns: a
// warp owns 128 columns, 8 warps split the rows, merged through shared
// memory), RECOMP (squared-Euclidean cost recomputed from coordinates: each
// thread owns 4 outputs, reduction points are staged in shared memory).
#include <cfloat>
#include <cmath>

#include "internal.h"
#include "ptx.cuh"

namespace treeot {

namespace {

#define kInf (__int_as_float(0x7f800000))

// shift all terms of a thread's chunk when its maximum leaves the frame
__device__ __forceinline__ void maybe_reframe(float cm, float& R, float* t, int cnt) {
  if ((cm > 0.f || cm < -64.f) && cm > -kInf) {
    R += cm;
    for (int i = 0; i < cnt; ++i) t[i] -= cm;
  }
}

__device__ void row_task(const ApplyArgs& A, const Task& t, float* sm) {
  const DEdgeD d = A.dedges[t.dedge];
  const EdgeD e = A.edges[d.edge];
  const float s = A.probs[d.prob].s2;
  const int n_owner = e.na;
  float* sh = sm;
  float* sl = sm + kRowCols;
  const int tid = threadIdx.x;
  for (int i = tid; i < kRowCols; i += kApplyThreads) {
    const bool v = i < t.rcount;
    sh[i] = v ? A.hh[d.rev_off + t.r0 + i] : 0.f;
    sl[i] = v ? A.hl[d.rev_off + t.r0 + i] : 0.f;
  }
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5;
  const int nvec = (t.rcount + 3) >> 2;
  const float4* sh4 = reinterpret_cast<const float4*>(sh);
  const float4* sl4 = reinterpret_cast<const float4*>(sl);
  const float2 negs = make_float2(-s, -s);
  for (int r = warp; r < t.ocount; r += kApplyThreads / 32) {
    const int x = t.o0 + r;
    const float4* row = reinterpret_cast<const float4*>(e.C + (int64_t)x * e.ld + t.r0);
    float4 c[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int v = lane + 32 * i;
      c[i] = v < nvec ? ldg_stream(row + v) : make_float4(kInf, kInf, kInf, kInf);
    }
    float R = frame_of(A.m[d.off + x]);
    const float2 negR = make_float2(-R, -R);
    float tv[32];
    float cm = -kInf;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int v = lane + 32 * i;
      const float4 H = sh4[v];
      const float4 L = sl4[v];
      const float2 d01 = add2(add2(make_float2(H.x, H.y), negR), make_float2(L.x, L.y));
      const float2 d23 = add2(add2(make_float2(H.z, H.w), negR), make_float2(L.z, L.w));
      const float2 t01 = fma2(make_float2(c[i].x, c[i].y), negs, d01);
      const float2 t23 = fma2(make_float2(c[i].z, c[i].w), negs, d23);
      tv[4 * i + 0] = t01.x;
      tv[4 * i + 1] = t01.y;
      tv[4 * i + 2] = t23.x;
      tv[4 * i + 3] = t23.y;
      cm = max3f(cm, t01.x, t01.y);
      cm = max3f(cm, t23.x, t23.y);
    }
    maybe_reframe(cm, R, tv, 32);
    // pairwise sum of the 32 terms
    float p[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) p[i] = ex2(tv[2 * i]) + ex2(tv[2 * i + 1]);
#pragma unroll
    for (int w = 8; w >= 1; w >>= 1)
#pragma unroll
      for (int i = 0; i < w; ++i) p[i] += p[i + w];
    float acc = p[0];
    const float Rm = warp_max(R);
    acc = (R == Rm) ? acc : acc * ex2(R - Rm);
    acc = warp_sum(acc);
    if (lane == 0) A.part32[d.part_off + (int64_t)t.split * n_owner + x] = make_float2(Rm, acc);
  }
  __syncthreads();
}

__device__ void col_task(const ApplyArgs& A, const Task& t, float* sm) {
  const DEdgeD d = A.dedges[t.dedge];
  const EdgeD e = A.edges[d.edge];
  const float s = A.probs[d.prob].s2;
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
  const int c0 = 4 * lane;                      // first of this lane's 4 columns (task-relative)
  const bool lane_on = c0 < t.ocount;
  float R[4], acc[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int col = t.o0 + c0 + k;
    R[k] = (lane_on && c0 + k < t.ocount) ? frame_of(A.m[d.off + col]) : 0.f;
    acc[k] = 0.f;
  }
  const float2 negs = make_float2(-s, -s);
  const float* base = e.C + t.o0 + c0;
  for (int rr = rr0; rr < rr1; rr += 8) {
    float4 c[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int xr = rr + i;
      c[i] = (lane_on && xr < rr1)
                 ? ldg_stream(reinterpret_cast<const float4*>(base + (int64_t)(t.r0 + xr) * e.ld))
                 : make_float4(kInf, kInf, kInf, kInf);
    }
    float tv[4][8];
    const float2 nR01 = make_float2(-R[0], -R[1]);
    const float2 nR23 = make_float2(-R[2], -R[3]);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int xr = min(rr + i, kColRows - 1);
      const float hh = sh[xr], hl = sl[xr];
      const float2 d01 = add2(add2(make_float2(hh, hh), nR01), make_float2(hl, hl));
      const float2 d23 = add2(add2(make_float2(hh, hh), nR23), make_float2(hl, hl));
      const float2 t01 = fma2(make_float2(c[i].x, c[i].y), negs, d01);
      const float2 t23 = fma2(make_float2(c[i].z, c[i].w), negs, d23);
      tv[0][i] = t01.x;
      tv[1][i] = t01.y;
      tv[2][i] = t23.x;
      tv[3][i] = t23.y;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float cm = max3f(tv[k][0], tv[k][1], tv[k][2]);
      cm = max3f(cm, tv[k][3], tv[k][4]);
      cm = max3f(cm, tv[k][5], tv[k][6]);
      cm = fmaxf(cm, tv[k][7]);
      if ((cm > 0.f || (acc[k] == 0.f && cm < -64.f)) && cm > -kInf) {
        acc[k] *= ex2(-cm);
        R[k] += cm;
#pragma unroll
        for (int i = 0; i < 8; ++i) tv[k][i] -= cm;
      }
      const float a = (ex2(tv[k][0]) + ex2(tv[k][1])) + (ex2(tv[k][2]) + ex2(tv[k][3]));
      const float b = (ex2(tv[k][4]) + ex2(tv[k][5])) + (ex2(tv[k][6]) + ex2(tv[k][7]));
      acc[k] += a + b;
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) comb[warp * kColCols + c0 + k] = make_float2(R[k], acc[k]);
  __syncthreads();
  for (int c = tid; c < t.ocount; c += kApplyThreads) {
    float Rm = -kInf;
#pragma unroll
    for (int w = 0; w < 8; ++w) Rm = fmaxf(Rm, comb[w * kColCols + c].x);
    float S = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      const float2 p = comb[w * kColCols + c];
      S += (p.x == Rm) ? p.y : p.y * ex2(p.x - Rm);
    }
    A.part32[d.part_off + (int64_t)t.split * n_owner + t.o0 + c] = make_float2(Rm, S);
  }
  __syncthreads();
}

// squared Euclidean cost from coordinates; D in {1,2,3}
template <int D>
__device__ void recomp_task(const ApplyArgs& A, const Task& t, float* sm) {
  const DEdgeD d = A.dedges[t.dedge];
  const NodeD own = A.nodes[d.owner];
  const NodeD nbn = A.nodes[d.nbr];
  const float s = A.probs[d.prob].s2_scaled;
  const int n_owner = own.n;
  const int tid = threadIdx.x;
  float4* st = reinterpret_cast<float4*>(sm);           // [256]: (-q0, -q1, -q2 or hh, hh or hl)
  float* stl = sm + 4 * kApplyThreads;                  // [256]: hl (D == 3)
  float px[4], py[4], pz[4], R[4], acc[4];
  bool on[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int lo = tid + kApplyThreads * i;
    on[i] = lo < t.ocount;
    const int o = t.o0 + (on[i] ? lo : 0);
    const float* p = A.coords + own.coord_off + (int64_t)o * D;
    px[i] = p[0];
    py[i] = D > 1 ? p[1] : 0.f;
    pz[i] = D > 2 ? p[2] : 0.f;
    R[i] = on[i] ? frame_of(A.m[d.off + o]) : 0.f;
    acc[i] = 0.f;
  }
  const float2 negs = make_float2(-s, -s);
  for (int ch = 0; ch < t.rcount; ch += kApplyThreads) {
    __syncthreads();
    {
      const int j = ch + tid;
      const bool v = j < t.rcount;
      const int y = t.r0 + (v ? j : 0);
      const float* q = A.coords + nbn.coord_off + (int64_t)y * D;
      const float hh = v ? A.hh[d.rev_off + y] : -kInf;
      const float hl = v ? A.hl[d.rev_off + y] : 0.f;
      if (D == 3) {
        st[tid] = make_float4(-q[0], -q[1], -q[2], hh);
        stl[tid] = hl;
      } else {
        st[tid] = make_float4(-q[0], D > 1 ? -q[1] : 0.f, hh, hl);
      }
    }
    __syncthreads();
    const int cnt = min(kApplyThreads, t.rcount - ch);
    const float2 nR01 = make_float2(-R[0], -R[1]);
    const float2 nR23 = make_float2(-R[2], -R[3]);
    const float2 px01 = make_float2(px[0], px[1]), px23 = make_float2(px[2], px[3]);
    const float2 py01 = make_float2(py[0], py[1]), py23 = make_float2(py[2], py[3]);
    const float2 pz01 = make_float2(pz[0], pz[1]), pz23 = make_float2(pz[2], pz[3]);
    for (int j = 0; j < cnt; j += 8) {
      float tv[4][8];
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        const float4 q = st[j + jj];       // entries past cnt hold hh = -inf: zero terms
        float hh, hl;
        if (D == 3) {
          hh = q.w;
          hl = stl[j + jj];
        } else {
          hh = q.z;
          hl = q.w;
        }
        const float2 qx = make_float2(q.x, q.x);
        float2 c01, c23;
        {
          const float2 dx01 = add2(px01, qx), dx23 = add2(px23, qx);
          c01 = mul2(dx01, dx01);
          c23 = mul2(dx23, dx23);
        }
        if (D > 1) {
          const float2 qy = make_float2(q.y, q.y);
          const float2 dy01 = add2(py01, qy), dy23 = add2(py23, qy);
          c01 = fma2(dy01, dy01, c01);
          c23 = fma2(dy23, dy23, c23);
        }
        if (D > 2) {
          const float2 qz = make_float2(q.z, q.z);
          const float2 dz01 = add2(pz01, qz), dz23 = add2(pz23, qz);
          c01 = fma2(dz01, dz01, c01);
          c23 = fma2(dz23, dz23, c23);
        }
        const float2 hh2 = make_float2(hh, hh), hl2 = make_float2(hl, hl);
        const float2 d01 = add2(add2(hh2, nR01), hl2);
        const float2 d23 = add2(add2(hh2, nR23), hl2);
        const float2 t01 = fma2(c01, negs, d01);
        const float2 t23 = fma2(c23, negs, d23);
        tv[0][jj] = t01.x;
        tv[1][jj] = t01.y;
        tv[2][jj] = t23.x;
        tv[3][jj] = t23.y;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        float cm = max3f(tv[k][0], tv[k][1], tv[k][2]);
        cm = max3f(cm, tv[k][3], tv[k][4]);
        cm = max3f(cm, tv[k][5], tv[k][6]);
        cm = fmaxf(cm, tv[k][7]);
        if ((cm > 0.f || (acc[k] == 0.f && cm < -64.f)) && cm > -kInf) {
          acc[k] *= ex2(-cm);
          R[k] += cm;
#pragma unroll
          for (int i = 0; i < 8; ++i) tv[k][i] -= cm;
        }
        const float a = (ex2(tv[k][0]) + ex2(tv[k][1])) + (ex2(tv[k][2]) + ex2(tv[k][3]));
        const float b = (ex2(tv[k][4]) + ex2(tv[k][5])) + (ex2(tv[k][6]) + ex2(tv[k][7]));
        acc[k] += a + b;
      }
    }
    // frames may have moved: the next chunk re-reads R
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (on[i]) {
      const int o = t.o0 + tid + kApplyThreads * i;
      A.part32[d.part_off + (int64_t)t.split * n_owner + o] = make_float2(R[i], acc[i]);
    }
  }
}

__global__ void __launch_bounds__(kApplyThreads, 2) apply_f32_kernel(ApplyArgs A) {
  __shared__ __align__(16) float sm[2 * kColRows + 2 * 8 * kColCols];  // 12 KB, covers all task kinds
  for (int ti = blockIdx.x; ti < A.ntasks; ti += gridDim.x) {
    const Task t = A.tasks[ti];
    const int prob = A.dedges[t.dedge].prob;
    if (A.done[prob]) continue;
    switch (t.kind) {
      case TASK_ROW:
        row_task(A, t, sm);
        break;
      case TASK_COL:
        col_task(A, t, sm);
        break;
      default: {
        const int D = A.probs[prob].dim;
        if (D == 1)
          recomp_task<1>(A, t, sm);
        else if (D == 2)
          recomp_task<2>(A, t, sm);
        else
          recomp_task<3>(A, t, sm);
        __syncthreads();
      }
    }
  }
}

}  // namespace

int apply_ctas_per_sm() {
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, apply_f32_kernel, kApplyThreads, 0);
  return n > 0 ? n : 1;
}

cudaError_t launch_apply_f32(const ApplyArgs& a, int grid, cudaStream_t s) {
  if (a.ntasks <= 0) return cudaSuccess;
  apply_f32_kernel<<<grid, kApplyThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace treeot
