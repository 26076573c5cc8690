// Shared-kernel BF16 phase: for a group of directed edges that share one
// squared-Euclidean Gibbs kernel, one colour's messages are one matrix product
// on the tensor cores (sk.h states the arithmetic).  Per group and colour:
//   sk_envelope(1)_kernel  M_j = max_y h_j(y), b(y) = max over the active columns of h_j(y) - M_j
//                          (one pass with per-CTA envelopes and sk_envelope_reduce_kernel, or two)
//   sk_kvbuild_kernel      R(x) and K'(x,y) = 2^(b(y) - R(x) - s C(x,y)) (sk_kbuild_row), and
//                          V'(y,j) = 2^(h_j(y) - M_j - b(y)) (sk_vbuild_cols), BF16 hi + lo
//   sk_gemm_tc_kernel      S = K'hi V'hi + K'hi V'lo + K'lo V'hi (tcgen05, FP32 accumulation in
//                          tensor memory; sk_gemm_kernel: mma.sync m16n8k16); S(x,j) per output
//   sk_fixup_kernel        outputs with S < 2^-96 recomputed as an FP32 log-sum-exp
// M, b and R live on the 2^-10 grid, so b - R and h - M - b are exact and the cost
// term is formed as in the recomputed-cost apply (FMAs with s = s_hi + s_lo).
#include <cudaTypedefs.h>  // PFN_cuTensorMapEncodeTiled (the encoder is fetched through the runtime)
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cfloat>
#include <cmath>
#include <cstdint>

#include "ptx.cuh"
#include "sk.h"

namespace treeot {
namespace {

#define kInf (__int_as_float(0x7f800000))

__device__ __forceinline__ float quant(float v) { return rintf(v * 1024.f) * (1.f / 1024.f); }

__device__ __forceinline__ bool col_active(const SkArgs& A, const SkCol& c) {
  return !A.done[c.prob] && A.lowp[c.prob] == 1;
}

// max of floats through integer atomics on their bit patterns
__device__ __forceinline__ void atomic_max_float(float* addr, float v) {
  if (!(v > -kInf)) return;  // -inf and NaN change nothing
  if (v >= 0.f)
    atomicMax(reinterpret_cast<int*>(addr), __float_as_int(v));
  else
    atomicMin(reinterpret_cast<unsigned int*>(addr), __float_as_uint(v));
}

constexpr int kEnvCols = kSkEnvCols;

// h + l of four consecutive points from a, b (16-byte aligned when y0 + 4 <= n)
__device__ __forceinline__ void load_sum4(const float* a, const float* b, int y0, int n, float* v) {
  if (y0 + 4 <= n) {
    const float4 h = *reinterpret_cast<const float4*>(a + y0);
    const float4 l = *reinterpret_cast<const float4*>(b + y0);
    v[0] = h.x + l.x;
    v[1] = h.y + l.y;
    v[2] = h.z + l.z;
    v[3] = h.w + l.w;
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = y0 + i < n ? a[y0 + i] + b[y0 + i] : -kInf;
  }
}

// one CTA per kEnvCols columns: each warp finds the maxima of 4 columns, then
// every thread folds its points' normalised values into the envelope.  A
// column's operand starts at a multiple of 32 points, so a thread reads four
// consecutive points with one 16-byte load of each of hh and hl.
__global__ void __launch_bounds__(256) sk_envelope_kernel(SkArgs A) {
  __shared__ float s_m[kEnvCols];
  __shared__ int64_t s_off[kEnvCols];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c0 = blockIdx.x * kEnvCols, nc = min(kEnvCols, A.ncols - c0);
  if (blockIdx.x == 0 && threadIdx.x == 0) *A.fix_count = 0;  // the previous fix-up is done
  for (int k = warp; k < kEnvCols; k += 8) {
    float m = -kInf;
    int64_t off = 0;
    if (k < nc) {
      const SkCol col = A.cols[c0 + k];
      off = col.h_off;
      if (col_active(A, col))
#pragma unroll 4
        for (int y0 = 4 * lane; y0 < A.ny; y0 += 4 * 32) {  // unrolled: several loads in flight
          float v[4];
          load_sum4(A.hh + off, A.hl + off, y0, A.ny, v);
          m = fmaxf(m, fmaxf(fmaxf(v[0], v[1]), fmaxf(v[2], v[3])));
        }
    }
    m = warp_max(m);
    if (lane == 0) {
      const float mq = m > -kInf ? quant(m) : -kInf;
      s_m[k] = mq;
      s_off[k] = off;
      if (k < nc) A.cmax[c0 + k] = mq;
    }
  }
  __syncthreads();
  for (int y0 = 4 * (int)threadIdx.x; y0 < A.ny; y0 += 4 * 256) {
    float e[4] = {-kInf, -kInf, -kInf, -kInf};
#pragma unroll 8
    for (int k = 0; k < nc; ++k) {  // unrolled: the columns' loads are independent
      if (!(s_m[k] > -kInf)) continue;
      const float* hh = A.hh + s_off[k];
      const float* hl = A.hl + s_off[k];
      if (y0 + 4 <= A.ny) {
        const float4 h = *reinterpret_cast<const float4*>(hh + y0);
        const float4 l = *reinterpret_cast<const float4*>(hl + y0);
        e[0] = fmaxf(e[0], (h.x - s_m[k]) + l.x);
        e[1] = fmaxf(e[1], (h.y - s_m[k]) + l.y);
        e[2] = fmaxf(e[2], (h.z - s_m[k]) + l.z);
        e[3] = fmaxf(e[3], (h.w - s_m[k]) + l.w);
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (y0 + i < A.ny) e[i] = fmaxf(e[i], (hh[y0 + i] - s_m[k]) + hl[y0 + i]);
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (y0 + i < A.ny) atomic_max_float(&A.b[y0 + i], e[i]);
  }
}

// Supports of at most 1024 points: one pass over the operands.  Thread t owns
// the points 4t .. 4t+3; columns come kEnvBatch at a time, their values are
// loaded once into registers, the batch's maxima are reduced across the CTA and
// the normalised values folded into the thread's envelope (the two-pass kernel
// above reads every operand twice, the second time mostly from DRAM again).
constexpr int kEnvBatch = 8;
__global__ void __launch_bounds__(256) sk_envelope1_kernel(SkArgs A) {
  __shared__ float s_part[8][kEnvBatch];
  __shared__ float s_m[kEnvBatch];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c0 = blockIdx.x * kEnvCols, nc = min(kEnvCols, A.ncols - c0);
  if (blockIdx.x == 0 && threadIdx.x == 0) *A.fix_count = 0;  // the previous fix-up is done
  const int y0 = 4 * (int)threadIdx.x;
  float e[4] = {-kInf, -kInf, -kInf, -kInf};
  for (int kb = 0; kb < nc; kb += kEnvBatch) {
    float v[kEnvBatch][4];
    float m[kEnvBatch];
#pragma unroll
    for (int i = 0; i < kEnvBatch; ++i) {
      const int k = kb + i;
      bool on = false;
      int64_t off = 0;
      if (k < nc) {
        const SkCol col = A.cols[c0 + k];
        on = col_active(A, col);
        off = col.h_off;
      }
      if (on && y0 < A.ny) {
        load_sum4(A.hh + off, A.hl + off, y0, A.ny, v[i]);
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) v[i][q] = -kInf;
      }
      m[i] = fmaxf(fmaxf(v[i][0], v[i][1]), fmaxf(v[i][2], v[i][3]));
    }
#pragma unroll
    for (int i = 0; i < kEnvBatch; ++i) m[i] = warp_max(m[i]);
    if (lane == 0)
#pragma unroll
      for (int i = 0; i < kEnvBatch; ++i) s_part[warp][i] = m[i];
    __syncthreads();
    if (threadIdx.x < kEnvBatch) {
      float mm = s_part[0][threadIdx.x];
#pragma unroll
      for (int w = 1; w < 8; ++w) mm = fmaxf(mm, s_part[w][threadIdx.x]);
      const float mq = mm > -kInf ? quant(mm) : -kInf;
      s_m[threadIdx.x] = mq;
      if (kb + (int)threadIdx.x < nc) A.cmax[c0 + kb + threadIdx.x] = mq;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kEnvBatch; ++i) {
      const float M = s_m[i];
      if (M > -kInf)
#pragma unroll
        for (int q = 0; q < 4; ++q) e[q] = fmaxf(e[q], v[i][q] - M);
    }
  }
  // this CTA's envelope (the reduction over CTAs follows in sk_envelope_reduce_kernel:
  // atomics here would meet ~500 times on every point and serialise)
  float* const part = A.benv + (int64_t)blockIdx.x * A.kd;
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (y0 + q < A.ny) part[y0 + q] = e[q];
}

// b(y) = the largest of the one-pass kernel's per-CTA envelopes: 32 points per
// CTA, its eight warps taking every eighth CTA's row
__global__ void __launch_bounds__(256) sk_envelope_reduce_kernel(SkArgs A, int32_t nblk) {
  __shared__ float s_m[8][33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int y = blockIdx.x * 32 + lane;
  float m = -kInf;
  if (y < A.ny) {
#pragma unroll 4
    for (int p = warp; p < nblk; p += 8) m = fmaxf(m, A.benv[(int64_t)p * A.kd + y]);
  }
  s_m[warp][lane] = m;
  __syncthreads();
  if (warp == 0 && y < A.ny) {
#pragma unroll
    for (int w = 1; w < 8; ++w) m = fmaxf(m, s_m[w][lane]);
    A.b[y] = m;
  }
}

__device__ __forceinline__ float sqdist(const float* p, const float* q, int dim) {
  float c = 0.f;
  for (int d = 0; d < dim; ++d) {
    const float t = p[d] - q[d];
    c = fmaf(t, t, c);
  }
  return c;
}

__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(v);
  lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// four BF16 (hi, lo) splits of consecutive values, packed for one 8-byte store each
__device__ __forceinline__ void store_split4(const float* v, __nv_bfloat16* hi, __nv_bfloat16* lo) {
  __align__(8) __nv_bfloat16 h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) split_bf16(v[i], h[i], l[i]);
  *reinterpret_cast<uint2*>(hi) = *reinterpret_cast<const uint2*>(h);
  *reinterpret_cast<uint2*>(lo) = *reinterpret_cast<const uint2*>(l);
}

// one CTA per row x, four consecutive columns y per thread and pass (kd is a
// multiple of kSkPadK); rows past nx and columns past ny are zero
__device__ __forceinline__ void sk_kbuild_row(const SkArgs& A, int x) {
  __shared__ float s_red[8];
  __nv_bfloat16* khi = A.khi + (int64_t)x * A.kd;
  __nv_bfloat16* klo = A.klo + (int64_t)x * A.kd;
  if (x >= A.nx) {
    const float z[4] = {0.f, 0.f, 0.f, 0.f};
    for (int y0 = 4 * (int)threadIdx.x; y0 < A.kd; y0 += 4 * 256) store_split4(z, khi + y0, klo + y0);
    if (threadIdx.x == 0) A.rf[x] = 0.f;
    return;
  }
  float p[3] = {0.f, 0.f, 0.f};
  for (int d = 0; d < A.dim; ++d) p[d] = A.xc[(int64_t)x * A.dim + d];
  float env = -kInf;
  for (int y = threadIdx.x; y < A.ny; y += 256)
    env = fmaxf(env, fmaf(-sqdist(p, A.yc + (int64_t)y * A.dim, A.dim), A.s_hi, quant(A.b[y])));
  env = warp_max(env);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = env;
  __syncthreads();
  env = s_red[0];
#pragma unroll
  for (int w = 1; w < 8; ++w) env = fmaxf(env, s_red[w]);
  const float R = env > -kInf ? quant(env) : 0.f;
  if (threadIdx.x == 0) A.rf[x] = R;
  for (int y0 = 4 * (int)threadIdx.x; y0 < A.kd; y0 += 4 * 256) {
    float v[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int y = y0 + i;
      v[i] = 0.f;
      if (y < A.ny && env > -kInf) {
        const float c = sqdist(p, A.yc + (int64_t)y * A.dim, A.dim);
        float t = fmaf(-c, A.s_hi, quant(A.b[y]) - R);
        t = fmaf(-c, A.s_lo, t);
        v[i] = ex2(t);
      }
    }
    store_split4(v, khi + y0, klo + y0);
  }
}

// one warp per column (eight per CTA), four consecutive points per lane and pass
// (the operand's offset is a multiple of 32 points, kd of kSkPadK); inactive
// columns are left alone (their outputs are not stored)
__device__ __forceinline__ void sk_vbuild_cols(const SkArgs& A, int blk) {
  const int lane = threadIdx.x & 31;
  const int j = blk * 8 + (threadIdx.x >> 5);
  if (j >= A.ncols) return;
  const SkCol col = A.cols[j];
  const float M = A.cmax[j];
  if (!col_active(A, col) || !(M > -kInf)) return;
  __nv_bfloat16* vhi = A.vhi + (int64_t)j * A.kd;
  __nv_bfloat16* vlo = A.vlo + (int64_t)j * A.kd;
  const float* hh = A.hh + col.h_off;
  const float* hl = A.hl + col.h_off;
#pragma unroll 4
  for (int y0 = 4 * lane; y0 < A.kd; y0 += 4 * 32) {
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (y0 + 4 <= A.ny) {
      const float4 h4 = *reinterpret_cast<const float4*>(hh + y0);
      const float4 l4 = *reinterpret_cast<const float4*>(hl + y0);
      const float4 b4 = *reinterpret_cast<const float4*>(A.b + y0);
      const float hv[4] = {h4.x, h4.y, h4.z, h4.w}, lv[4] = {l4.x, l4.y, l4.z, l4.w};
      const float bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (hv[i] > -kInf) v[i] = ex2(((hv[i] - M) - quant(bv[i])) + lv[i]);
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int y = y0 + i;
        if (y < A.ny && hh[y] > -kInf) v[i] = ex2(((hh[y] - M) - quant(A.b[y])) + hl[y]);
      }
    }
    store_split4(v, vhi + y0, vlo + y0);
  }
}

// both operand builds in one launch (they read the same envelope and nothing
// of each other): CTAs [0, mp) build rows of K', the rest columns of V'
__global__ void __launch_bounds__(256) sk_kvbuild_kernel(SkArgs A) {
  if ((int)blockIdx.x < A.mp)  // block-uniform
    sk_kbuild_row(A, blockIdx.x);
  else
    sk_vbuild_cols(A, (int)blockIdx.x - A.mp);
}

// ---------------------------------------------------------------------------
// the product: CTA tile 128 rows x 128 columns, 8 warps of 32 x 64, k-stages of
// 32 in a double-buffered cp.async pipeline, fragments by ldmatrix
// ---------------------------------------------------------------------------

constexpr int kSkThreads = 256;
constexpr int kSkLd = kSkTileK + 8;                    // row stride in shared memory (80 bytes)
constexpr int kSkMat = kSkTileM * kSkLd;               // one operand tile (TileM == TileN)
constexpr int kSkStage = 4 * kSkMat;                   // khi, klo, vhi, vlo
constexpr size_t kSkSmem = 2 * kSkStage * sizeof(__nv_bfloat16);  // 80 KB
static_assert(kSkTileM == kSkTileN, "operand tiles share one shape");

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem), "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

__device__ __forceinline__ void ldmatrix_x4(uint32_t* r, const void* smem) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(s));
}

// D += A (16x16 bf16, row) * B (16x8 bf16, col), FP32
__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void load_stage(const SkArgs& A, __nv_bfloat16* st, int m0, int n0, int k0) {
  for (int i = threadIdx.x; i < 4 * kSkTileM * (kSkTileK / 8); i += kSkThreads) {
    const int mat = i / (kSkTileM * (kSkTileK / 8));
    const int r = (i / (kSkTileK / 8)) % kSkTileM, ch = i % (kSkTileK / 8);
    __nv_bfloat16* dst = st + mat * kSkMat + r * kSkLd + ch * 8;
    if (mat < 2) {
      const __nv_bfloat16* src = (mat == 0 ? A.khi : A.klo) + (int64_t)(m0 + r) * A.kd + k0 + ch * 8;
      cp_async16(dst, src, true);
    } else {
      const int j = n0 + r;
      const bool valid = j < A.ncols;
      const __nv_bfloat16* src = (mat == 2 ? A.vhi : A.vlo) + (int64_t)(valid ? j : 0) * A.kd + k0 + ch * 8;
      cp_async16(dst, src, valid);
    }
  }
}

__global__ void __launch_bounds__(kSkThreads, 1) sk_gemm_kernel(SkArgs A) {
  extern __shared__ __align__(128) unsigned char sk_smem[];
  __nv_bfloat16* stages = reinterpret_cast<__nv_bfloat16*>(sk_smem);
  __shared__ SkCol s_cols[kSkTileN];
  __shared__ int s_act[kSkTileN];
  __shared__ float s_cm[kSkTileN];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // row tiles vary fastest: the CTAs that share a column tile of V' run together (L2 reuse)
  const int m0 = blockIdx.x * kSkTileM, n0 = blockIdx.y * kSkTileN;
  if (blockIdx.x == 0 && blockIdx.y == 0)  // the envelope is consumed: reset it for the next product
    for (int y = tid; y < A.kd; y += kSkThreads) A.b[y] = -kInf;
  bool any = false;
  if (tid < kSkTileN) {
    const int j = n0 + tid;
    int act = 0;
    if (j < A.ncols) {
      s_cols[tid] = A.cols[j];
      s_cm[tid] = A.cmax[j];
      act = col_active(A, s_cols[tid]) ? 1 : 0;  // (M = -inf: every term is zero)
    }
    s_act[tid] = act;
    any = act != 0;
  }
  if (!__syncthreads_or(any)) return;

  const int wm = (warp & 3) * 32, wn = (warp >> 2) * 64;
  float acc[2][8][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;

  const int nk = A.kd / kSkTileK;
  load_stage(A, stages, m0, n0, 0);
  cp_async_commit();
  for (int kt = 0; kt < nk; ++kt) {
    if (kt + 1 < nk) load_stage(A, stages + ((kt + 1) & 1) * kSkStage, m0, n0, (kt + 1) * kSkTileK);
    cp_async_commit();
    cp_async_wait1();
    __syncthreads();
    const __nv_bfloat16* st = stages + (kt & 1) * kSkStage;
    const __nv_bfloat16* sAh = st;
    const __nv_bfloat16* sAl = st + kSkMat;
    const __nv_bfloat16* sBh = st + 2 * kSkMat;
    const __nv_bfloat16* sBl = st + 3 * kSkMat;
#pragma unroll
    for (int ks = 0; ks < kSkTileK; ks += 16) {
      uint32_t ah[2][4], al[2][4];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int off = (wm + 16 * i + (lane & 15)) * kSkLd + ks + (lane >> 4) * 8;
        ldmatrix_x4(ah[i], sAh + off);
        ldmatrix_x4(al[i], sAl + off);
      }
#pragma unroll
      for (int jj = 0; jj < 8; jj += 2) {
        uint32_t bh[4], bl[4];
        const int off = (wn + 8 * jj + (lane & 7) + ((lane >> 4) << 3)) * kSkLd + ks + ((lane >> 3) & 1) * 8;
        ldmatrix_x4(bh, sBh + off);
        ldmatrix_x4(bl, sBl + off);
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          mma_bf16(acc[i][jj], ah[i], bh);
          mma_bf16(acc[i][jj], ah[i], bl);
          mma_bf16(acc[i][jj], al[i], bh);
          mma_bf16(acc[i][jj + 1], ah[i], bh + 2);
          mma_bf16(acc[i][jj + 1], ah[i], bl + 2);
          mma_bf16(acc[i][jj + 1], al[i], bh + 2);
        }
      }
    }
    __syncthreads();  // this stage is refilled by the next iteration's loads
  }

  // epilogue: the sum S(x,j) (the node update adds the frame R(x) + M_j)
  const int gid = lane >> 2, tig = lane & 3;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int x = m0 + wm + 16 * i + gid + (r >= 2 ? 8 : 0);
        const int cl = wn + 8 * j + 2 * tig + (r & 1);
        if (x >= A.nx || !s_act[cl]) continue;
        float* const so = A.sout + (int64_t)(n0 + cl) * A.ldo;
        if (!(s_cm[cl] > -kInf)) {  // an empty column (V' not built): no message
          so[x] = 0.f;
          continue;
        }
        const float S = acc[i][j][r];
        if (!(S >= kSkFixBelow)) {  // (also NaN) recomputed by the fix-up
          const int slot = atomicAdd(A.fix_count, 1);
          A.fix_list[slot] = make_int2(x, n0 + cl);
          so[x] = -1.f;
          continue;
        }
        so[x] = fminf(S, FLT_MAX);
      }
}

// ---------------------------------------------------------------------------
// tcgen05 variant of the product: a persistent, warp-specialised kernel in two
// forms.  One CTA per SM walking 128 x 128 output tiles, or (the default) CTA
// pairs, clusters of two CTAs on two SMs, walking 256 x 256 tiles: the even
// CTA issues cta_group::2 MMAs (M = 256) that read K' rows 0-127 and the first
// half of the tile's V' rows from its own shared memory and K' rows 128-255
// and the second half of V' from its peer's, and accumulate each CTA's 128
// rows in that CTA's tensor memory.  Tiles go round-robin, row tiles fastest
// (so the CTAs working on one column tile of V' at a time share it through
// L2); a last round that would leave most units idle is split into half-width
// tiles.  A stage holds 64 reduction points of K'hi, K'lo, V'hi and V'lo, each
// a 64-wide BF16 box of 128 rows brought by one TMA copy
// (cp.async.bulk.tensor) in the 128-byte-swizzled K-major layout the MMA
// descriptors describe; three 64 KB stages per CTA.
//   warp 0 (one lane): TMA producer -- waits for a stage to be free (empty
//     barrier), posts its transaction count and the four copies (full
//     barrier; the pair's copies all complete on the even CTA's, which the
//     even CTA's producer arms with both CTAs' bytes);
//   warp 1 (one lane, the even CTA's): MMA issuer -- per stage waits for the
//     copies, issues 12 tcgen05.mma (kind::f16: BF16 operands from shared
//     memory, FP32 accumulators in tensor memory: the three split products
//     over four 16-point steps), commits them to the stage's empty barrier
//     (both CTAs' for a pair); after a tile's last stage commits to that
//     accumulator's full barrier;
//   warps 2-9: epilogue -- read a finished accumulator with tcgen05.ld (each
//     warp its 32-lane quarter of tensor memory, warp % 4, one output row per
//     thread, and one half of the tile's columns), write the sums, release
//     the accumulator (the even CTA's empty barrier, one arrival per warp of
//     either CTA).
// Two accumulators let the epilogue of one tile run under the MMAs of the
// next, and the producer runs up to three stages ahead across tile
// boundaries.  The epilogue writes one float per output, the sum S (the node
// update adds the frame R(x) + M_j), through per-warp staging buffers and TMA
// stores.  On 2000 stars (n = 1024): one CTA per tile, 90 us; pairs with
// 128-column tiles, 91 us; pairs with 256-column tiles, 87 us, and 81 us with
// the last round split.  Tiles whose columns are all inactive are skipped by
// every role alike (the same test on the same data).  Every wait is bounded;
// a wait that runs out sets bit 1 of the error word and stops its CTA's
// roles (the peer's waits then run out too); before tensor memory is
// released the MMA issuer waits (bounded) for its last commit and the
// producers for every copy they issued, and a pair's CTAs meet at a cluster
// barrier so neither leaves while the other may still touch its memory.
// ---------------------------------------------------------------------------
constexpr int kTcEpiWarps = 8;                        // two per tensor-memory lane quarter (4 or 8)
constexpr int kTcThreads = 64 + 32 * kTcEpiWarps;     // producer, MMA, epilogue warps
constexpr int kTcK = 64;                              // reduction points per stage: 64 (128-byte rows,
                                                      // 128-byte swizzle) or 32 (64-byte rows and swizzle)
constexpr int kTcN = 128;                             // output columns per tile of one CTA (MMA N: 128 or 256)
constexpr int kTcN2 = 256;                            // output columns per tile of a CTA pair (128 or 256)
constexpr int kTcRowBytes = kTcK * 2;                 // one operand row of a stage (the swizzle span)
constexpr int kTcTileBytes = kSkTileM * kTcRowBytes;  // one K' part (128 rows)
constexpr int kTcAcc = 2;                             // accumulators in tensor memory
constexpr int kTcMaxTiles = 512;                      // tiles one CTA may own (the grid grows beyond)
constexpr int kTcStgCols = 16;                                // columns per TMA store of the epilogue
constexpr int kTcStgBytes = 32 * kTcStgCols * 4;              // one epilogue warp's staging buffer
constexpr uint64_t kTcWaitNs = 250ull * 1000 * 1000;  // a wait gives up after 250 ms
static_assert(kSkTileM == 128 && (kTcN == 128 || kTcN == 256) && (kTcN2 == 128 || kTcN2 == 256) &&
                  (kTcK == 64 || kTcK == 32) && kSkPadK % kTcK == 0,
              "tcgen05 tile 128 x N x 32 or 64");

// shapes of the product over kCta CTAs (1, or 2: a CTA pair of one cluster whose
// MMAs, issued by the even CTA, span 256 rows: each CTA holds its 128 rows of K'
// and half of the tile's V' rows, and its 128 rows of the accumulator)
template <int kCta>
struct TcCfg {
  static constexpr int kN = kCta == 1 ? kTcN : kTcN2;   // output columns per tile (MMA N)
  static constexpr int kBRows = kN / kCta;              // V' rows (output columns) one CTA loads
  static constexpr int kBBytes = kBRows * kTcRowBytes;  // one V' part of a stage
  static constexpr int kStageBytes = 2 * kTcTileBytes + 2 * kBBytes;
  static constexpr int kStages = std::min(8, (200 * 1024) / kStageBytes);  // as many as shared memory holds
  static constexpr size_t kSmem = kStages * kStageBytes + kTcEpiWarps * kTcStgBytes + 1024;  // + alignment slack
  static constexpr int kRows = kSkTileM * kCta;         // rows of one tile (MMA M)
  static constexpr uint32_t kCols = kTcAcc * kN;       // tensor memory columns (per CTA)
  // instruction descriptor: D FP32, A and B BF16, both K-major, M = kRows, N = w (kN or kN / 2)
  __host__ __device__ static constexpr uint32_t idesc(int w) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(w >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);
  }
  static_assert(kCta == 1 || kCta == 2, "one CTA or a CTA pair");
  static_assert(kSmem + 8 * 1024 <= 227 * 1024, "stages, staging and static tables fit in shared memory");
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// the shared::cluster address of the same shared variable in CTA `rank` of this cluster
__device__ __forceinline__ uint32_t peer_addr(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}

// every thread of both CTAs of the cluster
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// shared-memory matrix descriptor of a K-major tile swizzled over its row span
// (128 or 64 bytes: layout codes 2 and 4), 8-row groups 8 rows apart
__device__ __forceinline__ uint64_t sw_desc(uint32_t saddr) {
  constexpr uint64_t layout = kTcRowBytes == 128 ? 2 : 4;
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)((8 * kTcRowBytes) >> 4) << 32) |
         ((uint64_t)1 << 46) | (layout << 61);
}

template <int kCta>
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if constexpr (kCta == 1)
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  else
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tc_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// one 2-D box (x = reduction index, y = row) into this CTA's shared memory; the
// completion goes to the mbarrier at shared::cluster address `bar`, in this CTA
// (kCta 1) or in either CTA of the pair (kCta 2)
template <int kCta>
__device__ __forceinline__ void tma_box(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  if constexpr (kCta == 1)
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
  else
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
        "%3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// bounded wait on an mbarrier phase: kTcWaitNs of wall time, 2^24 polls at most
// (the pair product's barriers see arrivals from the peer CTA: cluster-scope acquire)
template <int kCta = 1>
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t addr = smem_u32(bar);
  uint64_t start = 0;
  for (uint32_t i = 0; i < (1u << 24); ++i) {
    uint32_t ok;
    if constexpr (kCta == 1)
      asm volatile(
          "{\n\t.reg .pred p;\n\t"
          "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
          "selp.u32 %0, 1, 0, p;\n\t}"
          : "=r"(ok)
          : "r"(addr), "r"(parity)
          : "memory");
    else
      asm volatile(
          "{\n\t.reg .pred p;\n\t"
          "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
          "selp.u32 %0, 1, 0, p;\n\t}"
          : "=r"(ok)
          : "r"(addr), "r"(parity)
          : "memory");
    if (ok) return true;
    if ((i & 63) == 63) {
      uint64_t now;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
      if (start == 0)
        start = now;
      else if (now - start > kTcWaitNs)
        return false;
      __nanosleep(256);
    }
  }
  return false;
}

// whether any column of the column tile [n0, n0 + w) takes part in this product
__device__ __forceinline__ bool tc_tile_active(const SkArgs& A, int n0, int w) {
  for (int c = 0; c < w; ++c) {
    const int j = n0 + c;
    if (j >= A.ncols) break;
    if (col_active(A, A.cols[j])) return true;  // (an empty column still gets S = 0 written)
  }
  return false;
}

__device__ __forceinline__ void tc_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// one arrival on the mbarrier at shared::cluster address `bar` (this CTA's or the peer's)
__device__ __forceinline__ void tc_arrive_cluster(uint32_t bar) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar) : "memory");
}

// arrive on `bar` once every tcgen05.mma issued before has completed; for the
// pair, on the barrier at the same offset in both CTAs
template <int kCta>
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  if constexpr (kCta == 1)
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
  else
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            smem_u32(bar)),
        "h"((uint16_t)3)
        : "memory");
}

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"n"(32 * kTcEpiWarps) : "memory"); }

// kCta 1: one CTA per SM, 128 x kTcN tiles.  kCta 2: launched in clusters of two;
// a pair owns 256 x kTcN2 tiles, the even CTA issues the MMAs (M = 256) over both
// CTAs' stages, their copies complete on its full barriers (the odd CTA's through
// the cta_group::2 form of the copy), its commits arrive on both CTAs' barriers,
// and both CTAs' epilogue warps release an accumulator on its empty barrier.
template <int kCta>
__global__ void __launch_bounds__(kTcThreads, 1)
    sk_gemm_tc_kernel(const __grid_constant__ SkArgs A, const __grid_constant__ CUtensorMap tkhi,
                      const __grid_constant__ CUtensorMap tklo, const __grid_constant__ CUtensorMap tvhi,
                      const __grid_constant__ CUtensorMap tvlo, const __grid_constant__ CUtensorMap tout) {
  using Cfg = TcCfg<kCta>;
  constexpr int kStages = Cfg::kStages, kStageBytes = Cfg::kStageBytes, kBBytes = Cfg::kBBytes;
  extern __shared__ __align__(16) unsigned char tc_raw[];
  constexpr int kN = Cfg::kN;
  __shared__ int64_t s_off[kN];  // the tile's columns: offset of their sums in sout (-1: inactive)
  __shared__ float s_cm[kN];     // and column maximum (-inf: an empty column, S = 0)
  __shared__ __align__(8) uint64_t s_full[kStages], s_empty[kStages], s_afull[kTcAcc], s_aempty[kTcAcc];
  __shared__ uint32_t s_tmem;
  __shared__ int2 s_tiles[kTcMaxTiles];  // this CTA's (pair's) active tiles, in order: (row tile, 2 n0 + whole)
  __shared__ int s_ntiles;
  __shared__ volatile int s_abort;
  __shared__ int s_epi_ok;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t rank = kCta == 1 ? 0u : cluster_rank();  // this CTA's half of a pair tile
  const int unit = (int)blockIdx.x / kCta, nunits = (int)gridDim.x / kCta;
  const int mt = (A.mp + Cfg::kRows - 1) / Cfg::kRows;          // row tiles
  const int ntiles = mt * ((A.ncols + kN - 1) / kN);
  if (blockIdx.x == 0)  // the envelope is consumed: reset it for the next product
    for (int y = tid; y < A.kd; y += kTcThreads) A.b[y] = -kInf;
  // this CTA's (pair's) tiles, the inactive ones left out; both CTAs of a pair build the
  // same list.  Tiles t (row tiles fastest) go round-robin (t = unit + i nunits) in
  // whole rounds; the last, partial round's tiles are split into two kN / 2 column
  // halves, dealt round-robin as well, when the halves fit one round
  if (tid == 0) {
    const int rounds = ntiles / nunits, left = ntiles - rounds * nunits;
    const bool split = left > 0 && 2 * left <= nunits;
    const int whole = split ? rounds * nunits : ntiles;
    int n = 0;
    for (int t = unit; t < whole && n < kTcMaxTiles; t += nunits) {
      const int n0 = (t / mt) * kN;
      if (tc_tile_active(A, n0, kN)) s_tiles[n++] = make_int2(t % mt, 2 * n0 + 1);
    }
    for (int h = unit; split && h < 2 * left && n < kTcMaxTiles; h += nunits) {
      const int t = whole + h / 2;
      const int n0 = (t / mt) * kN + (h & 1) * (kN / 2);
      if (n0 < A.ncols && tc_tile_active(A, n0, kN / 2)) s_tiles[n++] = make_int2(t % mt, 2 * n0);
    }
    s_ntiles = n;
    s_abort = 0;
  }
  __syncthreads();
  const int nt = s_ntiles;
  if (nt == 0) return;  // uniform across the block and the pair

  // stages on a 1024-byte boundary (the swizzle pattern follows the address bits)
  const uint32_t raw = smem_u32(tc_raw);
  const uint32_t stage0 = (raw + 1023u) & ~1023u;
  if (tid == 0) {
    for (int i = 0; i < kStages; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_full[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_empty[i])));
    }
    for (int i = 0; i < kTcAcc; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_afull[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&s_aempty[i])), "n"(kCta * kTcEpiWarps));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    if constexpr (kCta == 1) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                   "r"(Cfg::kCols));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    } else {
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                   "r"(Cfg::kCols));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if constexpr (kCta == 2) cluster_sync();  // both CTAs' barriers and tensor memory exist
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  const int nk = A.kd / kTcK;

  if (warp == 0) {
    // ---- TMA producer (each CTA its own stages) ----
    if (lane == 0) {
      int g = 0;  // stage uses so far, across tiles
      bool ok = true;
      for (int i = 0; i < nt && ok; ++i) {
        const int2 t = s_tiles[i];
        const int w = (t.y & 1) ? kN : kN / 2;  // the tile's columns (a V' box holds kBRows rows:
                                                 // a half tile leaves the box's far half unused)
        const int m0 = t.x * Cfg::kRows + (int)rank * kSkTileM;
        const int n0 = (t.y >> 1) + (int)rank * (w / kCta);
        for (int kt = 0; kt < nk; ++kt, ++g) {
          const int b = g % kStages;
          if (g >= kStages && !tc_wait<kCta>(&s_empty[b], ((g / kStages) - 1) & 1)) {
            ok = false;
            break;
          }
          if (s_abort) {
            ok = false;
            break;
          }
          const uint32_t dst = stage0 + b * kStageBytes;
          // the pair's copies complete on the even CTA's full barrier, which expects both halves
          const uint32_t full = kCta == 1 ? smem_u32(&s_full[b]) : peer_addr(smem_u32(&s_full[b]), 0);
          if (rank == 0) tc_expect(&s_full[b], kCta * kStageBytes);
          tma_box<kCta>(dst, &tkhi, kt * kTcK, m0, full);
          tma_box<kCta>(dst + kTcTileBytes, &tklo, kt * kTcK, m0, full);
          tma_box<kCta>(dst + 2 * kTcTileBytes, &tvhi, kt * kTcK, n0, full);
          tma_box<kCta>(dst + 2 * kTcTileBytes + kBBytes, &tvlo, kt * kTcK, n0, full);
        }
      }
      if (!ok) {
        s_abort = 1;
        atomicOr(A.err, 2);
      }
      // every copy issued lands before the CTA may leave (bounded): the even CTA sees
      // them on its full barriers; the odd CTA through the empty barriers, which the
      // MMAs that read its copies release
      for (int q = (g > kStages ? g - kStages : 0); q < g; ++q) {
        if (rank == 0)
          (void)tc_wait<kCta>(&s_full[q % kStages], (q / kStages) & 1);
        else
          (void)tc_wait<kCta>(&s_empty[q % kStages], (q / kStages) & 1);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---- MMA issuer (the even CTA of a pair) ----
    if (lane == 0 && rank == 0) {
      int g = 0;
      bool ok = true;
      int last_acc = -1, last_use = 0;
      for (int i = 0; i < nt && ok; ++i) {
        const int a = i % kTcAcc;
        if (i >= kTcAcc && !tc_wait<kCta>(&s_aempty[a], ((i / kTcAcc) - 1) & 1)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + (uint32_t)(a * kN);
        const uint32_t idesc = Cfg::idesc((s_tiles[i].y & 1) ? kN : kN / 2);
        for (int kt = 0; kt < nk; ++kt, ++g) {
          const int b = g % kStages;
          if (!tc_wait<kCta>(&s_full[b], (g / kStages) & 1) || s_abort) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t sa = stage0 + b * kStageBytes;
          const uint64_t ah = sw_desc(sa), al = sw_desc(sa + kTcTileBytes);
          const uint64_t bh = sw_desc(sa + 2 * kTcTileBytes), bl = sw_desc(sa + 2 * kTcTileBytes + kBBytes);
          for (int k = 0; k < kTcK / 16; ++k) {
            const uint64_t dk = (uint64_t)((k * 32) >> 4);  // 16 BF16 further along K
            tc_mma<kCta>(d, ah + dk, bh + dk, idesc, (kt | k) != 0 ? 1u : 0u);
            tc_mma<kCta>(d, ah + dk, bl + dk, idesc, 1u);
            tc_mma<kCta>(d, al + dk, bh + dk, idesc, 1u);
          }
          tc_commit<kCta>(&s_empty[b]);  // the stage's buffers are free once these MMAs have read them
        }
        if (!ok) break;
        tc_commit<kCta>(&s_afull[a]);  // the tile's accumulator is complete once every MMA before it is
        last_acc = a;
        last_use = i / kTcAcc;
      }
      if (!ok) {
        s_abort = 1;
        atomicOr(A.err, 2);
      }
      // the last commit covers every MMA issued before it: wait for it before tensor memory goes
      if (last_acc >= 0) (void)tc_wait<kCta>(&s_afull[last_acc], last_use & 1);
      if (g > 0) (void)tc_wait<kCta>(&s_empty[(g - 1) % kStages], ((g - 1) / kStages) & 1);
    }
    __syncwarp();
  } else {
    // ---- epilogue: warps 2..9, tensor-memory lane quarter warp % 4, column half (warp - 2) / 4 ----
    const int et = tid - 64;  // 0 .. 32 kTcEpiWarps - 1 within the epilogue group
    const int quarter = warp & 3;
    float* const stg = reinterpret_cast<float*>(tc_raw + (stage0 - raw) + kStages * kStageBytes +
                                                (warp - 2) * kTcStgBytes);
    const uint32_t stg_s = smem_u32(stg);
    static_assert(kTcEpiWarps == 8 && kN / 4 >= 32, "two column halves of at least 32 columns");
    for (int i = 0; i < nt; ++i) {
      const int a = i % kTcAcc;
      const int2 t = s_tiles[i];
      const int w = (t.y & 1) ? kN : kN / 2;
      const int span = w / 2;                          // columns per warp
      const int c_beg = ((warp - 2) >> 2) * span;
      const int m0 = t.x * Cfg::kRows + (int)rank * kSkTileM, n0 = t.y >> 1;
      epi_sync();  // the previous tile's column table is no longer read
      for (int c = et; c < w; c += 32 * kTcEpiWarps) {  // the tile's column table
        const int j = n0 + c;
        float cm = -kInf;
        int64_t off = -1;
        if (j < A.ncols && col_active(A, A.cols[j])) {
          cm = A.cmax[j];
          off = (int64_t)j * A.ldo;
        }
        s_off[c] = off;
        s_cm[c] = cm;
      }
      if (et == 0) s_epi_ok = tc_wait<kCta>(&s_afull[a], (i / kTcAcc) & 1) && !s_abort ? 1 : 0;
      epi_sync();
      if (!s_epi_ok) {
        if (et == 0) {
          s_abort = 1;
          atomicOr(A.err, 2);
        }
        break;  // uniform across the epilogue group
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int x = m0 + quarter * 32 + lane;  // tensor-memory lane = output row
      const bool row_in = x < A.nx;
      float* const sout = A.sout;
      for (int c0 = c_beg; c0 < c_beg + span; c0 += 32) {
        uint32_t v[32];
        const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(a * kN + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
              "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
              "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
              "=r"(v[30]), "=r"(v[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (A.store_tma) {
          // through this warp's staging buffer ([column][32 rows] FP32) and one TMA store
          // per 16 columns; rows past nx and columns past ncols are clipped by the tensor
          // map, inactive columns get values nothing reads
#pragma unroll
          for (int hb = 0; hb < 32; hb += kTcStgCols) {
            if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");  // buffer free again
            __syncwarp();
#pragma unroll
            for (int q = 0; q < kTcStgCols; ++q) {
              const int cl = c0 + hb + q;
              float val = 0.f;  // inactive or empty column
              if (row_in && s_off[cl] >= 0 && s_cm[cl] > -kInf) {
                const float S = __uint_as_float(v[hb + q]);
                if (!(S >= kSkFixBelow)) {  // (also NaN) recomputed by the fix-up
                  const int slot = atomicAdd(A.fix_count, 1);
                  A.fix_list[slot] = make_int2(x, n0 + cl);
                  val = -1.f;
                } else {
                  val = fminf(S, FLT_MAX);
                }
              }
              stg[q * 32 + lane] = val;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the bulk copy
            __syncwarp();
            if (lane == 0 && m0 + quarter * 32 < A.nx && n0 + c0 + hb < A.ncols)  // (a box wholly outside: none)
              asm volatile(
                  "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];\n\t"
                  "cp.async.bulk.commit_group;" ::"l"(reinterpret_cast<uint64_t>(&tout)),
                  "r"(m0 + quarter * 32), "r"(n0 + c0 + hb), "r"(stg_s)
                  : "memory");
          }
          continue;
        }
        if (!row_in) continue;
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          const int cl = c0 + q;
          const int64_t off = s_off[cl];
          if (off < 0) continue;
          if (s_cm[cl] == -kInf) {  // an empty column (V' not built): no message
            sout[off + x] = 0.f;
            continue;
          }
          const float S = __uint_as_float(v[q]);
          if (!(S >= kSkFixBelow)) {  // (also NaN) recomputed by the fix-up
            const int slot = atomicAdd(A.fix_count, 1);
            A.fix_list[slot] = make_int2(x, n0 + cl);
            sout[off + x] = -1.f;
            continue;
          }
          sout[off + x] = fminf(S, FLT_MAX);
        }
      }
      // this warp's reads of the accumulator are done: release it to the MMA issuer
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        if constexpr (kCta == 1)
          tc_arrive(&s_aempty[a]);
        else
          tc_arrive_cluster(peer_addr(smem_u32(&s_aempty[a]), 0));  // the even CTA's
      }
    }
  }
  if (warp >= 2 && lane == 0 && A.store_tma) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  // the pair: neither CTA leaves (nor frees tensor memory) while the other may still
  // touch its barriers, stages or tensor memory
  if constexpr (kCta == 2) cluster_sync();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 1) {
    if constexpr (kCta == 1)
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Cfg::kCols));
    else
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Cfg::kCols));
  }
}

// one CTA per listed output (eight warps over the reduction points, so an output
// costs two rounds of loads): frame = the largest term on the 2^-10 grid, then
// the sum of 2^(term - frame) with the recomputed-cost apply's argument
__global__ void __launch_bounds__(256) sk_fixup_kernel(SkArgs A) {
  __shared__ float red[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nfix = *A.fix_count;
  for (int w = blockIdx.x; w < nfix; w += gridDim.x) {  // block-uniform
    const int2 e = A.fix_list[w];
    const int x = e.x;
    const SkCol col = A.cols[e.y];
    const float* hh = A.hh + col.h_off;
    const float* hl = A.hl + col.h_off;
    float p[3] = {0.f, 0.f, 0.f};
    for (int d = 0; d < A.dim; ++d) p[d] = A.xc[(int64_t)x * A.dim + d];
    float mx = -kInf;
#pragma unroll 4
    for (int y = threadIdx.x; y < A.ny; y += 256)
      mx = fmaxf(mx, fmaf(-sqdist(p, A.yc + (int64_t)y * A.dim, A.dim), A.s_hi, hh[y]));
    mx = warp_max(mx);
    __syncthreads();  // red is free (previous output)
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    mx = red[0];
#pragma unroll
    for (int i = 1; i < 8; ++i) mx = fmaxf(mx, red[i]);
    float R = 0.f, S = 0.f;
    if (mx > -kInf) {
      R = quant(mx);
#pragma unroll 4
      for (int y = threadIdx.x; y < A.ny; y += 256) {
        if (!(hh[y] > -kInf)) continue;
        const float c = sqdist(p, A.yc + (int64_t)y * A.dim, A.dim);
        float t = fmaf(-c, A.s_hi, hh[y] - R);
        t = fmaf(-c, A.s_lo, t);
        S += ex2(t + hl[y]);
      }
      S = warp_sum(S);
      __syncthreads();
      if (lane == 0) red[warp] = S;
      __syncthreads();
      S = 0.f;
#pragma unroll
      for (int i = 0; i < 8; ++i) S += red[i];
    }
    if (threadIdx.x == 0) A.part32[col.part_off + x] = make_float2(R, S);
  }
}

__global__ void sk_reset_kernel(float* b, int32_t kd) {
  for (int y = blockIdx.x * blockDim.x + threadIdx.x; y < kd; y += gridDim.x * blockDim.x) b[y] = -kInf;
}

// dynamic shared memory above 48 KB is a per-device function attribute
bool sk_gemm_ready() {
  constexpr int kMaxDevices = 64;
  static std::atomic<int> state[kMaxDevices];  // 0 unknown, 1 set, 2 refused
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return false;
  int st = state[dev].load();
  if (st == 0) {
    st = cudaFuncSetAttribute(sk_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSkSmem) ==
                 cudaSuccess
             ? 1
             : 2;
    state[dev].store(st);
  }
  return st == 1;
}

// resident units of the tcgen05 product on the current device: CTAs (kCta 1) or
// CTA pairs (kCta 2, clusters of two); 0 when it cannot run
template <int kCta>
int sk_tc_units() {
  constexpr int kMaxDevices = 64;
  static std::atomic<int> state[kMaxDevices];  // 0 unknown, else units + 1
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 0;
  int st = state[dev].load();
  if (st == 0) {
    const auto kern = sk_gemm_tc_kernel<kCta>;
    constexpr size_t smem = TcCfg<kCta>::kSmem;
    int units = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess) {
      if constexpr (kCta == 1) {
        int blocks = 0, sms = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, kTcThreads, smem) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
          units = blocks >= 1 ? sms : 0;  // one CTA per SM
      } else {
        cudaLaunchConfig_t cfg{};
        cudaLaunchAttribute attr{};
        attr.id = cudaLaunchAttributeClusterDimension;
        attr.val.clusterDim.x = 2;
        attr.val.clusterDim.y = 1;
        attr.val.clusterDim.z = 1;
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cfg.gridDim = dim3((unsigned)std::max(2, sms & ~1));
        cfg.blockDim = dim3(kTcThreads);
        cfg.dynamicSmemBytes = smem;
        cfg.attrs = &attr;
        cfg.numAttrs = 1;
        int clusters = 0;
        if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) == cudaSuccess) units = clusters;
      }
    }
    cudaGetLastError();  // (a refused query leaves no error behind)
    st = units + 1;
    state[dev].store(st);
  }
  return st - 1;
}

bool sk_tc_ready(int pair) { return pair ? sk_tc_units<2>() > 0 : sk_tc_units<1>() > 0; }

}  // namespace

bool sk_tc_available() { return sk_tc_ready(0); }

bool sk_tc_pair_available() { return sk_tc_ready(1); }

bool sk_encode_maps(const SkArgs& a, SkMaps* m) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  static std::atomic<int> state{0};  // 0 unknown, 1 found, 2 not
  if (state.load() == 0) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    const bool ok = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                        cudaSuccess &&
                    q == cudaDriverEntryPointSuccess && fn != nullptr;
    if (ok) encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    state.store(ok ? 1 : 2);
  }
  if (state.load() != 1 || a.ncols <= 0) return false;
  auto make = [&](CUtensorMap* map, const void* base, int64_t rows, int box_rows) {
    const cuuint64_t dims[2] = {(cuuint64_t)a.kd, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)a.kd * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kTcK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, kTcRowBytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  };
  if (!(make(&m->khi, a.khi, a.mp, kSkTileM) && make(&m->klo, a.klo, a.mp, kSkTileM) &&
        make(&m->vhi, a.vhi, a.ncols, a.tc_pair ? TcCfg<2>::kBRows : TcCfg<1>::kBRows) &&
        make(&m->vlo, a.vlo, a.ncols, a.tc_pair ? TcCfg<2>::kBRows : TcCfg<1>::kBRows)))
    return false;
  if (a.store_tma) {  // sums: FP32 [ncols][ldo] (valid x < nx), 32 x 16 boxes, no swizzle
    const cuuint64_t dims[2] = {(cuuint64_t)a.nx, (cuuint64_t)a.ncols};
    const cuuint64_t strides[1] = {(cuuint64_t)a.ldo * 4};
    const cuuint32_t box[2] = {32, (cuuint32_t)kTcStgCols};
    const cuuint32_t estr[2] = {1, 1};
    if (encode(&m->sout, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, a.sout, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  return true;
}

cudaError_t launch_sk(const SkArgs& a, const SkMaps* maps, cudaStream_t s, cudaEvent_t before_product,
                      cudaEvent_t after_product) {
  if (a.ncols <= 0) return cudaSuccess;
  if (a.use_tc && !maps) return cudaErrorInvalidValue;
  if (!(a.use_tc ? sk_tc_ready(a.tc_pair) : sk_gemm_ready())) return cudaErrorInvalidConfiguration;
  const int nenv = (a.ncols + kEnvCols - 1) / kEnvCols;
  if (a.ny <= 4 * 256 && a.benv) {
    sk_envelope1_kernel<<<nenv, 256, 0, s>>>(a);
    sk_envelope_reduce_kernel<<<(a.ny + 31) / 32, 256, 0, s>>>(a, nenv);
  } else {
    sk_envelope_kernel<<<nenv, 256, 0, s>>>(a);
  }
  sk_kvbuild_kernel<<<a.mp + (a.ncols + 7) / 8, 256, 0, s>>>(a);
  if (before_product) cudaEventRecord(before_product, s);
  const dim3 grid(a.mp / kSkTileM, (a.ncols + kSkTileN - 1) / kSkTileN);
  if (a.use_tc && a.tc_pair) {
    // persistent: as many CTA pairs as can be resident (one CTA per SM), more only if
    // a pair would own more tiles than its table holds
    const int mt = (a.mp + 2 * kSkTileM - 1) / (2 * kSkTileM);
    const int ntiles = mt * ((a.ncols + kTcN2 - 1) / kTcN2);
    const int pairs = std::max(std::min(ntiles, sk_tc_units<2>()), (ntiles + kTcMaxTiles - 2) / (kTcMaxTiles - 1));
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr{};
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = 2;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(2 * pairs));
    cfg.blockDim = dim3(kTcThreads);
    cfg.dynamicSmemBytes = TcCfg<2>::kSmem;
    cfg.stream = s;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    const cudaError_t e =
        cudaLaunchKernelEx(&cfg, sk_gemm_tc_kernel<2>, a, maps->khi, maps->klo, maps->vhi, maps->vlo, maps->sout);
    if (e != cudaSuccess) return e;
  } else if (a.use_tc) {
    // persistent: one CTA per SM (shared memory allows no second), more only if a CTA
    // would own more tiles than its table holds
    const int ntiles = (int)grid.x * ((a.ncols + kTcN - 1) / kTcN);
    const int ctas = std::max(std::min(ntiles, sk_tc_units<1>()), (ntiles + kTcMaxTiles - 2) / (kTcMaxTiles - 1));
    sk_gemm_tc_kernel<1><<<ctas, kTcThreads, TcCfg<1>::kSmem, s>>>(a, maps->khi, maps->klo, maps->vhi, maps->vlo,
                                                                     maps->sout);
  } else {
    sk_gemm_kernel<<<grid, kSkThreads, kSkSmem, s>>>(a);
  }
  if (after_product) cudaEventRecord(after_product, s);
  sk_fixup_kernel<<<152 * 8, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_sk_reset(float* b, int32_t kd, cudaStream_t s) {
  if (kd <= 0) return cudaSuccess;
  sk_reset_kernel<<<(kd + 255) / 256, 256, 0, s>>>(b, kd);
  return cudaGetLastError();
}

}  // namespace treeot
