// Warm-start predictor: a 3-layer MLP (in -> hidden -> hidden -> out, GELU
// after the first two layers) with BF16 weights and activations feeding
// tensor-core MMAs (mma.sync m16n8k16, FP32 accumulation), FP32 master
// weights and Adam.  Forward, backward and the optimiser step are all kernels
// of this file; the host side lives in api.cpp (tree_ot_mlp_*).
//
// GEMM convention: C[M,N] = sum_k A(m,k) B(k,n), with A(m,k) read from a
// row-major array either as A[m*lda + k] (plain) or A[k*lda + m] (transposed),
// and the same for B(k,n) = B[k*ldb + n] or B[n*ldb + k].
#include <cuda_bf16.h>

#include <cmath>
#include <cstdint>

#include "internal.h"

namespace treeot {
namespace {

constexpr int kTM = 64, kTN = 64, kTK = 32;  // CTA tile; 4 warps, each 32x32

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// D = A (16x16, bf16, row) * B (16x8, bf16, col) + C, FP32
__device__ __forceinline__ void mma16816(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C (FP32) = A * B (+ bias[n]) ; optional accumulate into C (beta = 1)
__global__ void __launch_bounds__(128) gemm_bf16_kernel(const __nv_bfloat16* A, int lda, int ta,
                                                        const __nv_bfloat16* B, int ldb, int tb, float* C, int ldc,
                                                        int M, int N, int K, const float* bias, int accumulate) {
  __shared__ __nv_bfloat16 As[kTM][kTK + 8];  // As[m][k]
  __shared__ __nv_bfloat16 Bs[kTN][kTK + 8];  // Bs[n][k]
  const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * kTN;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int gid = lane >> 2, tig = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
  const __nv_bfloat16 zero = __float2bfloat16(0.f);
  for (int k0 = 0; k0 < K; k0 += kTK) {
    for (int idx = tid; idx < kTM * kTK; idx += 128) {
      const int mm = idx / kTK, kk = idx % kTK;
      const int m = m0 + mm, k = k0 + kk;
      __nv_bfloat16 v = zero;
      if (m < M && k < K) v = ta ? A[(int64_t)k * lda + m] : A[(int64_t)m * lda + k];
      As[mm][kk] = v;
    }
    for (int idx = tid; idx < kTN * kTK; idx += 128) {
      const int nn = idx / kTK, kk = idx % kTK;
      const int n = n0 + nn, k = k0 + kk;
      __nv_bfloat16 v = zero;
      if (n < N && k < K) v = tb ? B[(int64_t)n * ldb + k] : B[(int64_t)k * ldb + n];
      Bs[nn][kk] = v;
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < kTK; ks += 16) {
      uint32_t af[2][4], bfr[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r0 = wm + 16 * i + gid;
        af[i][0] = pack_bf16(As[r0][ks + 2 * tig], As[r0][ks + 2 * tig + 1]);
        af[i][1] = pack_bf16(As[r0 + 8][ks + 2 * tig], As[r0 + 8][ks + 2 * tig + 1]);
        af[i][2] = pack_bf16(As[r0][ks + 2 * tig + 8], As[r0][ks + 2 * tig + 9]);
        af[i][3] = pack_bf16(As[r0 + 8][ks + 2 * tig + 8], As[r0 + 8][ks + 2 * tig + 9]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = wn + 8 * j + gid;
        bfr[j][0] = pack_bf16(Bs[c][ks + 2 * tig], Bs[c][ks + 2 * tig + 1]);
        bfr[j][1] = pack_bf16(Bs[c][ks + 2 * tig + 8], Bs[c][ks + 2 * tig + 9]);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma16816(acc[i][j], af[i], bfr[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int m = m0 + wm + 16 * i + gid + (r >= 2 ? 8 : 0);
        const int n = n0 + wn + 8 * j + 2 * tig + (r & 1);
        if (m < M && n < N) {
          float v = acc[i][j][r];
          if (bias) v += bias[n];
          float* dst = C + (int64_t)m * ldc + n;
          *dst = accumulate ? *dst + v : v;
        }
      }
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  const float cdf = 0.5f * (1.f + erff(z * 0.70710678118654752f));
  const float pdf = 0.39894228040143268f * expf(-0.5f * z * z);
  return cdf + z * pdf;
}

// a = gelu(z) -> BF16 (next layer input); z kept in FP32 for the backward pass
__global__ void gelu_fwd_kernel(const float* z, __nv_bfloat16* a, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a[i] = __float2bfloat16(gelu(z[i]));
}

// dz = da * gelu'(z), stored as BF16 (operand of the next backward GEMMs) and FP32 (bias gradient)
__global__ void gelu_bwd_kernel(const float* da, const float* z, __nv_bfloat16* dz16, float* dz32, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float g = da[i] * gelu_grad(z[i]);
    dz32[i] = g;
    dz16[i] = __float2bfloat16(g);
  }
}

// first-layer input: the first `nlog` features of every row become
// log(max(x, floor)) * scale (the marginal enters as log-probabilities), the rest pass through
__global__ void input_kernel(const float* x, __nv_bfloat16* y, int64_t rows, int cols, int nlog, float floor_,
                             float scale) {
  const int64_t n = rows * cols;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % cols);
    float v = x[i];
    if (c < nlog) v = logf(fmaxf(v, floor_)) * scale;
    y[i] = __float2bfloat16(v);
  }
}

__global__ void to_bf16_kernel(const float* x, __nv_bfloat16* y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16(x[i]);
}

// loss = mean((y - t)^2); dy = 2 (y - t) / count (FP32 and BF16 copies); loss summed into *loss (FP64)
__global__ void mse_kernel(const float* y, const float* t, float* dy32, __nv_bfloat16* dy16, int64_t n, double* loss) {
  __shared__ double red[8];
  double local = 0.0;
  const float scale = 2.f / (float)n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float d = y[i] - t[i];
    local += (double)d * d;
    const float g = scale * d;
    dy32[i] = g;
    dy16[i] = __float2bfloat16(g);
  }
  for (int o = 16; o; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = local;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    atomicAdd(loss, s / (double)n);
  }
}

// db[n] = sum_m dz[m, n]
__global__ void colsum_kernel(const float* dz, int M, int N, float* db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int m = 0; m < M; ++m) s += dz[(int64_t)m * N + n];
  db[n] = s;
}

// Adam on FP32 master weights, refresh of the BF16 working copy (bias-corrected moments)
__global__ void adam_kernel(float* w, const float* g, float* m1, float* m2, __nv_bfloat16* w16, int64_t n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    const float wi = w[i] - lr * (a / c1) / (sqrtf(b / c2) + eps);
    w[i] = wi;
    if (w16) w16[i] = __float2bfloat16(wi);
  }
}

int blocks_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b > 2048 ? 2048 : (b < 1 ? 1 : b));
}

}  // namespace

cudaError_t mlp_gemm(const void* A, int lda, int ta, const void* B, int ldb, int tb, float* C, int ldc, int M, int N,
                     int K, const float* bias, int accumulate, cudaStream_t s) {
  dim3 grid((N + kTN - 1) / kTN, (M + kTM - 1) / kTM);
  gemm_bf16_kernel<<<grid, 128, 0, s>>>(static_cast<const __nv_bfloat16*>(A), lda, ta,
                                        static_cast<const __nv_bfloat16*>(B), ldb, tb, C, ldc, M, N, K, bias,
                                        accumulate);
  return cudaGetLastError();
}

cudaError_t mlp_gelu_fwd(const float* z, void* a16, int64_t n, cudaStream_t s) {
  gelu_fwd_kernel<<<blocks_for(n), 256, 0, s>>>(z, static_cast<__nv_bfloat16*>(a16), n);
  return cudaGetLastError();
}

cudaError_t mlp_gelu_bwd(const float* da, const float* z, void* dz16, float* dz32, int64_t n, cudaStream_t s) {
  gelu_bwd_kernel<<<blocks_for(n), 256, 0, s>>>(da, z, static_cast<__nv_bfloat16*>(dz16), dz32, n);
  return cudaGetLastError();
}

cudaError_t mlp_input(const float* x, void* y, int64_t rows, int cols, int nlog, float floor_, float scale,
                      cudaStream_t s) {
  input_kernel<<<blocks_for(rows * cols), 256, 0, s>>>(x, static_cast<__nv_bfloat16*>(y), rows, cols, nlog, floor_,
                                                       scale);
  return cudaGetLastError();
}

cudaError_t mlp_to_bf16(const float* x, void* y, int64_t n, cudaStream_t s) {
  to_bf16_kernel<<<blocks_for(n), 256, 0, s>>>(x, static_cast<__nv_bfloat16*>(y), n);
  return cudaGetLastError();
}

cudaError_t mlp_mse(const float* y, const float* t, float* dy32, void* dy16, int64_t n, double* loss,
                    cudaStream_t s) {
  mse_kernel<<<blocks_for(n), 256, 0, s>>>(y, t, dy32, static_cast<__nv_bfloat16*>(dy16), n, loss);
  return cudaGetLastError();
}

cudaError_t mlp_colsum(const float* dz, int M, int N, float* db, cudaStream_t s) {
  colsum_kernel<<<(N + 127) / 128, 128, 0, s>>>(dz, M, N, db);
  return cudaGetLastError();
}

cudaError_t mlp_adam(float* w, const float* g, float* m1, float* m2, void* w16, int64_t n, float lr, float b1, float b2,
                     float eps, float c1, float c2, cudaStream_t s) {
  adam_kernel<<<blocks_for(n), 256, 0, s>>>(w, g, m1, m2, static_cast<__nv_bfloat16*>(w16), n, lr, b1, b2, eps, c1,
                                            c2);
  return cudaGetLastError();
}

}  // namespace treeot
