// Unit-rate microbenchmark for the roofline denominators of the recomputed-cost
// apply: FP32 FMA lanes per clock and SM (scalar and packed f32x2), MUFU ex2 per
// clock and SM, and the relative error of ex2.approx.ftz.f32 against FP64 exp2;
// for the node update, FP64 FMA lanes and float <-> double conversion pairs per
// clock and SM.
// A standalone program (not part of the library); bench.py --unit-rates builds
// and runs it.  Prints one JSON object.
#include <cmath>
#include <cstdio>
#include <cuda_runtime.h>

namespace {

__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm volatile("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
               "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
               "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
               : "=f"(d.x), "=f"(d.y)
               : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}

// 8 independent FMA chains per thread
__global__ void k_ffma(float* out, int iters, float b) {
  float a[8];
  for (int i = 0; i < 8; ++i) a[i] = threadIdx.x * 1e-3f + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = fmaf(a[i], b, 0.5f);
  }
  float s = 0.f;
  for (int i = 0; i < 8; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// 8 independent packed chains per thread (16 lanes of work)
__global__ void k_ffma2(float* out, int iters, float b) {
  float2 a[8];
  for (int i = 0; i < 8; ++i) a[i] = make_float2(threadIdx.x * 1e-3f + i, i + 0.5f);
  const float2 bb = make_float2(b, b), cc = make_float2(0.5f, 0.5f);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = fma2(a[i], bb, cc);
  }
  float s = 0.f;
  for (int i = 0; i < 8; ++i) s += a[i].x + a[i].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// 8 independent ex2 chains per thread (one FMUL each to keep values bounded)
__global__ void k_ex2(float* out, int iters, float b) {
  float a[8];
  for (int i = 0; i < 8; ++i) a[i] = threadIdx.x * 1e-3f + i * 0.01f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      float y;
      asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[i]));
      a[i] = y * b;
    }
  }
  float s = 0.f;
  for (int i = 0; i < 8; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// 8 independent FP64 FMA chains per thread
__global__ void k_dfma(float* out, int iters, float b) {
  double a[8];
  const double bd = b;
  for (int i = 0; i < 8; ++i) a[i] = threadIdx.x * 1e-3 + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = fma(a[i], bd, 0.5);
  }
  double s = 0.0;
  for (int i = 0; i < 8; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}

// 8 independent chains per thread of a float -> double -> float conversion pair
__global__ void k_cvt(float* out, int iters, float b) {
  float a[8];
  for (int i = 0; i < 8; ++i) a[i] = threadIdx.x * 1e-3f + i + b;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      double d;
      asm volatile("cvt.f64.f32 %0, %1;" : "=d"(d) : "f"(a[i]));
      asm volatile("cvt.rn.f32.f64 %0, %1;" : "=f"(a[i]) : "d"(d));
    }
  }
  float s = 0.f;
  for (int i = 0; i < 8; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// relative error of ex2.approx over t in [-24, 1): sum, sum of squares, max |.|
__global__ void k_ex2_err(double* stats, long n) {
  double s = 0.0, s2 = 0.0, mx = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const float t = -24.f + (float)((double)i * (25.0 / (double)n));
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(t));
    const double r = (double)y / exp2((double)t) - 1.0;
    s += r;
    s2 += r * r;
    mx = fmax(mx, fabs(r));
  }
  atomicAdd(&stats[0], s);
  atomicAdd(&stats[1], s2);
  atomicMax(reinterpret_cast<unsigned long long*>(&stats[2]), (unsigned long long)__double_as_longlong(mx));
}

}  // namespace

int main() {
  int sms = 0, clk_khz = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, 0);
  const int blocks = sms * 8, threads = 256, iters = 4096;
  float* out = nullptr;
  if (cudaMalloc(&out, sizeof(float) * blocks * threads) != cudaSuccess) return 1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double rate[5] = {0, 0, 0, 0, 0};
  for (int k = 0; k < 5; ++k) {
    const int kiters = k >= 3 ? iters / 16 : iters;  // FP64 work is much slower
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {  // the first launch warms up
      cudaEventRecord(e0);
      if (k == 0) k_ffma<<<blocks, threads>>>(out, iters, 0.999f);
      if (k == 1) k_ffma2<<<blocks, threads>>>(out, iters, 0.999f);
      if (k == 2) k_ex2<<<blocks, threads>>>(out, iters, 0.999f);
      if (k == 3) k_dfma<<<blocks, threads>>>(out, kiters, 0.999f);
      if (k == 4) k_cvt<<<blocks, threads>>>(out, kiters, 0.999f);
      cudaEventRecord(e1);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ms, e0, e1);
    }
    const double lanes = (double)blocks * threads * kiters * 8 * (k == 1 ? 2 : 1);
    rate[k] = lanes / (ms * 1e-3);  // lane operations per second
  }
  const long n = 1L << 26;
  double* st = nullptr;
  if (cudaMalloc(&st, sizeof(double) * 3) != cudaSuccess) return 1;
  cudaMemset(st, 0, sizeof(double) * 3);
  k_ex2_err<<<1024, 256>>>(st, n);
  double h[3];
  cudaMemcpy(h, st, sizeof(h), cudaMemcpyDeviceToHost);
  const cudaError_t err = cudaGetLastError();
  const double ghz = clk_khz * 1e-6;
  printf("{\"sms\": %d, \"max_clock_ghz\": %.3f, \"ffma_lanes_per_clk_sm\": %.2f, \"ffma2_lanes_per_clk_sm\": %.2f, "
         "\"ex2_per_clk_sm\": %.2f, \"dfma_lanes_per_clk_sm\": %.3f, \"cvt_f32_f64_pairs_per_clk_sm\": %.3f, "
         "\"ex2_rel_err\": {\"mean\": %.3e, \"rms\": %.3e, \"max\": %.3e}, "
         "\"note\": \"per clock at the device's maximum SM clock\", \"status\": \"%s\"}\n",
         sms, ghz, rate[0] / (ghz * 1e9) / sms, rate[1] / (ghz * 1e9) / sms, rate[2] / (ghz * 1e9) / sms,
         rate[3] / (ghz * 1e9) / sms, rate[4] / (ghz * 1e9) / sms,
         h[0] / n, sqrt(h[1] / n), h[2], cudaGetErrorString(err));
  cudaFree(st);
  cudaFree(out);
  return err == cudaSuccess ? 0 : 1;
}
