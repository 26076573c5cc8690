// Plan entries B(x,y) = exp(a(x) + b(y) - C(x,y)/eps) in double-float arithmetic
// (pairs of FP32 values with error-free transformations), shared by the FP64-grade
// check and the rounding kernels: the exponent is exact to ~1e-12 before one
// accurate expf of its high part, so every entry has ~1e-7 relative error with no
// systematic part, at FP32-pipe speed (FP64 runs at a small fraction of that here).
#pragma once
#include <cuda_runtime.h>

#include "internal.h"

namespace treeot {

struct DF {
  float hi, lo;
};

// The error-free transformations below use the _rn intrinsics, which the
// compiler never contracts into FMAs: a product fused into a neighbouring
// addition would no longer be the rounded value the error term was taken from.
__device__ __forceinline__ DF two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

// exact-ish square of (p - q) as a double-float
__device__ __forceinline__ DF sq_diff(float p, float q) {
  const DF d = two_sum(p, -q);
  const float h = __fmul_rn(d.hi, d.hi);
  const float e = fmaf(2.f * d.hi, d.lo, fmaf(d.hi, d.hi, -h));
  return {h, e};
}

__device__ __forceinline__ DF df_add(DF a, DF b) {
  const DF s = two_sum(a.hi, b.hi);
  return {s.hi, s.lo + a.lo + b.lo};
}

// squared distance of two D-dimensional FP32 points (D <= 3) as a double-float
__device__ __forceinline__ DF sq_dist_df(int D, const float* pa, const float* pb) {
  DF c = sq_diff(pa[0], pb[0]);
  if (D > 1) c = df_add(c, sq_diff(pa[1], pb[1]));
  if (D > 2) c = df_add(c, sq_diff(pa[2], pb[2]));
  return c;
}

// C(x,y) as a double-float (rows x of the stored matrix); dense costs are exact FP32 values
__device__ __forceinline__ DF cost_df(const EdgeD& e, const ProbD& P, int x, int y, const float* pa,
                                     const float* pb) {
  if (P.cost_kind == 0) return {e.C[(int64_t)x * e.ld + y], 0.f};
  return sq_dist_df(P.dim, pa, pb);
}

// B = exp(a + b - C * k), k = scale / eps as (kh, kl); returns B and, in cost_out,
// C / scale rounded to FP32
__device__ __forceinline__ float plan_entry(float ah, float al, float bh, float bl, DF c, float kh, float kl,
                                            float& cost_out) {
  const DF s = two_sum(ah, bh);
  const float p = __fmul_rn(c.hi, kh);  // the rounded product; pe holds what it lost
  const float pe = fmaf(c.hi, kl, fmaf(c.lo, kh, fmaf(c.hi, kh, -p)));
  const DF d = two_sum(s.hi, -p);
  const float lo = (s.lo + d.lo) + (al + bl) - pe;
  cost_out = c.hi + c.lo;
  const float E = expf(d.hi);
  return E == 0.f ? 0.f : E * (1.f + lo);
}

}  // namespace treeot
