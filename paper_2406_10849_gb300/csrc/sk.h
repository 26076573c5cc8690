// Shared-kernel BF16 phase (squared-Euclidean costs): plan structures and
// launchers shared by the host planner (api.cpp) and apply_sk.cu.
//
// Directed edges whose owner supports, neighbour supports, cost scale and eps
// coincide share one Gibbs kernel K(x,y) = 2^(-s C(x,y)), s = scale log2(e)/eps
// (every edge of a star whose nodes sit on one grid, across a batch of such
// stars).  One colour's messages of such a group are then one matrix product:
//   m_j(x) = log2 sum_y K(x,y) 2^(h_j(y)),   j = the group's active columns.
// In the phase it is evaluated as
//   M_j   = max_y h_j(y) on the 2^-10 grid         (column maximum)
//   b(y)  = max_j (h_j(y) - M_j) on the grid       (envelope of the normalised columns)
//   R(x)  = max_y (b(y) - s C(x,y)) on the grid    (row frame)
//   K'(x,y) = 2^(b(y) - R(x) - s C(x,y)) in (0, 1],  V'(y,j) = 2^(h_j(y) - M_j - b(y)) in (0, 1]
//   S(x,j) = sum_y K'(x,y) V'(y,j),   m_j(x) = R(x) + M_j + log2 S(x,j)
// (the column maxima take out each column's own offset, which differs from
// problem to problem by the potentials' free constants).
// with K' and V' each split into two BF16 parts (hi + lo) and
// S = K'hi V'hi + K'hi V'lo + K'lo V'hi accumulated in FP32 on the tensor cores.
#pragma once
#include <cuda.h>  // CUtensorMap (the type only; the encoder is fetched through the runtime)
#include <cuda_bf16.h>
#include <cstdint>

#include "internal.h"

namespace treeot {

constexpr int kSkTileM = 128;  // rows (x) per GEMM CTA
constexpr int kSkTileN = 128;  // columns (directed edges) per GEMM CTA
constexpr int kSkTileK = 32;   // reduction points (y) per stage (mma.sync variant)
constexpr int kSkPadK = 64;    // reduction length padding (a multiple of both products' stages)
constexpr int kSkEnvCols = 32;  // columns per envelope CTA (one partial envelope each)

// Outputs whose sum S(x,j) falls below 2^-96 (the column's message more than
// ~96 binades under the row frame R(x), where its terms' factors may have left
// the BF16/FP32 range) are listed by the product and recomputed by
// sk_fixup_kernel as a plain FP32 log-sum-exp over y.
constexpr float kSkFixBelow = 1.2621774e-29f;  // 2^-96

// one column of a group: a directed edge of one colour
struct SkCol {
  int64_t h_off;     // its operand (hh, hl of the reverse directed edge), length ny
  int64_t part_off;  // its partial: part32[part_off + x] (piece 0), written by the
                     // exact fix-up for the outputs it recomputes
  int32_t prob;
  int32_t dedge;     // the directed edge whose message the column is
};

struct SkArgs {
  const SkCol* cols;
  int32_t ncols;
  int32_t nx, ny, dim;
  int32_t mp, kd;         // rows padded to kSkTileM, reduction length padded to kSkPadK
  int32_t use_tc;         // 1: tcgen05 product (tensor memory accumulators), 0: mma.sync
  int32_t tc_pair;        // 1: the tcgen05 product over CTA pairs (256-row MMAs), 0: one CTA per tile
  const float* hh;
  const float* hl;
  const int32_t* done;
  const int32_t* lowp;    // the phase runs on problems with lowp == 1
  const float* xc;        // row (owner) support, nx x dim
  const float* yc;        // column (neighbour) support, ny x dim
  float s_hi, s_lo;       // scale log2(e) / eps as a two-float
  float* b;               // [kd] envelope; -inf between uses
  float* benv;            // [ceil(ncols / kSkEnvCols)][kd] per-CTA envelopes of the one-pass envelope kernel
  float* cmax;            // [ncols] column maxima M_j (-inf: inactive)
  float* rf;              // [mp] row frames R(x)
  __nv_bfloat16* khi;     // [mp][kd]
  __nv_bfloat16* klo;
  __nv_bfloat16* vhi;     // [ncols][kd]
  __nv_bfloat16* vlo;
  float2* part32;
  float* sout;            // [ncols][ldo] sums S(x, j) (-1: listed for the fix-up, which writes part32)
  int32_t ldo;            // sout's row stride: nx rounded up to 32 floats
  int32_t store_tma;      // 1: the tcgen05 product writes sout through a TMA tensor map (SkMaps::sout)
  int32_t* fix_count;     // outputs listed for the exact fix-up (reset by the envelope launch)
  int2* fix_list;         // (x, column), capacity nx * ncols
  int32_t* err;           // error word: bit 1 = a bounded wait of the tcgen05 product ran out
};

// tensor maps of the tcgen05 product's operands (64-wide BF16 boxes of 128 rows, V' boxes
// of 64 rows for the pair product; 128-byte swizzle)
struct SkMaps {
  CUtensorMap khi, klo, vhi, vlo;
  CUtensorMap sout;  // FP32 [ncols][ldo], 32 x 16 boxes (outputs x columns); valid when store_tma
};
// fills `m` for the operands of `a`; false when cuTensorMapEncodeTiled is unavailable or refuses them
bool sk_encode_maps(const SkArgs& a, SkMaps* m);

// whether the tcgen05 product can run on the current device
bool sk_tc_available();
// whether its CTA-pair form (clusters of two) can run on the current device
bool sk_tc_pair_available();

// the five launches of one group and colour (nothing to do when ncols == 0)
// before_product / after_product (may be null): events recorded around the product launch
cudaError_t launch_sk(const SkArgs& a, const SkMaps* maps, cudaStream_t s, cudaEvent_t before_product = nullptr,
                      cudaEvent_t after_product = nullptr);
// b := -inf (once at create; afterwards each product resets it)
cudaError_t launch_sk_reset(float* b, int32_t kd, cudaStream_t s);

}  // namespace treeot
