// Device functions of the recomputed-cost edge apply (squared-Euclidean costs
// formed from point coordinates in the kernel), shared by the per-half-step
// apply kernel and the persistent forest kernel, with the helpers the
// stored-cost tasks use too.
#pragma once
#include <cfloat>
#include <cmath>

#include "grid.cuh"
#include "internal.h"
#include "ptx.cuh"

namespace treeot {
namespace {


#define kInf (__int_as_float(0x7f800000))
constexpr float kWindow = 12.f;   // a frame up to this far above the chunk maximum is kept
// The plain recomputed-cost apply moves a frame (see recomp_task):
constexpr float kWindowRec = 64.f;  //   down, for a fresh output, only when the chunk lies this far below it,
constexpr float kRoomRec = 32.f;    //   and then to this far above the chunk's maximum;
constexpr float kShiftRec = 2.f;    //   up by at most this much by shifting the chunk's terms
constexpr int kRecPts = 4;        // RECOMP: reduction points per frame check (per thread: 4 outputs x 4)


// t = (hh - R) - c*s + hl, s = s_hi + s_lo
__device__ __forceinline__ float arg1(float hh, float R, float c, float shi, float slo, float hl) {
  float t = fmaf(-c, shi, hh - R);
  t = fmaf(-c, slo, t);
  return t + hl;
}

// the four terms t of one float4 of costs against one float4 of operand
__device__ __forceinline__ void terms4(float4 c, float4 H, float4 L, float2 negR, float2 nhi, float2 nlo,
                                       float2& t01, float2& t23) {
  t01 = fma2(make_float2(c.x, c.y), nhi, add2(make_float2(H.x, H.y), negR));
  t23 = fma2(make_float2(c.z, c.w), nhi, add2(make_float2(H.z, H.w), negR));
  t01 = add2(fma2(make_float2(c.x, c.y), nlo, t01), make_float2(L.x, L.y));
  t23 = add2(fma2(make_float2(c.z, c.w), nlo, t23), make_float2(L.z, L.w));
}

// merge (frame, sum) pieces, skipping empty ones; result written as one piece
__device__ __forceinline__ float2 merge_pieces(const float2* p, int n, int stride) {
  float Rm = -kInf;
  for (int w = 0; w < n; ++w)
    if (p[w * stride].y > 0.f) Rm = fmaxf(Rm, p[w * stride].x);
  if (Rm == -kInf) return make_float2(0.f, 0.f);
  float S = 0.f;
  for (int w = 0; w < n; ++w) {
    const float2 q = p[w * stride];
    if (q.y > 0.f) S += (q.x == Rm) ? q.y : q.y * ex2(q.x - Rm);
  }
  return make_float2(Rm, S);
}

// squared Euclidean cost from coordinates; D in {1,2,3}
template <int D>
__device__ __forceinline__ float sqdist(float px, float py, float pz, float4 q) {
  // q holds the negated coordinates of the reduction point
  const float dx = px + q.x;
  float c = dx * dx;
  if (D > 1) {
    const float dy = py + q.y;
    c = fmaf(dy, dy, c);
  }
  if (D > 2) {
    const float dz = pz + q.z;
    c = fmaf(dz, dz, c);
  }
  return c;
}

// The CTA's 8 warps form G = t.pad groups (1, 2, 4 or 8).  Every group owns all
// of the task's outputs (4 per thread, up to 1024/G per task) and a 1/G share of
// each staged chunk of reduction points; groups merge through shared memory at
// the end.  Small supports (a few hundred points) thus keep all warps busy.
//
// The argument is t = (hh - R) - s |p - q|^2 with s = s_hi + s_lo (exact
// product inside the FMAs), and the term 2^t w with the point's weight
// w = 2^hl (the operand's low part, |hl| <= 2^-11, staged once per point): one
// FMA per term instead of an add to t and another to the sum.  Staged values
// are stored duplicated, (v, v) pairs, so every packed f32x2 operation reads
// its operands straight from shared memory.
template <int D>
__device__ void recomp_task(const ApplyArgs& A, const Task& t, float* sm) {
  const DEdgeD d = A.dedges[t.dedge];
  const NodeD own = A.nodes[d.owner];
  const NodeD nbn = A.nodes[d.nbr];
  const ProbD P = A.probs[d.prob];
  const float2 nhi = make_float2(-P.s2_scaled, -P.s2_scaled), nlo = make_float2(-P.s2_scaled_lo, -P.s2_scaled_lo);
  const float shi = P.s2_scaled, slo = P.s2_scaled_lo;
  const int n_owner = own.n;
  const int tid = threadIdx.x;
  const int G = t.pad;
  const int gs = kApplyThreads / G;  // threads per group
  const int g = tid / gs, tg = tid - g * gs;
  float4* sq = reinterpret_cast<float4*>(sm);                       // [256]: (-qx,-qx,-qy,-qy)
  float4* sz = sq + kApplyThreads;                                  // [256]: (-qz,-qz, *, *) (D == 3)
  float4* shl = sq + 2 * kApplyThreads;                             // [256]: (hh,hh,hl,hl)
  float2* comb = reinterpret_cast<float2*>(sm + 12 * kApplyThreads);  // [G][4 gs] group results
  float2 px01, px23, py01, py23, pz01, pz23;
  float R[4], acc[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int lo = tg + gs * i;
    const bool on = lo < t.ocount;
    const int o = t.o0 + (on ? lo : 0);
    const float* p = A.coords + own.coord_off + (int64_t)o * D;
    const float x0 = p[0], y0 = D > 1 ? p[1] : 0.f, z0 = D > 2 ? p[2] : 0.f;
    if (i == 0) { px01.x = x0; py01.x = y0; pz01.x = z0; }
    if (i == 1) { px01.y = x0; py01.y = y0; pz01.y = z0; }
    if (i == 2) { px23.x = x0; py23.x = y0; pz23.x = z0; }
    if (i == 3) { px23.y = x0; py23.y = y0; pz23.y = z0; }
    R[i] = on ? A.fr[d.off + o] : 0.f;
    acc[i] = 0.f;
  }
  const int per = kApplyThreads / G;  // staged points per group per chunk (multiple of kRecPts)
  for (int ch = 0; ch < t.rcount; ch += kApplyThreads) {
    __syncthreads();
    {
      const int j = ch + tid;
      const bool v = j < t.rcount;
      const int y = t.r0 + (v ? j : 0);
      const float* q = A.coords + nbn.coord_off + (int64_t)y * D;
      const float hh = v ? A.hh[d.rev_off + y] : -kInf;
      const float hl = v ? A.hl[d.rev_off + y] : 0.f;
      const float qy = D > 1 ? -q[1] : 0.f;
      sq[tid] = make_float4(-q[0], -q[0], qy, qy);
      if (D == 3) sz[tid] = make_float4(-q[2], -q[2], 0.f, 0.f);
      // the operand's low part as a weight of the point's terms: w = 2^hl by its
      // Taylor series in u = hl ln 2 to the cubic term (|hl| <= 2^-11 after the
      // node update's regrid: truncation below 2^-40, one FP32 rounding or so)
      const float u = hl * 0.69314718f;
      const float w = fmaf(u, fmaf(u, fmaf(u, 1.f / 6.f, 0.5f), 1.f), 1.f);
      shl[tid] = make_float4(hh, hh, w, w);
    }
    __syncthreads();
    const int cnt = min(kApplyThreads, t.rcount - ch);
    const int jend = min(g * per + per, cnt);
    for (int j = g * per; j < jend; j += kRecPts) {
      float tv[4][kRecPts];
      const float2 nR01 = make_float2(-R[0], -R[1]);
      const float2 nR23 = make_float2(-R[2], -R[3]);
#pragma unroll
      for (int jj = 0; jj < kRecPts; ++jj) {
        const float4 qq = sq[j + jj];  // entries past cnt hold hh = -inf: zero terms
        const float4 hv = shl[j + jj];
        const float2 qx = make_float2(qq.x, qq.y);
        float2 c01, c23;
        {
          const float2 dx01 = add2(px01, qx), dx23 = add2(px23, qx);
          c01 = mul2(dx01, dx01);
          c23 = mul2(dx23, dx23);
        }
        if (D > 1) {
          const float2 qy = make_float2(qq.z, qq.w);
          const float2 dy01 = add2(py01, qy), dy23 = add2(py23, qy);
          c01 = fma2(dy01, dy01, c01);
          c23 = fma2(dy23, dy23, c23);
        }
        if (D > 2) {
          const float4 zz = sz[j + jj];
          const float2 qz = make_float2(zz.x, zz.y);
          const float2 dz01 = add2(pz01, qz), dz23 = add2(pz23, qz);
          c01 = fma2(dz01, dz01, c01);
          c23 = fma2(dz23, dz23, c23);
        }
        const float2 h2 = make_float2(hv.x, hv.y);
        float2 t01 = fma2(c01, nhi, add2(h2, nR01));
        float2 t23 = fma2(c23, nhi, add2(h2, nR23));
        t01 = fma2(c01, nlo, t01);
        t23 = fma2(c23, nlo, t23);
        tv[0][jj] = t01.x;
        tv[1][jj] = t01.y;
        tv[2][jj] = t23.x;
        tv[3][jj] = t23.y;
      }
      float cmk[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        cmk[k] = fmaxf(tv[k][0], tv[k][1]);
#pragma unroll
        for (int jj = 2; jj < kRecPts; jj += 2) cmk[k] = max3f(cmk[k], tv[k][jj], tv[k][jj + 1]);
      }
      // one test for the four outputs in the common case (frames fit, sums started).
      // A frame moves up when a term exceeds it by more than 0.5, and down (before
      // anything is summed) when the chunk's terms all lie more than kWindowRec
      // below it; a term at t below its frame carries a rounding error of about
      // |t| 2^-24 but weighs 2^t, so terms far below their frame cost no
      // accuracy.  Moving down, the frame stops kRoomRec above the chunk's
      // maximum (later, larger terms then rarely move it up again), and the terms
      // shift with it: t - d is exact there (|t - d| < |t|, d on the 2^-10 grid).
      // Moving up by at most kShiftRec the terms shift too: the largest, now near
      // 0, keeps the rounding error of |t| <= 2 (at most 2^-23).  A larger move
      // up recomputes the chunk's terms from the moved frame.
      const bool fresh = (acc[0] == 0.f) | (acc[1] == 0.f) | (acc[2] == 0.f) | (acc[3] == 0.f);
      if (fresh || fmaxf(max3f(cmk[0], cmk[1], cmk[2]), cmk[3]) > 0.5f) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float cm = cmk[k];
          const bool up = cm > 0.5f, down = acc[k] == 0.f && cm < -kWindowRec;
          if ((up || down) && cm > -kInf) {
            const float dlt = down ? quant(cm) + kRoomRec : quant(cm);
            const float Rn = R[k] + dlt;
            acc[k] = acc[k] == 0.f ? 0.f : acc[k] * ex2(R[k] - Rn);
            R[k] = Rn;
            if (!up || cm <= kShiftRec) {
#pragma unroll
              for (int jj = 0; jj < kRecPts; ++jj) tv[k][jj] -= dlt;
              continue;
            }
            const float pxk = k == 0 ? px01.x : k == 1 ? px01.y : k == 2 ? px23.x : px23.y;
            const float pyk = k == 0 ? py01.x : k == 1 ? py01.y : k == 2 ? py23.x : py23.y;
            const float pzk = k == 0 ? pz01.x : k == 1 ? pz01.y : k == 2 ? pz23.x : pz23.y;
#pragma unroll
            for (int jj = 0; jj < kRecPts; ++jj) {
              const float4 qq = sq[j + jj];
              const float4 hv = shl[j + jj];
              const float dx = pxk + qq.x;
              float c = dx * dx;
              if (D > 1) {
                const float dy = pyk + qq.z;
                c = fmaf(dy, dy, c);
              }
              if (D > 2) {
                const float dz = pzk + sz[j + jj].x;
                c = fmaf(dz, dz, c);
              }
              tv[k][jj] = fmaf(-c, slo, fmaf(-c, shi, hv.x - Rn));
            }
          }
        }
      }
      // sum of 2^t 2^hl (the weight: t leaves out the operand's low part)
      float2 w2[kRecPts];
#pragma unroll
      for (int jj = 0; jj < kRecPts; ++jj) {
        const float w = shl[j + jj].z;
        w2[jj] = make_float2(w, w);
      }
#pragma unroll
      for (int k = 0; k < 4; k += 2) {
        float2 s01 = mul2(make_float2(ex2(tv[k][0]), ex2(tv[k + 1][0])), w2[0]);
#pragma unroll
        for (int jj = 1; jj < kRecPts; ++jj) s01 = fma2(make_float2(ex2(tv[k][jj]), ex2(tv[k + 1][jj])), w2[jj], s01);
        acc[k] += s01.x;
        acc[k + 1] += s01.y;
      }
    }
  }
  if (G == 1) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (tg + gs * i < t.ocount)
        A.part32[d.part_off + (int64_t)t.split * n_owner + t.o0 + tg + gs * i] = make_float2(R[i], acc[i]);
    return;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) comb[g * (4 * gs) + tg + gs * i] = make_float2(R[i], acc[i]);
  __syncthreads();
  for (int c = tid; c < t.ocount; c += kApplyThreads)
    A.part32[d.part_off + (int64_t)t.split * n_owner + t.o0 + c] = merge_pieces(comb + c, G, 4 * gs);
}

// Exact-distance variant for problems refined past the FP32 floor of the plain
// recomputation.  Rounding |p - q|^2 in FP32 perturbs the cost by a relative
// 2^-23, i.e. C/eps by up to ~1e-4 for C/eps in the hundreds, which settles
// the iterate ~1e-7..1e-6 (max marginal L1) away from the true fixed point.
// Here every coordinate arrives split as hi + lo, hi on a grid of
// unit = 2^-10 sigma (sigma a power of two >= max |coordinate| of the problem).
// Then p_hi - q_hi is exact (at most 12 significant bits), its square is exact
// (at most 22 bits) and so is the sum over D <= 3 dimensions (< 2^24 units^2):
//   c_hi = sum_d (p_hi - q_hi)^2                      (exact)
//   c_lo = sum_d dl (2 (p_hi - q_hi) + dl),  dl = p_lo - q_lo   (small)
//   t    = (hh - R) - c_hi s_hi - c_hi s_lo - c_lo s_hi + hl,
// so the argument keeps the exactness of the stored-cost kernels.
template <int D>
__device__ void recomp_task_exact(const ApplyArgs& A, const Task& t, float* sm) {
  const DEdgeD d = A.dedges[t.dedge];
  const NodeD own = A.nodes[d.owner];
  const NodeD nbn = A.nodes[d.nbr];
  const ProbD P = A.probs[d.prob];
  const float2 nhi = make_float2(-P.s2_scaled, -P.s2_scaled), nlo = make_float2(-P.s2_scaled_lo, -P.s2_scaled_lo);
  const float2 two = make_float2(2.f, 2.f);
  const int n_owner = own.n;
  const int tid = threadIdx.x;
  const int G = t.pad;
  const int gs = kApplyThreads / G;
  const int g = tid / gs, tg = tid - g * gs;
  float4* sxh = reinterpret_cast<float4*>(sm);                        // (-qx_hi, -qx_hi, -qy_hi, -qy_hi)
  float4* sxl = sxh + kApplyThreads;                                  // (-qx_lo, -qx_lo, -qy_lo, -qy_lo)
  float4* sz = sxh + 2 * kApplyThreads;                               // (-qz_hi, -qz_hi, -qz_lo, -qz_lo)
  float4* shl = sxh + 3 * kApplyThreads;                              // (hh, hh, hl, hl)
  float2* comb = reinterpret_cast<float2*>(sm + 16 * kApplyThreads);  // [G][4 gs]
  float ph[4][3], pl[4][3];
  float R[4], acc[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int lo = tg + gs * i;
    const bool on = lo < t.ocount;
    const int o = t.o0 + (on ? lo : 0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      ph[i][k] = k < D ? A.coords_hi[own.coord_off + (int64_t)o * D + k] : 0.f;
      pl[i][k] = k < D ? A.coords_lo[own.coord_off + (int64_t)o * D + k] : 0.f;
    }
    R[i] = on ? A.fr[d.off + o] : 0.f;
    acc[i] = 0.f;
  }
  const float2 pxh01 = make_float2(ph[0][0], ph[1][0]), pxh23 = make_float2(ph[2][0], ph[3][0]);
  const float2 pxl01 = make_float2(pl[0][0], pl[1][0]), pxl23 = make_float2(pl[2][0], pl[3][0]);
  const float2 pyh01 = make_float2(ph[0][1], ph[1][1]), pyh23 = make_float2(ph[2][1], ph[3][1]);
  const float2 pyl01 = make_float2(pl[0][1], pl[1][1]), pyl23 = make_float2(pl[2][1], pl[3][1]);
  const float2 pzh01 = make_float2(ph[0][2], ph[1][2]), pzh23 = make_float2(ph[2][2], ph[3][2]);
  const float2 pzl01 = make_float2(pl[0][2], pl[1][2]), pzl23 = make_float2(pl[2][2], pl[3][2]);
  const int per = kApplyThreads / G;
  for (int ch = 0; ch < t.rcount; ch += kApplyThreads) {
    __syncthreads();
    {
      const int j = ch + tid;
      const bool v = j < t.rcount;
      const int y = t.r0 + (v ? j : 0);
      const float* qh = A.coords_hi + nbn.coord_off + (int64_t)y * D;
      const float* ql = A.coords_lo + nbn.coord_off + (int64_t)y * D;
      const float hh = v ? A.hh[d.rev_off + y] : -kInf;
      const float hl = v ? A.hl[d.rev_off + y] : 0.f;
      const float yh = D > 1 ? -qh[1] : 0.f, yl = D > 1 ? -ql[1] : 0.f;
      sxh[tid] = make_float4(-qh[0], -qh[0], yh, yh);
      sxl[tid] = make_float4(-ql[0], -ql[0], yl, yl);
      if (D == 3) sz[tid] = make_float4(-qh[2], -qh[2], -ql[2], -ql[2]);
      shl[tid] = make_float4(hh, hh, hl, hl);
    }
    __syncthreads();
    const int cnt = min(kApplyThreads, t.rcount - ch);
    const int jend = min(g * per + per, cnt);
    for (int j = g * per; j < jend; j += kRecPts) {
      float tv[4][kRecPts];
      // all terms of the chunk relative to the current frames
      auto terms = [&]() {
        const float2 nR01 = make_float2(-R[0], -R[1]);
        const float2 nR23 = make_float2(-R[2], -R[3]);
#pragma unroll
        for (int jj = 0; jj < kRecPts; ++jj) {
          const float4 qh = sxh[j + jj], ql = sxl[j + jj], hv = shl[j + jj];
          float2 ch01, ch23, cl01, cl23;
          {
            const float2 dh01 = add2(pxh01, make_float2(qh.x, qh.y)), dh23 = add2(pxh23, make_float2(qh.x, qh.y));
            const float2 dl01 = add2(pxl01, make_float2(ql.x, ql.y)), dl23 = add2(pxl23, make_float2(ql.x, ql.y));
            ch01 = mul2(dh01, dh01);
            ch23 = mul2(dh23, dh23);
            cl01 = mul2(dl01, fma2(two, dh01, dl01));
            cl23 = mul2(dl23, fma2(two, dh23, dl23));
          }
          if (D > 1) {
            const float2 dh01 = add2(pyh01, make_float2(qh.z, qh.w)), dh23 = add2(pyh23, make_float2(qh.z, qh.w));
            const float2 dl01 = add2(pyl01, make_float2(ql.z, ql.w)), dl23 = add2(pyl23, make_float2(ql.z, ql.w));
            ch01 = fma2(dh01, dh01, ch01);
            ch23 = fma2(dh23, dh23, ch23);
            cl01 = fma2(dl01, fma2(two, dh01, dl01), cl01);
            cl23 = fma2(dl23, fma2(two, dh23, dl23), cl23);
          }
          if (D > 2) {
            const float4 zz = sz[j + jj];
            const float2 dh01 = add2(pzh01, make_float2(zz.x, zz.y)), dh23 = add2(pzh23, make_float2(zz.x, zz.y));
            const float2 dl01 = add2(pzl01, make_float2(zz.z, zz.w)), dl23 = add2(pzl23, make_float2(zz.z, zz.w));
            ch01 = fma2(dh01, dh01, ch01);
            ch23 = fma2(dh23, dh23, ch23);
            cl01 = fma2(dl01, fma2(two, dh01, dl01), cl01);
            cl23 = fma2(dl23, fma2(two, dh23, dl23), cl23);
          }
          const float2 h2 = make_float2(hv.x, hv.y), l2 = make_float2(hv.z, hv.w);
          float2 t01 = fma2(ch01, nhi, add2(h2, nR01));
          float2 t23 = fma2(ch23, nhi, add2(h2, nR23));
          t01 = fma2(cl01, nhi, fma2(ch01, nlo, t01));
          t23 = fma2(cl23, nhi, fma2(ch23, nlo, t23));
          t01 = add2(t01, l2);
          t23 = add2(t23, l2);
          tv[0][jj] = t01.x;
          tv[1][jj] = t01.y;
          tv[2][jj] = t23.x;
          tv[3][jj] = t23.y;
        }
      };
      terms();
      float cmk[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        cmk[k] = fmaxf(tv[k][0], tv[k][1]);
#pragma unroll
        for (int jj = 2; jj < kRecPts; jj += 2) cmk[k] = max3f(cmk[k], tv[k][jj], tv[k][jj + 1]);
      }
      const bool fresh = (acc[0] == 0.f) | (acc[1] == 0.f) | (acc[2] == 0.f) | (acc[3] == 0.f);
      if (fresh || fmaxf(max3f(cmk[0], cmk[1], cmk[2]), cmk[3]) > 0.5f) {
        bool moved = false;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float cm = cmk[k];
          if ((cm > 0.5f || (acc[k] == 0.f && cm < -kWindow)) && cm > -kInf) {
            const float Rn = R[k] + quant(cm);
            acc[k] = acc[k] == 0.f ? 0.f : acc[k] * ex2(R[k] - Rn);
            R[k] = Rn;
            moved = true;
          }
        }
        if (moved) terms();  // rare: the chunk again from the moved frames
      }
#pragma unroll
      for (int k = 0; k < 4; k += 2) {
        float2 s01 = make_float2(ex2(tv[k][0]), ex2(tv[k + 1][0]));
#pragma unroll
        for (int jj = 1; jj < kRecPts; ++jj) s01 = add2(s01, make_float2(ex2(tv[k][jj]), ex2(tv[k + 1][jj])));
        acc[k] += s01.x;
        acc[k + 1] += s01.y;
      }
    }
  }
  if (G == 1) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (tg + gs * i < t.ocount)
        A.part32[d.part_off + (int64_t)t.split * n_owner + t.o0 + tg + gs * i] = make_float2(R[i], acc[i]);
    return;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) comb[g * (4 * gs) + tg + gs * i] = make_float2(R[i], acc[i]);
  __syncthreads();
  for (int c = tid; c < t.ocount; c += kApplyThreads)
    A.part32[d.part_off + (int64_t)t.split * n_owner + t.o0 + c] = merge_pieces(comb + c, G, 4 * gs);
}

}  // namespace
}  // namespace treeot
