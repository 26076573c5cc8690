// Stored-cost edge apply with bulk-copy staged tiles.
//
// Same tasks and per-element arithmetic as the ROW / COL tasks of
// apply_dense_kernel (apply_f32.cu).  Everything a task reads reaches shared
// memory through bulk asynchronous copies (cp.async.bulk, completion counted
// on mbarriers) issued by one producer warp:
//   * the cost tile, a row at a time, into a ring of kStages 32 KB stages;
//   * the reduction-side operand (hh, hl) and the outputs' frame sources (m)
//     into one of two per-task buffers.
// The consumer warps (kGroups groups of eight) compute from shared memory only,
// so no consumer ever stalls on a global load; group g takes the stages whose
// running index (over all of the CTA's tasks) is g (mod kGroups).  kStages is a
// multiple of kGroups, so every ring slot is always read by the same group and a
// group waits on each of its slots' phases in order: a parity wait is never more
// than one phase ahead of its barrier (one phase ahead would read as already
// complete).  The producer keeps up to kStages stages plus the next task's
// vectors in flight (about 150 KB per SM).  Task records are resolved on the
// host (StreamTask): one load per task, no pointer chasing.
//
//   ROW task (<= 64 rows x 1024 columns): one stage = 8 rows; consumer warp w
//     of the stage's group takes row w (warp-uniform frame, two passes).
//   COL task (<= 512 rows x 128 columns): one stage = 64 rows of 128 columns;
//     warp w of the group takes rows 8w..8w+7 of its stages for its lane's 4
//     columns and keeps running frames; the warps merge at the task's end.
//
// Every mbarrier wait is bounded (kWaitLimitNs of wall time, with back-off).  A
// wait that runs out sets bit 1 of the error word (TREE_OT_ERR_TIMEOUT) and
// the ring's abort flag; from then on the producer issues no copies and every
// consumer warp skips its work but still arrives on every barrier and reaches
// every named barrier of the CTA, so nothing waits forever.  Before exiting,
// the producer waits (bounded) until every copy it issued has landed.
#include <atomic>
#include <cfloat>
#include <cmath>
#include <cstdint>

#include "internal.h"
#include "ptx.cuh"

namespace treeot {
namespace {

#define kInf (__int_as_float(0x7f800000))
constexpr int kStages = 4;  // measured against 6: 0.643 vs 0.662 ms per launch on the 64-node tree
constexpr int kStageBytes = 32 * 1024;
constexpr int kGroupWarps = 8;  // consumer warps per group (one per stage row block)
// Consumer groups take turns on stages.  The register file is split between the
// SM's four schedulers, so a CTA of 1 + 8 g warps fits only if every scheduler's
// share (up to ceil((1 + 8 g) / 4) warps) holds its registers: g = 2 needs at
// most 102 registers per thread, which the shared-memory-resident rows allow.
constexpr int kGroups = 2;
constexpr int kConsumers = kGroupWarps * kGroups;  // consumer warps
static_assert(kStages % kGroups == 0, "each ring slot must belong to one consumer group");
constexpr int kTmaThreads = (kConsumers + 1) * 32;
constexpr float kWindowT = 12.f;
constexpr uint64_t kWaitLimitNs = 250ull * 1000 * 1000;  // a wait gives up after 250 ms
constexpr uint32_t kWaitPolls = 1u << 24;                 // or after this many polls
// per-task buffer: hh[1024], hl[1024], frames[128] (floats)
constexpr int kVecFloats = kRowCols;
constexpr int kFrameMax = kColCols;  // >= 8 * kRowRowsPerWarp
constexpr int kTaskBufBytes = (2 * kVecFloats + kFrameMax) * 4;

__device__ __forceinline__ float quant(float v) { return rintf(v * 1024.f) * (1.f / 1024.f); }

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// bounded wait: kWaitLimitNs of wall time (checked every 64 polls) and, as a
// backstop, kWaitPolls polls; false when either ran out
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  uint64_t start = 0;
  for (uint32_t i = 0; i < kWaitPolls; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63) == 63) {
      const uint64_t now = global_ns();
      if (start == 0) start = now;
      else if (now - start > kWaitLimitNs) return false;
      __nanosleep(256);
    }
  }
  return false;
}

// warp-uniform bounded wait (any lane seeing the phase complete counts)
__device__ __forceinline__ bool mbar_wait_warp(uint64_t* bar, uint32_t parity) {
  return __any_sync(0xffffffffu, mbar_wait(bar, parity));
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// named barrier among the consumer warps only
__device__ __forceinline__ void consumers_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kConsumers * 32)); }

struct Ring {
  uint64_t full[kStages];
  uint64_t empty[kStages];
  uint64_t tfull[2];   // per-task vectors landed
  uint64_t tempty[2];  // consumers done with a per-task buffer
  volatile int abort;
};

struct TaskBuf {
  float* hh;
  float* hl;
  float* fr;
};

__device__ __forceinline__ TaskBuf task_buf(char* base, int b) {
  float* p = reinterpret_cast<float*>(base + b * kTaskBufBytes);
  return TaskBuf{p, p + kVecFloats, p + 2 * kVecFloats};
}

// number of stages a task occupies
__device__ __forceinline__ int task_stages(const StreamTask& t) {
  return t.kind == TASK_ROW ? (t.ocount + 7) / 8 : (t.rcount + 63) / 64;
}

__device__ __forceinline__ bool skipped(const ApplyArgs& A, const StreamTask& t) {
  return A.done[t.prob] || A.lowp[t.prob] == 1;
}

__device__ void producer(const ApplyArgs& A, char* stages, char* tbufs, Ring* ring) {
  const int lane = threadIdx.x & 31;
  uint32_t it = 0;  // stages issued
  uint32_t tc = 0;  // task buffers issued
  if (A.test_stall) return;  // test hook: nothing arrives, every consumer wait runs out
  bool alive = true;
  for (int ti = blockIdx.x; ti < A.ntasks && alive; ti += gridDim.x) {
    const StreamTask t = A.stasks[ti];
    if (skipped(A, t)) continue;
    {
      const int b = tc & 1;
      if (ring->abort || !mbar_wait_warp(&ring->tempty[b], ((tc >> 1) & 1) ^ 1)) {
        alive = false;
        break;
      }
      // vectors rounded up to 16 bytes (the arena pads every vector to 32 entries)
      const uint32_t hb = 4u * (uint32_t)((t.rcount + 3) & ~3);
      const uint32_t fb = 4u * (uint32_t)((t.ocount + 3) & ~3);
      TaskBuf tb = task_buf(tbufs, b);
      if (lane == 0) mbar_expect_tx(&ring->tfull[b], 2 * hb + fb);
      __syncwarp();
      if (lane == 0) bulk_g2s(tb.hh, A.hh + t.h_off, hb, &ring->tfull[b]);
      if (lane == 1) bulk_g2s(tb.hl, A.hl + t.h_off, hb, &ring->tfull[b]);
      if (lane == 2) bulk_g2s(tb.fr, A.fr + t.m_off, fb, &ring->tfull[b]);
      ++tc;
    }
    const int ns = task_stages(t);
    for (int s = 0; s < ns; ++s) {
      const int slot = it % kStages;
      if (ring->abort || !mbar_wait_warp(&ring->empty[slot], ((it / kStages) & 1) ^ 1)) {
        alive = false;
        break;
      }
      char* dst = stages + slot * kStageBytes;
      if (t.kind == TASK_ROW) {
        // 8 rows of up to 1024 columns; the cost's row stride is a multiple of 4
        // floats with +inf pads, so rounding the length up to 16 bytes stays in the row
        const int r0 = 8 * s;
        const int nrows = min(8, t.ocount - r0);
        const uint32_t rb = 4u * (uint32_t)((t.rcount + 3) & ~3);
        if (lane == 0) mbar_expect_tx(&ring->full[slot], rb * nrows);
        __syncwarp();
        if (lane < nrows) bulk_g2s(dst + lane * 4096, t.C + (int64_t)(r0 + lane) * t.ld, rb, &ring->full[slot]);
      } else {
        // 64 rows of up to 128 columns
        const int r0 = 64 * s;
        const int nrows = min(64, t.rcount - r0);
        const uint32_t rb = 4u * (uint32_t)((t.ocount + 3) & ~3);
        if (lane == 0) mbar_expect_tx(&ring->full[slot], rb * nrows);
        __syncwarp();
        for (int r = lane; r < nrows; r += 32)
          bulk_g2s(dst + r * 512, t.C + (int64_t)(r0 + r) * t.ld, rb, &ring->full[slot]);
      }
      ++it;
    }
  }
  if (!alive && lane == 0) {
    ring->abort = 1;
    atomicOr(A.err, 2);
  }
  // drain: every copy issued into the last kStages stages and the last two task
  // buffers has landed before the CTA may exit
  if (lane == 0) {
    const uint32_t first = it > (uint32_t)kStages ? it - kStages : 0;
    for (uint32_t j = first; j < it; ++j) (void)mbar_wait(&ring->full[j % kStages], (j / kStages) & 1);
    const uint32_t tfirst = tc > 2u ? tc - 2 : 0;
    for (uint32_t j = tfirst; j < tc; ++j) (void)mbar_wait(&ring->tfull[j & 1], (j >> 1) & 1);
  }
}

// the four terms of one float4 of costs against one float4 of operand
__device__ __forceinline__ void terms4(float4 c, float4 H, float4 L, float2 negR, float2 nhi, float2 nlo,
                                       float2& t01, float2& t23) {
  t01 = fma2(make_float2(c.x, c.y), nhi, add2(make_float2(H.x, H.y), negR));
  t23 = fma2(make_float2(c.z, c.w), nhi, add2(make_float2(H.z, H.w), negR));
  t01 = add2(fma2(make_float2(c.x, c.y), nlo, t01), make_float2(L.x, L.y));
  t23 = add2(fma2(make_float2(c.z, c.w), nlo, t23), make_float2(L.z, L.w));
}

// one row of a ROW task, read from the stage: every term formed once (maximum
// and sum relative to the row's frame); summed again from shared memory only
// when the maximum leaves the frame's window.  Nothing of the row is held in
// registers, which keeps the consumers small enough for 16 warps per SM.
__device__ __forceinline__ float2 consume_row(const StreamTask& t, const float* srow, const float* sh,
                                              const float* sl, float R) {
  const float2 nhi = make_float2(-t.s2, -t.s2), nlo = make_float2(-t.s2_lo, -t.s2_lo);
  const int lane = threadIdx.x & 31;
  const int nvec = (t.rcount + 3) >> 2;
  const float4* c4 = reinterpret_cast<const float4*>(srow);
  const float4* sh4 = reinterpret_cast<const float4*>(sh);
  const float4* sl4 = reinterpret_cast<const float4*>(sl);
  float cm = -kInf, acc = 0.f;
  {
    const float2 negR = make_float2(-R, -R);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int v = lane + 32 * i;
      if (v < nvec) {
        float2 t01, t23;
        terms4(c4[v], sh4[v], sl4[v], negR, nhi, nlo, t01, t23);
        cm = max3f(cm, t01.x, t01.y);
        cm = max3f(cm, t23.x, t23.y);
        acc += (ex2(t01.x) + ex2(t01.y)) + (ex2(t23.x) + ex2(t23.y));
      }
    }
  }
  const float cw = warp_max(cm);
  if ((cw > 0.5f || cw < -kWindowT) && cw > -kInf) {
    R += quant(cw);
    acc = 0.f;
    const float2 negR = make_float2(-R, -R);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int v = lane + 32 * i;
      if (v < nvec) {
        float2 t01, t23;
        terms4(c4[v], sh4[v], sl4[v], negR, nhi, nlo, t01, t23);
        acc += (ex2(t01.x) + ex2(t01.y)) + (ex2(t23.x) + ex2(t23.y));
      }
    }
  }
  return make_float2(R, warp_sum(acc));
}

__device__ __forceinline__ float2 merge_pieces_t(const float2* p, int n, int stride) {
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

__device__ void consumers(const ApplyArgs& A, char* stages, char* tbufs, Ring* ring, float2* comb) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = warp / kGroupWarps, gw = warp % kGroupWarps;  // group, warp within the group
  uint32_t it = 0, tc = 0;
  bool dead = false;  // warp-uniform: a wait ran out; skip work, keep the barrier schedule
  auto ready = [&](uint64_t* bar, uint32_t parity) {
    if (!dead && (ring->abort || !mbar_wait_warp(bar, parity))) {
      dead = true;
      if (lane == 0) {
        ring->abort = 1;
        atomicOr(A.err, 2);
      }
    }
    return !dead;
  };
  for (int ti = blockIdx.x; ti < A.ntasks; ti += gridDim.x) {
    const StreamTask t = A.stasks[ti];
    if (skipped(A, t)) continue;
    const int b = tc & 1;
    const bool vec_ok = ready(&ring->tfull[b], (tc >> 1) & 1);
    ++tc;
    const TaskBuf tb = task_buf(tbufs, b);
    const int ns = task_stages(t);
    if (t.kind == TASK_ROW) {
      for (int s = 0; s < ns; ++s, ++it) {
        if ((it % kGroups) != grp) continue;  // the other group's stage (and slot)
        const int slot = it % kStages;
        const bool ok = ready(&ring->full[slot], (it / kStages) & 1) && vec_ok;
        const int r = 8 * s + gw;
        if (ok && r < t.ocount) {
          const float2 pr = consume_row(t, reinterpret_cast<const float*>(stages + slot * kStageBytes + gw * 4096),
                                        tb.hh, tb.hl, tb.fr[r]);
          if (lane == 0) A.part32[t.out_off + r] = pr;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&ring->empty[slot]);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&ring->tempty[b]);
    } else {
      const float2 nhi = make_float2(-t.s2, -t.s2), nlo = make_float2(-t.s2_lo, -t.s2_lo);
      const int c0 = 4 * lane;
      const bool lane_on = c0 < t.ocount;
      float R[4], acc[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        R[k] = (vec_ok && c0 + k < t.ocount) ? tb.fr[c0 + k] : 0.f;
        acc[k] = 0.f;
      }
      for (int s = 0; s < ns; ++s, ++it) {
        if ((it % kGroups) != grp) continue;
        const int slot = it % kStages;
        if (!(ready(&ring->full[slot], (it / kStages) & 1) && vec_ok)) {
          __syncwarp();
          if (lane == 0) mbar_arrive(&ring->empty[slot]);
          continue;
        }
        const char* stage = stages + slot * kStageBytes;
        const int rbase = 64 * s + 8 * gw;  // task-relative first row of this warp
        const int nr = lane_on ? min(8, t.rcount - rbase) : 0;  // rows of this warp in the stage
        float cm[4] = {-kInf, -kInf, -kInf, -kInf};
        float2 a01 = make_float2(0.f, 0.f), a23 = make_float2(0.f, 0.f);
        {
          const float2 nR01 = make_float2(-R[0], -R[1]), nR23 = make_float2(-R[2], -R[3]);
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            if (i < nr) {
              const float4 c = reinterpret_cast<const float4*>(stage + (8 * gw + i) * 512)[lane];
              const float hv = tb.hh[rbase + i], lv = tb.hl[rbase + i];
              const float2 h2 = make_float2(hv, hv), l2 = make_float2(lv, lv);
              float2 t01 = fma2(make_float2(c.x, c.y), nhi, add2(h2, nR01));
              float2 t23 = fma2(make_float2(c.z, c.w), nhi, add2(h2, nR23));
              t01 = add2(fma2(make_float2(c.x, c.y), nlo, t01), l2);
              t23 = add2(fma2(make_float2(c.z, c.w), nlo, t23), l2);
              cm[0] = fmaxf(cm[0], t01.x);
              cm[1] = fmaxf(cm[1], t01.y);
              cm[2] = fmaxf(cm[2], t23.x);
              cm[3] = fmaxf(cm[3], t23.y);
              a01 = add2(a01, make_float2(ex2(t01.x), ex2(t01.y)));
              a23 = add2(a23, make_float2(ex2(t23.x), ex2(t23.y)));
            }
          }
        }
        float part[4] = {a01.x, a01.y, a23.x, a23.y};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if ((cm[k] > 0.5f || (acc[k] == 0.f && cm[k] < -kWindowT)) && cm[k] > -kInf) {
            // rare after the first half-steps: move the frame, sum this column's rows again
            const float Rn = R[k] + quant(cm[k]);
            acc[k] = acc[k] == 0.f ? 0.f : acc[k] * ex2(R[k] - Rn);
            R[k] = Rn;
            float sk = 0.f;
            for (int i = 0; i < nr; ++i) {
              const float ck = reinterpret_cast<const float*>(stage + (8 * gw + i) * 512)[4 * lane + k];
              float tk = fmaf(-ck, t.s2, tb.hh[rbase + i] - Rn);
              tk = fmaf(-ck, t.s2_lo, tk);
              sk += ex2(tk + tb.hl[rbase + i]);
            }
            part[k] = sk;
          }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[k] += part[k];
        __syncwarp();
        if (lane == 0) mbar_arrive(&ring->empty[slot]);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&ring->tempty[b]);
      consumers_sync();  // every warp is done reading comb of the previous COL task
#pragma unroll
      for (int k = 0; k < 4; ++k) comb[warp * kColCols + c0 + k] = make_float2(R[k], acc[k]);
      consumers_sync();
      if (!dead)
        for (int c = threadIdx.x; c < t.ocount; c += kConsumers * 32)
          A.part32[t.out_off + c] = merge_pieces_t(comb + c, kConsumers, kColCols);
    }
  }
}

constexpr size_t kTmaSmem = (size_t)kStages * kStageBytes + 2 * (size_t)kTaskBufBytes +
                            (size_t)kConsumers * kColCols * sizeof(float2);

__global__ void __launch_bounds__(kTmaThreads, 1) apply_dense_tma_kernel(ApplyArgs A) {
  // every problem retired or in a BF16 phase: nothing to apply (the same for every CTA)
  if (A.fp32_live && *((volatile const int32_t*)A.fp32_live) <= 0) return;
  extern __shared__ __align__(128) char dyn[];
  char* stages = dyn;                                 // kStages x 32 KB
  char* tbufs = dyn + kStages * kStageBytes;          // 2 x (hh, hl, frames)
  float2* comb = reinterpret_cast<float2*>(tbufs + 2 * kTaskBufBytes);  // [16][128]
  __shared__ Ring ring;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&ring.full[i], 1);
      mbar_init(&ring.empty[i], kGroupWarps);  // one group consumes a stage
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&ring.tfull[i], 1);
      mbar_init(&ring.tempty[i], kConsumers);
    }
    ring.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // task buffers start at zero: entries past a task's vectors then hold finite
  // or -inf operands, never NaN (rows read them against +inf costs)
  for (int i = threadIdx.x; i < 2 * kTaskBufBytes / 4; i += kTmaThreads) reinterpret_cast<float*>(tbufs)[i] = 0.f;
  __syncthreads();
  if ((int)(threadIdx.x >> 5) == kConsumers)
    producer(A, stages, tbufs, &ring);
  else
    consumers(A, stages, tbufs, &ring, comb);
}

}  // namespace

// Function attributes are per device: the answer is kept per device id.
bool apply_tma_available() {
  constexpr int kMaxDevices = 64;
  static std::atomic<int> state[kMaxDevices];  // 0 unknown, 1 available, 2 not
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return false;
  int st = state[dev].load();
  if (st == 0) {
    int blocks = 0;
    const bool ok =
        cudaFuncSetAttribute(apply_dense_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTmaSmem) ==
            cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, apply_dense_tma_kernel, kTmaThreads, kTmaSmem) ==
            cudaSuccess &&
        blocks >= 1;
    st = ok ? 1 : 2;
    state[dev].store(st);
  }
  return st == 1;
}

cudaError_t launch_apply_tma(const ApplyArgs& a, int grid, cudaStream_t s) {
  if (a.ntasks <= 0) return cudaSuccess;
  if (!a.stasks || !apply_tma_available()) return cudaErrorInvalidConfiguration;
  apply_dense_tma_kernel<<<grid, kTmaThreads, kTmaSmem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace treeot
