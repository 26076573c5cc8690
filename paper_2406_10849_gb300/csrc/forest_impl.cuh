// The persistent forest kernel (see forest.cu for the schedule).  Included by
// forest_d1.cu, forest_d2.cu and forest_d3.cu, each instantiating one point
// dimension FOREST_D, so the three compile in parallel.
#pragma once
#include <cmath>

#include "forest.h"
#include "node_chunk.cuh"
#include "recomp_task.cuh"

namespace treeot {
namespace {

constexpr uint64_t kForestWaitNs = 1000000000ull;  // 1 s of wall time per wait

__device__ __forceinline__ uint64_t forest_clock() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// bounded wait for *p >= target (one thread); false when it ran out
__device__ bool forest_wait(const int32_t* p, int32_t target) {
  if (*((volatile const int32_t*)p) >= target) return true;
  const uint64_t t0 = forest_clock();
  uint32_t ns = 32;
  for (uint32_t it = 0; it < (1u << 26); ++it) {
    if (*((volatile const int32_t*)p) >= target) return true;
    if ((it & 63u) == 63u && forest_clock() - t0 > kForestWaitNs) return false;
    __nanosleep(ns);
    if (ns < 1024) ns <<= 1;
  }
  return false;
}

// items of problem p of a colour-alternating run: count through half-step k
// (k + 1 half-steps starting with colour c0), per-colour counts n[0], n[1]
__device__ __forceinline__ int32_t through(int64_t k, int32_t n_c0, int32_t n_c1) {
  if (k < 0) return 0;
  const int64_t m = k + 1;
  return (int32_t)(((m + 1) / 2) * n_c0 + (m / 2) * n_c1);
}

// One apply item (a recomputed-cost task of colour A at half-step h); returns
// -1 when the wait for its problem ran out, else 0 or 1 (work done).
template <int D, bool EXACT>
__device__ __forceinline__ int apply_item(const ForestArgs& F, const ApplyArgs& A, int idx, int h, float* sm) {
  __shared__ int s_go;
  const int tid = threadIdx.x;
  const Task task = A.tasks[idx];
  const int p = A.dedges[task.dedge].prob;
  if (tid == 0) {
    const int32_t* cnt = F.cnt + 4 * p;
    int go = ((volatile const int32_t*)A.done)[p] == 0 ? 1 : 0;
    if (go) {
      if (!forest_wait(&F.nod_done[p], through(h - 1, cnt[2 + F.c0], cnt[3 - F.c0]))) {
        atomicOr(F.err, 2);
        go = -1;
      }
      __threadfence();
      if (go == 1 && ((volatile const int32_t*)A.done)[p] != 0) go = 0;  // it may have retired meanwhile
    }
    s_go = go;
  }
  __syncthreads();
  const int go = s_go;
  if (go == 1) {
    if (EXACT && A.exact[p])
      recomp_task_exact<D>(A, task, sm);
    else
      recomp_task<D>(A, task, sm);
  }
  __syncthreads();
  if (tid == 0 && go >= 0) {
    __threadfence();
    atomicAdd(&F.app_done[p], 1);
  }
  return go;
}

// One node item (chunk idx of colour N at half-step h); returns -1 when the wait ran out.
__device__ __forceinline__ int node_item(const ForestArgs& F, const NodeArgs& N, int idx, int h, int64_t hs0,
                                         unsigned char* node_sm, double* red) {
  __shared__ int s_go;
  const int tid = threadIdx.x;
  const NodeChunk c = N.chunks[idx];
  const int p = N.nodes[c.node].prob;
  if (tid == 0) {
    const int32_t* cnt = F.cnt + 4 * p;
    int go = 1;
    if (((volatile const int32_t*)N.done)[p] == 0 && !forest_wait(&F.app_done[p], through(h, cnt[F.c0], cnt[1 - F.c0]))) {
      atomicOr(F.err, 2);
      go = -1;
    }
    __threadfence();
    s_go = go;
  }
  __syncthreads();
  const int go = s_go;
  if (go == 1) node_chunk_item<false>(N, c, hs0 + h, node_sm, red);  // skips retired problems itself
  __syncthreads();
  if (tid == 0 && go == 1 && !F.test_stall) {
    __threadfence();
    atomicAdd(&F.nod_done[p], 1);
  }
  return go;
}

template <int D, bool EXACT, int MINB>
__global__ void __launch_bounds__(kApplyThreads, MINB) forest_kernel(ForestArgs F) {
  extern __shared__ __align__(16) unsigned char node_sm[];
  __shared__ __align__(16) float sm[16 * kApplyThreads + 2 * 4 * kApplyThreads];  // apply staging, 24 KB
  __shared__ double red[kNodeThreads / 32];
  __shared__ int s_t;
  const int tid = threadIdx.x;
  const int c0 = F.c0, c1 = 1 - F.c0;
  const int A0 = F.ap[c0].ntasks, N0 = F.nd[c0].nchunks, A1 = F.ap[c1].ntasks, N1 = F.nd[c1].nchunks;
  const int64_t per2 = (int64_t)A0 + N0 + A1 + N1;
  const int64_t total = (int64_t)(F.G / 2) * per2 + (F.G % 2 ? (int64_t)A0 + N0 : 0);
  const int64_t hs0 = *((volatile const int64_t*)F.hs);
  bool abort = false;
  for (;;) {
    if (tid == 0) s_t = atomicAdd(&F.ctl[0], 1);
    __syncthreads();
    const int64_t t = s_t;
    __syncthreads();
    if (t >= total || abort) break;
    const int64_t pair = t / per2;
    int64_t r = t - pair * per2;
    int h = (int)(2 * pair), kind, idx;
    if (r < A0) {
      kind = 0, idx = (int)r;
    } else if (r < A0 + N0) {
      kind = 1, idx = (int)(r - A0);
    } else if (r < A0 + N0 + A1) {
      kind = 0, idx = (int)(r - A0 - N0), h += 1;
    } else {
      kind = 1, idx = (int)(r - A0 - N0 - A1), h += 1;
    }
    const int colour = (c0 + h) & 1;
    // the per-colour tables are selected with constant indices (no local copy of the arguments)
    int go;
    if (kind == 0)
      go = colour ? apply_item<D, EXACT>(F, F.ap[1], idx, h, sm) : apply_item<D, EXACT>(F, F.ap[0], idx, h, sm);
    else
      go = colour ? node_item(F, F.nd[1], idx, h, hs0, node_sm, red) : node_item(F, F.nd[0], idx, h, hs0, node_sm, red);
    if (go < 0) abort = true;
  }
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(&F.ctl[1], 1) == (int)gridDim.x - 1) {
      for (int p = 0; p < F.nprob; ++p) {
        F.app_done[p] = 0;
        F.nod_done[p] = 0;
      }
      F.ctl[0] = 0;
      F.ctl[1] = 0;
      *F.hs += F.G;
      __threadfence();
    }
  }
}

// the instantiations of this translation unit's dimension
void* forest_pick(bool exact, int minb) {
  if (exact) return reinterpret_cast<void*>(forest_kernel<FOREST_D, true, 2>);
  if (minb == 3) return reinterpret_cast<void*>(forest_kernel<FOREST_D, false, 3>);
  return reinterpret_cast<void*>(forest_kernel<FOREST_D, false, 2>);
}

}  // namespace

template <>
void* forest_kernel_ptr<FOREST_D>(bool exact, int minb) {
  return forest_pick(exact, minb);
}

}  // namespace treeot
