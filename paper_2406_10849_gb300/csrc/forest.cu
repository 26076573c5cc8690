// Persistent forest launch: G half-steps of a batch of independent trees in
// one launch, the problems advancing on their own phase counters.
//
// Work items are numbered ("tickets") in schedule order: for each half-step h
// of the launch, every recomputed-cost apply task of colour c(h) (sorted by
// cost, as in the per-half-step launch), then every node-update chunk of that
// colour.  A CTA takes the next ticket from an atomic counter and waits only
// for its own problem:
//   apply task of problem p at half-step h:  p's node chunks of half-steps < h done
//   node chunk of problem p at half-step h:  p's apply tasks of half-steps <= h done
// (per-problem counters of finished items; the targets follow from p's item
// counts per colour, the colours alternating).  Problems are independent, so a
// small tree's node update runs while large trees still apply, and no launch
// boundary separates half-steps.  A ticket is only ever taken by a running
// CTA and only waits for smaller tickets, so the smallest unfinished ticket
// never waits: progress does not depend on how many CTAs are resident.  Every
// wait is bounded (kForestWaitNs of %globaltimer, with back-off and an
// iteration cap); a wait that runs out sets an error bit, and the CTA stops
// taking tickets, so every other wait runs out in turn and the launch ends.
// A retired problem's items do no work and do not wait.  Data produced inside
// the launch is read with ordinary loads after the waiting thread's acquire
// fence and the block barrier (no read-only-path loads on the apply side).
// The last CTA to finish resets the counters and advances the half-step count.
#include "forest.h"

namespace treeot {

int forest_ctas_per_sm(int D, bool exact, int minb, uint32_t smem) {
  const void* fn = D == 1 ? forest_kernel_ptr<1>(exact, minb)
                 : D == 2 ? forest_kernel_ptr<2>(exact, minb)
                 : D == 3 ? forest_kernel_ptr<3>(exact, minb) : nullptr;
  if (!fn) return 0;
  // static (24 KB of apply staging) plus dynamic shared memory may pass the default 48 KB
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, kApplyThreads, smem) != cudaSuccess) return 0;
  return n;
}

cudaError_t launch_forest(const ForestArgs& a, int D, bool exact, int minb, uint32_t smem, int grid,
                          cudaStream_t s) {
  if (a.G <= 0) return cudaSuccess;
  if (D < 1 || D > 3 || grid < 1) return cudaErrorInvalidValue;
  const void* fn = D == 1 ? forest_kernel_ptr<1>(exact, minb)
                 : D == 2 ? forest_kernel_ptr<2>(exact, minb) : forest_kernel_ptr<3>(exact, minb);
  const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void* args[] = {const_cast<ForestArgs*>(&a)};
  return cudaLaunchKernel(fn, dim3(grid), dim3(kApplyThreads), args, smem, s);
}

}  // namespace treeot
