// Persistent forest launch (forest.cu): one launch runs G half-steps of every
// problem of a batch whose costs are all recomputed from points of one
// dimension, with per-problem phase counters instead of launch boundaries.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"

namespace treeot {

struct ForestArgs {
  ApplyArgs ap[2];        // per colour: that colour's recomputed-cost tasks (cost-sorted)
  NodeArgs nd[2];         // per colour: that colour's node-update chunks
  const int32_t* cnt;     // per problem: apply tasks of colour 0, of colour 1, node chunks of colour 0, of 1
  int32_t* app_done;      // per problem: apply items finished in this launch
  int32_t* nod_done;      // per problem: node items finished in this launch
  int32_t* ctl;           // [0] next ticket, [1] CTAs finished (reset by the last CTA)
  int32_t* err;           // bit 1 (value 2): a bounded wait ran out
  int64_t* hs;            // half-steps done; advanced by G by the last CTA
  int32_t nprob;
  int32_t G;              // half-steps in this launch
  int32_t c0;             // colour of the first of them
  int32_t test_stall;     // test hook: node items never report completion, so waits run out
};

// the kernel of dimension D (defined in forest_dD.cu): exact distances (2-CTA
// register budget) or the plain recomputation at minb (2 or 3) CTAs per SM
template <int D>
void* forest_kernel_ptr(bool exact, int minb);

// D: point dimension of every problem; exact: some problem recomputes squared
// distances exactly (always the 2-CTA register budget); minb: 2 or 3 CTAs per SM
// register budget; smem: dynamic shared memory (the node update's largest chunk).
cudaError_t launch_forest(const ForestArgs& a, int D, bool exact, int minb, uint32_t smem, int grid,
                          cudaStream_t s);
// CTAs per SM the persistent kernel reaches with that dynamic shared memory (0 if none)
int forest_ctas_per_sm(int D, bool exact, int minb, uint32_t smem);

}  // namespace treeot
