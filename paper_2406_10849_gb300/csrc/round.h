// Rounding to feasible plans (round.cu): plan tables of the rounding passes.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"

namespace treeot {

// Rounding (round.cu).  A task is 64 rows of one plan with its rows on the
// colour class S being rounded (the directed edge's owner is in S).
constexpr int kRoundAcc = 6;  // per edge: <C,F>, <C,F''>, err_r^T C err_c, E = ||err_r||_1, C_inf (bits), ||F||_1
struct RoundTask {
  int32_t dedge;        // directed edge j -> k, j in S
  int32_t o0, ocount;   // rows (points of j)
  int32_t pad;
};
struct RoundArgs {
  const RoundTask* tasks;
  int32_t ntasks;
  const DEdgeD* dedges;
  int32_t ndedges;
  const EdgeD* edges;
  const NodeD* nodes;
  const ProbD* probs;
  const int32_t* node_dedges;
  const int32_t* side;    // per problem: the colour class S being rounded
  const double* nmass;    // per node: sum of mu (fixed nodes)
  const float* ah;        // FP32 handles: check operand f/eps - Z + log gamma as (hi, lo)
  const float* al;
  const double* f;        // FP64 handles: potentials f', Z and log gamma read directly
  const double* Z;
  const double* logg;
  const double* mu;       // node-level mu (fixed nodes)
  const float* coords;
  // arenas (layout of the potentials): "S" = offsets of directed edges owned by S (rows),
  // "K" = offsets of the other directed edges (columns)
  double* rsum;           // S: F 1;  K: F^T 1
  double* tgt;            // S: row target;  K: column target (the owner's marginal, unit mass)
  double* xy;             // S: row scale x;  K: column scale y
  double* s2;             // S: F'' 1;  K: F'^T 1
  double* er;             // S: err_r
  double* edge_acc;       // per edge: kRoundAcc doubles
  double* plan_out;       // pass 5: the rounded plan of the tasks' edge, rows = node a, row stride plan_ld
  int64_t plan_ld;
};

// the rounding's passes over the plans and the per-point steps between them
cudaError_t launch_round(const RoundArgs& a, bool f64, cudaStream_t s);
// write out the rounded plans of a.tasks (one edge)
cudaError_t launch_round_plan(const RoundArgs& a, bool f64, cudaStream_t s);

}  // namespace treeot
