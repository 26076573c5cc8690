// Edge apply in FP64 (precision mode for small problems that must reach
// stopping tolerances far below FP32 resolution).  Same tasks as the FP32
// kernel; one warp per output x, lanes stride over the whole reduction range:
//   m_(j,k)(x) = LSE_y [ (f_(k,j)(y) - C(x,y)) / eps + log gamma_k(y) ]    (base e)
// written as a (max, sum) pair with a single split.
#include <cmath>

#include "internal.h"
#include "ptx.cuh"

namespace treeot {
namespace {

__device__ __forceinline__ double cost_f64(const ApplyArgs& A, const EdgeD& e, const DEdgeD& d, const ProbD& P,
                                           int kind, int x, int y) {
  if (kind == TASK_ROW) return (double)e.C[(int64_t)x * e.ld + y];
  if (kind == TASK_COL) return (double)e.C[(int64_t)y * e.ld + x];
  const NodeD own = A.nodes[d.owner];
  const NodeD nb = A.nodes[d.nbr];
  const float* p = A.coords + own.coord_off + (int64_t)x * P.dim;
  const float* q = A.coords + nb.coord_off + (int64_t)y * P.dim;
  double c = 0.0;
  for (int k = 0; k < P.dim; ++k) {
    const double dd = (double)p[k] - (double)q[k];
    c += dd * dd;
  }
  return P.cost_scale * c;
}

__global__ void __launch_bounds__(kApplyThreads) apply_f64_kernel(ApplyArgs A) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int ti = blockIdx.x; ti < A.ntasks; ti += gridDim.x) {
    const Task t = A.tasks[ti];
    const DEdgeD d = A.dedges[t.dedge];
    if (A.done[d.prob]) continue;
    const ProbD P = A.probs[d.prob];
    const EdgeD e = A.edges[d.edge];
    const NodeD own = A.nodes[d.owner];
    const NodeD nb = A.nodes[d.nbr];
    for (int r = warp; r < t.ocount; r += kApplyThreads / 32) {
      const int x = t.o0 + r;
      double M = -INFINITY, S = 0.0;
      for (int y = t.r0 + lane; y < t.r0 + t.rcount; y += 32) {
        const double a = (A.f[d.rev_off + y] - cost_f64(A, e, d, P, t.kind, x, y)) * P.inv_eps +
                         A.logg[nb.node_off + y];
        if (a > M) {
          S = S * exp(M - a) + 1.0;
          M = a;
        } else if (a > -INFINITY) {
          S += exp(a - M);
        }
      }
      const double Mw = warp_max_d(M);
      S = (M > -INFINITY) ? S * exp(M - Mw) : 0.0;
      S = warp_sum_d(S);
      if (lane == 0) A.part64[d.part_off + (int64_t)t.split * own.n + x] = make_double2(Mw, S);
    }
  }
}

}  // namespace

cudaError_t launch_apply_f64(const ApplyArgs& a, int grid, cudaStream_t s) {
  if (a.ntasks <= 0) return cudaSuccess;
  apply_f64_kernel<<<grid, kApplyThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace treeot
