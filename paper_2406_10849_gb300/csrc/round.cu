// Rounding to feasible plans: the rounding algorithm of Sec. 3.1 (each plan of
// the colour class S that missed its marginals in the last half-step goes through
// Altschuler, Weed and Rigollet's Algorithm 2), with the transport cost of the
// rounded plans and the quantities of lemmas lem:round / lem:round_applied.
//
// For a plan F = B_(j,k), j in S (rows), k the other endpoint (columns), with
// row target t (the marginal j must get: mu_j, or qbar_j = mean_k B_(j,k) 1 for
// a free j) and column target c (the marginal k already has):
//   x   = min(t / F 1, 1)          F'  = diag(x) F          (rows scaled down to t)
//   y   = min(c / F'^T 1, 1)       F'' = F' diag(y)         (columns scaled down to c)
//   err_r = t - F'' 1,  err_c = c - F''^T 1,  E = ||err_r||_1
//   B^  = F'' + err_r err_c^T / E
// so B^ 1 = t and B^T 1 = c.  The paper takes c = F^T 1, which the last
// half-step made equal to k's marginal (thm:tree_dual_var); in FP32 iterates that
// holds only to the iterate's accuracy, so here c is k's marginal itself (mu_k,
// or the mean of k's plan marginals), and every target is scaled to unit mass
// (exactly 1 by lemma cor:tree_mass).  Then the rounded plans meet every
// constraint of the unregularised problem to FP64 rounding; in exact arithmetic
// y = 1 and this is the paper's rounding.
//
// The rounded plans are never stored: they are (x, y, err_r, E) plus the
// potentials, and <C, B^> = <C, F''> + err_r^T C err_c / E.  Entries are the
// double-float plan entries of the check (FP32 pipe; FP64 handles: FP64), every
// sum over them is FP64.  Passes over the plans (one CTA per task of 64 rows of
// one plan, rows on S), with per-point steps between them:
//   1  F 1, F^T 1, <C, F>, ||F||_1     -> targets t and c, row scales x
//   2  F'^T 1                          -> column scales y
//   3  F'' 1, <C, F''>                 -> err_r, E
//   4  err_r^T C err_c, max |C|        (no exponentials)
//   5  (one edge, on request) B^ written out in the edge's stored orientation
#include <cmath>

#include "internal.h"
#include "plan_entry.cuh"
#include "ptx.cuh"
#include "round.h"

namespace treeot {
namespace {

constexpr int kRndRows = 8;  // rows per warp (task = 8 warps x 8 rows)

// FP64 handles: a(x) = f'/eps - Z_owner + log gamma_owner of the directed edge stored at off
__device__ __forceinline__ double a64_of(const RoundArgs& A, int64_t off, int32_t owner, const NodeD& own,
                                         double inv_eps, int x) {
  const double lg = A.logg[own.node_off + x];
  if (lg == -INFINITY) return -INFINITY;
  return A.f[off + x] * inv_eps - A.Z[owner] + lg;
}

// the plan entry (row i on the task's owner, column y on its neighbour) as a double;
// cst returns C(i,y) (cost units, +inf allowed)
template <bool F64>
__device__ __forceinline__ double round_entry(const ProbD& P, float rah, float ral, double ra64, float bh, float bl,
                                              double b64, DF c, float kh, float kl, double cscale, double& cst) {
  cst = ((double)c.hi + (double)c.lo) * cscale;
  if (F64) {
    if (!(ra64 > -INFINITY) || !(b64 > -INFINITY) || cst == INFINITY) return 0.0;
    return exp(ra64 + b64 - cst * P.inv_eps);
  }
  float cu;
  return (double)plan_entry(rah, ral, bh, bl, c, kh, kl, cu);
}

template <int PASS, bool F64>
__global__ void __launch_bounds__(256) round_pass_kernel(RoundArgs A) {
  __shared__ double s_col[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int ti = blockIdx.x; ti < A.ntasks; ti += gridDim.x) {
    const RoundTask t = A.tasks[ti];
    const DEdgeD d = A.dedges[t.dedge];
    const EdgeD e = A.edges[d.edge];
    const ProbD P = A.probs[d.prob];
    const NodeD nj = A.nodes[d.owner], nk = A.nodes[d.nbr];
    // cost rows on the owner: C itself (owner = row node), C^T when kept, else C's columns
    const bool own_rows = d.dir == 0 || e.CT != nullptr;
    const float* Cm = d.dir == 0 ? e.C : (e.CT ? e.CT : e.C);
    const int64_t cld = d.dir == 0 ? e.ld : (e.CT ? e.ldt : e.ld);
    const double cscale = P.cost_kind == 0 ? 1.0 : P.cost_scale;
    const double kd = cscale * P.inv_eps;
    const float kh = (float)kd, kl = (float)(kd - (double)kh);
    const int D = P.dim;
    const double E = PASS == 5 ? A.edge_acc[kRoundAcc * d.edge + 3] : 0.0;
    float rah[kRndRows], ral[kRndRows], rp[kRndRows][3];
    double ra64[kRndRows], xr[kRndRows], err[kRndRows], racc[kRndRows], tacc[kRndRows];
    double cmax = 0.0;
#pragma unroll
    for (int r = 0; r < kRndRows; ++r) {
      const int ir = warp * kRndRows + r;
      const bool on = ir < t.ocount;
      const int i = t.o0 + (on ? ir : 0);
      rah[r] = on && !F64 ? A.ah[d.off + i] : -INFINITY;
      ral[r] = on && !F64 ? A.al[d.off + i] : 0.f;
      ra64[r] = on && F64 ? a64_of(A, d.off, d.owner, nj, P.inv_eps, i) : -INFINITY;
      for (int k = 0; k < 3; ++k)
        rp[r][k] = (nj.coord_off >= 0 && k < D) ? A.coords[nj.coord_off + (int64_t)i * D + k] : 0.f;
      xr[r] = (PASS >= 2 && on) ? A.xy[d.off + i] : 0.0;
      err[r] = (PASS >= 4 && on) ? A.er[d.off + i] : 0.0;
      racc[r] = tacc[r] = 0.0;
    }
    for (int y0 = 0; y0 < nk.n; y0 += 32) {
      const int y = y0 + lane;
      const bool on = y < nk.n;
      const float bh = on && !F64 ? A.ah[d.rev_off + y] : -INFINITY;
      const float bl = on && !F64 ? A.al[d.rev_off + y] : 0.f;
      const double b64 = on && F64 ? a64_of(A, d.rev_off, d.nbr, nk, P.inv_eps, y) : -INFINITY;
      float pb[3] = {0.f, 0.f, 0.f};
      if (on && nk.coord_off >= 0)
        for (int k = 0; k < D; ++k) pb[k] = A.coords[nk.coord_off + (int64_t)y * D + k];
      const double ycol = (PASS >= 3 && on) ? A.xy[d.rev_off + y] : 0.0;
      // err_c = c - F''^T 1, F''^T 1 = y F'^T 1
      const double ecy = (PASS >= 4 && on) ? fmax(A.tgt[d.rev_off + y] - ycol * A.s2[d.rev_off + y], 0.0) : 0.0;
      double cs = 0.0;
      if (on) {
#pragma unroll
        for (int r = 0; r < kRndRows; ++r) {
          const int ir = warp * kRndRows + r;
          if (ir >= t.ocount) continue;
          const int i = t.o0 + ir;
          DF c;
          if (P.cost_kind == 0)
            c = {own_rows ? Cm[(int64_t)i * cld + y] : Cm[(int64_t)y * cld + i], 0.f};
          else
            c = sq_dist_df(D, rp[r], pb);
          if (PASS == 4) {
            const double C = ((double)c.hi + (double)c.lo) * cscale;
            if (C != INFINITY) cmax = fmax(cmax, fabs(C));
            const double w = err[r] * ecy;
            if (w > 0.0) tacc[r] += w * C;
            continue;
          }
          double cst;
          const double B = round_entry<F64>(P, rah[r], ral[r], ra64[r], bh, bl, b64, c, kh, kl, cscale, cst);
          if (PASS == 1) {
            racc[r] += B;
            if (B > 0.0) tacc[r] += B * cst;
            cs += B;
          } else if (PASS == 2) {
            cs += xr[r] * B;
          } else if (PASS == 3) {
            const double B2 = xr[r] * B * ycol;
            racc[r] += B2;
            if (B2 > 0.0) tacc[r] += B2 * cst;
          } else {  // PASS 5: the rounded plan, in the edge's stored orientation (rows = node a)
            const double G = xr[r] * B * ycol + (E > 0.0 ? err[r] * ecy / E : 0.0);
            const int64_t o = d.dir == 0 ? (int64_t)i * A.plan_ld + y : (int64_t)y * A.plan_ld + i;
            A.plan_out[o] = G;
          }
        }
      }
      if (PASS == 1 || PASS == 2) {  // column sums: combined across the warps, one FP64 atomic per column
        s_col[warp][lane] = cs;
        __syncthreads();
        if (warp == 0 && on) {
          double v = 0.0;
#pragma unroll
          for (int w = 0; w < 8; ++w) v += s_col[w][lane];
          if (v != 0.0) atomicAdd(PASS == 1 ? &A.rsum[d.rev_off + y] : &A.s2[d.rev_off + y], v);
        }
        __syncthreads();
      }
    }
    if (PASS == 2 || PASS == 5) continue;
    double tsum = 0.0, msum = 0.0;
#pragma unroll
    for (int r = 0; r < kRndRows; ++r) {
      const int ir = warp * kRndRows + r;
      const double tr = warp_sum_d(tacc[r]);
      if (PASS == 1 || PASS == 3) {
        const double row = warp_sum_d(racc[r]);
        // each row belongs to one task
        if (lane == 0 && ir < t.ocount) (PASS == 1 ? A.rsum : A.s2)[d.off + t.o0 + ir] = row;
        if (ir < t.ocount) msum += row;
      }
      if (ir < t.ocount) tsum += tr;
    }
    double* acc = A.edge_acc + kRoundAcc * d.edge;
    if (lane == 0 && tsum != 0.0) atomicAdd(&acc[PASS == 1 ? 0 : PASS == 3 ? 1 : 2], tsum);
    if (PASS == 1 && lane == 0 && msum != 0.0) atomicAdd(&acc[5], msum);
    if (PASS == 4) {
      cmax = warp_max_d(cmax);
      if (lane == 0 && cmax > 0.0)
        atomicMax((unsigned long long*)&acc[4], (unsigned long long)__double_as_longlong(cmax));
    }
  }
}

// Per-point steps, one CTA row per directed edge (grid.y), points over grid.x.
//   STEP 1 (every directed edge): target = the owner's marginal at unit mass (mu_o / sum mu_o,
//          or the mean of o's plan marginals over the mean of its plans' masses); S side: x.
//   STEP 2 (directed edges not owned by S): y = min(c / F'^T 1, 1).
//   STEP 3 (directed edges owned by S): err_r = t - F'' 1, E += sum err_r.
template <int STEP>
__global__ void round_points_kernel(RoundArgs A, int32_t d0) {
  __shared__ double red[8];
  const DEdgeD d = A.dedges[d0 + blockIdx.y];
  const NodeD no = A.nodes[d.owner];
  const bool in_s = no.colour == A.side[d.prob];
  if ((STEP == 2 && in_s) || (STEP == 3 && !in_s)) return;  // block-uniform
  double mass = 1.0;
  if (STEP == 1) {
    if (no.fixed) {
      mass = A.nmass[d.owner];
    } else {
      mass = 0.0;
      for (int k = 0; k < no.deg; ++k)
        mass += A.edge_acc[kRoundAcc * A.dedges[A.node_dedges[no.dedge_begin + k]].edge + 5];
      mass /= no.deg;
    }
  }
  double esum = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < no.n; i += gridDim.x * blockDim.x) {
    if (STEP == 1) {
      double tg;
      if (no.fixed) {
        tg = A.mu[no.node_off + i];
      } else {
        double q = 0.0;
        for (int k = 0; k < no.deg; ++k) q += A.rsum[A.dedges[A.node_dedges[no.dedge_begin + k]].off + i];
        tg = q / no.deg;
      }
      tg = mass > 0.0 ? tg / mass : tg;
      A.tgt[d.off + i] = tg;
      if (in_s) {
        const double r = A.rsum[d.off + i];
        A.xy[d.off + i] = r > 0.0 ? fmin(tg / r, 1.0) : 1.0;
      }
    } else if (STEP == 2) {
      const double c1 = A.s2[d.off + i];
      A.xy[d.off + i] = c1 > 0.0 ? fmin(A.tgt[d.off + i] / c1, 1.0) : 1.0;
    } else {
      const double er = fmax(A.tgt[d.off + i] - A.s2[d.off + i], 0.0);
      A.er[d.off + i] = er;
      esum += er;
    }
  }
  if (STEP != 3) return;
  esum = warp_sum_d(esum);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = esum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
    if (tot != 0.0) atomicAdd(&A.edge_acc[kRoundAcc * d.edge + 3], tot);
  }
}

template <int PASS>
void pass(const RoundArgs& a, bool f64, int grid, cudaStream_t s) {
  if (f64)
    round_pass_kernel<PASS, true><<<grid, 256, 0, s>>>(a);
  else
    round_pass_kernel<PASS, false><<<grid, 256, 0, s>>>(a);
}

template <int STEP>
void points(const RoundArgs& a, cudaStream_t s) {
  for (int32_t d0 = 0; d0 < a.ndedges; d0 += 65535) {
    const int32_t cnt = a.ndedges - d0 < 65535 ? a.ndedges - d0 : 65535;
    round_points_kernel<STEP><<<dim3(4, cnt), 256, 0, s>>>(a, d0);
  }
}

int grid_for(int ntasks) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return ntasks < 4 * sms ? ntasks : 4 * sms;
}

}  // namespace

cudaError_t launch_round(const RoundArgs& a, bool f64, cudaStream_t s) {
  if (a.ntasks <= 0) return cudaSuccess;
  const int grid = grid_for(a.ntasks);
  pass<1>(a, f64, grid, s);
  points<1>(a, s);
  pass<2>(a, f64, grid, s);
  points<2>(a, s);
  pass<3>(a, f64, grid, s);
  points<3>(a, s);
  pass<4>(a, f64, grid, s);
  return cudaGetLastError();
}

cudaError_t launch_round_plan(const RoundArgs& a, bool f64, cudaStream_t s) {
  if (a.ntasks <= 0) return cudaSuccess;
  pass<5>(a, f64, grid_for(a.ntasks), s);
  return cudaGetLastError();
}

}  // namespace treeot
