// Final check of the current potentials: row and column sums of every plan
//   B_e(x,y) = exp( a(x) + b(y) - C_e(x,y)/eps ),
//   a = f_(a,b)/eps + log gamma_a,  b = f_(b,a)/eps + log gamma_b,
// plus sum_e <C_e,B_e> and ||B_e||_1, accumulated in FP64 per row / column.
//
// GB300 runs FP64 at a small fraction of its FP32 rate, so the exponent is
// formed in double-float arithmetic: a and b arrive as (hi, lo) FP32 pairs
// computed from the FP64 potentials, C/eps is an exact FP32 x (hi, lo) product
// (Dekker's product via FMA), and the sums use Knuth's error-free TwoSum, so
// the exponent is exact to ~1e-12 before one accurate expf of its high part.
// Each plan entry then has ~1e-7 relative error with no systematic part.
#include <cmath>

#include "internal.h"
#include "plan_entry.cuh"
#include "ptx.cuh"

namespace treeot {
namespace {

// One pass over every plan entry.  A ROW task covers up to 64 rows of an edge
// (8 warps x 8 rows); the warps walk the columns together, 32 at a time (a lane
// per column), and evaluate each entry once: row sums (and the transport cost)
// stay in the lanes' registers until the task ends, column sums are combined
// across the warps in shared memory and added to the column marginal with one
// FP64 atomic per column and task.  Sums inside a task use Kahan compensation.
// COL tasks belong to the FP64 check and are skipped here.
constexpr int kChkRows = 8;  // rows per warp

__global__ void __launch_bounds__(256) check_kernel(CheckArgs A) {
  __shared__ float s_col[8][32];
  __shared__ float s_cmp[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int ti = blockIdx.x; ti < A.ntasks; ti += gridDim.x) {
    const Task t = A.tasks[ti];
    if (t.kind != TASK_ROW) continue;  // block-uniform
    const DEdgeD d = A.dedges[t.dedge];
    if (A.mask && !A.mask[d.prob]) continue;  // block-uniform
    const EdgeD e = A.edges[d.edge];
    const ProbD P = A.probs[d.prob];
    const double kd = (P.cost_kind == 0 ? 1.0 : P.cost_scale) * P.inv_eps;
    const float kh = (float)kd, kl = (float)(kd - (double)kh);
    const float cscale = P.cost_kind == 0 ? 1.f : (float)P.cost_scale;
    const NodeD na = A.nodes[e.a], nb = A.nodes[e.b];
    // a-side operand: rows (owner a, dedge 2e) ; b-side: columns (owner b, dedge 2e+1)
    const int64_t a_off = d.dir == 0 ? d.off : d.rev_off;
    const int64_t b_off = d.dir == 0 ? d.rev_off : d.off;
    const int D = P.dim;
    // this warp's rows
    float rah[kChkRows], ral[kChkRows], rp[kChkRows][3];
    float rs[kChkRows], rc[kChkRows], ts[kChkRows], tcmp[kChkRows];
#pragma unroll
    for (int r = 0; r < kChkRows; ++r) {
      const int xr = warp * kChkRows + r;
      const bool on = xr < t.ocount;
      const int x = t.o0 + (on ? xr : 0);
      rah[r] = on ? A.ah[a_off + x] : -INFINITY;
      ral[r] = on ? A.al[a_off + x] : 0.f;
      for (int k = 0; k < 3; ++k) rp[r][k] = (na.coord_off >= 0 && k < D) ? A.coords[na.coord_off + (int64_t)x * D + k] : 0.f;
      rs[r] = rc[r] = ts[r] = tcmp[r] = 0.f;
    }
    for (int y0 = 0; y0 < e.nb; y0 += 32) {
      const int y = y0 + lane;
      const bool on = y < e.nb;
      const float bh = on ? A.ah[b_off + y] : -INFINITY;
      const float bl = on ? A.al[b_off + y] : 0.f;
      float pb[3] = {0.f, 0.f, 0.f};
      if (on && nb.coord_off >= 0)
        for (int k = 0; k < D; ++k) pb[k] = A.coords[nb.coord_off + (int64_t)y * D + k];
      float cs = 0.f, cc = 0.f;  // this column's sum over the warp's rows (Kahan)
      if (bh > -INFINITY) {
#pragma unroll
        for (int r = 0; r < kChkRows; ++r) {
          if (!(rah[r] > -INFINITY)) continue;
          const int x = t.o0 + warp * kChkRows + r;
          float cst;
          const float B = plan_entry(rah[r], ral[r], bh, bl, cost_df(e, P, x, y, rp[r], pb), kh, kl, cst);
          float y1 = B - rc[r];
          float t1 = rs[r] + y1;
          rc[r] = (t1 - rs[r]) - y1;
          rs[r] = t1;
          const float cb = cst * cscale * B;
          y1 = cb - tcmp[r];
          t1 = ts[r] + y1;
          tcmp[r] = (t1 - ts[r]) - y1;
          ts[r] = t1;
          y1 = B - cc;
          t1 = cs + y1;
          cc = (t1 - cs) - y1;
          cs = t1;
        }
      }
      s_col[warp][lane] = cs;
      s_cmp[warp][lane] = cc;
      __syncthreads();
      if (warp == 0 && on) {
        double v = 0.0;
#pragma unroll
        for (int w = 0; w < 8; ++w) v += (double)s_col[w][lane] - (double)s_cmp[w][lane];
        if (v != 0.0) atomicAdd(&A.marg[b_off + y], v);
      }
      __syncthreads();
    }
    double tc_acc = 0.0, mass_acc = 0.0;
#pragma unroll
    for (int r = 0; r < kChkRows; ++r) {
      const int xr = warp * kChkRows + r;
      const double row = warp_sum_d((double)rs[r] - (double)rc[r]);
      const double tr = warp_sum_d((double)ts[r] - (double)tcmp[r]);
      if (lane == 0 && xr < t.ocount) {
        A.marg[a_off + t.o0 + xr] = row;
        tc_acc += tr;
        mass_acc += row;
      }
    }
    if (lane == 0 && (tc_acc != 0.0 || mass_acc != 0.0)) {
      atomicAdd(&A.edge_tc[d.edge], tc_acc);
      atomicAdd(&A.edge_mass[d.edge], mass_acc);
    }
  }
}

// FP64 version of the check for FP64 handles (small problems): every plan entry
// exp(a + b - C/eps) in double precision.
__device__ __forceinline__ double a64(const CheckArgs& A, const DEdgeD& d, const NodeD& own, double inv_eps,
                                      int64_t off, int x) {
  const double lg = A.logg[own.node_off + x];
  if (lg == -INFINITY) return -INFINITY;
  return A.f[off + x] * inv_eps - A.Z[d.owner] + lg;
}

__global__ void __launch_bounds__(256) check64_kernel(CheckArgs A) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int ti = blockIdx.x; ti < A.ntasks; ti += gridDim.x) {
    const Task t = A.tasks[ti];
    const DEdgeD d = A.dedges[t.dedge];
    if (A.mask && !A.mask[d.prob]) continue;  // block-uniform
    const EdgeD e = A.edges[d.edge];
    const ProbD P = A.probs[d.prob];
    const NodeD na = A.nodes[e.a], nb = A.nodes[e.b];
    const DEdgeD dr = A.dedges[t.dedge ^ 1];
    const DEdgeD& da = d.dir == 0 ? d : dr;   // owner a (rows)
    const DEdgeD& db = d.dir == 0 ? dr : d;   // owner b (columns)
    const int D = P.dim;
    // output index i of this task's owner; the other side is reduced
    for (int r = warp; r < t.ocount; r += 8) {
      const int i = t.o0 + r;
      double sum = 0.0, tc = 0.0;
      const int nother = t.kind == TASK_ROW ? e.nb : e.na;
      const double ai = t.kind == TASK_ROW ? a64(A, da, na, P.inv_eps, da.off, i) : a64(A, db, nb, P.inv_eps, db.off, i);
      if (ai > -INFINITY) {
        for (int j = lane; j < nother; j += 32) {
          const int x = t.kind == TASK_ROW ? i : j;
          const int y = t.kind == TASK_ROW ? j : i;
          const double bj = t.kind == TASK_ROW ? a64(A, db, nb, P.inv_eps, db.off, y) : a64(A, da, na, P.inv_eps, da.off, x);
          if (!(bj > -INFINITY)) continue;
          double C;
          if (P.cost_kind == 0) {
            C = (double)e.C[(int64_t)x * e.ld + y];
          } else {
            C = 0.0;
            for (int k = 0; k < D; ++k) {
              const double dd = (double)A.coords[na.coord_off + (int64_t)x * D + k] -
                                (double)A.coords[nb.coord_off + (int64_t)y * D + k];
              C += dd * dd;
            }
            C *= P.cost_scale;
          }
          const double B = exp(ai + bj - C * P.inv_eps);
          sum += B;
          tc += B * C;
        }
      }
      sum = warp_sum_d(sum);
      tc = warp_sum_d(tc);
      if (lane == 0) {
        A.marg[d.off + i] = sum;
        if (t.kind == TASK_ROW) {
          atomicAdd(&A.edge_tc[d.edge], tc);
          atomicAdd(&A.edge_mass[d.edge], sum);
        }
      }
    }
  }
}

// v = (f'/eps - Z_owner + log gamma_owner) * scale, split into FP32 (hi, lo), per
// directed-edge entry.  Z may be null (the apply operand leaves Z out).
__global__ void operand_kernel(const double* f, const double* Z, const double* logg, const DEdgeD* dedges,
                               const NodeD* nodes, const ProbD* probs, int32_t d0, int32_t ndedges, double scale,
                               bool quantize, float* vh, float* vl) {
  const int di = d0 + blockIdx.y;
  if (di >= ndedges) return;
  const DEdgeD d = dedges[di];
  const NodeD nd = nodes[d.owner];
  const double inv_eps = probs[d.prob].inv_eps;
  const double z = Z ? Z[d.owner] : 0.0;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nd.n; x += gridDim.x * blockDim.x) {
    const double lg = logg[nd.node_off + x];
    const double a = (f[d.off + x] * inv_eps - z + lg) * scale;
    const float hi = quantize ? (float)(rint(a * kGrid) / kGrid) : (float)a;
    vh[d.off + x] = (lg == -INFINITY) ? -INFINITY : hi;
    vl[d.off + x] = isfinite(a) ? (float)(a - (double)hi) : 0.f;
  }
}

// batched potential set: pass 0 flags non-finite values, pass 1 writes the
// normalised potential f' = f + eps Z_owner and records the directed edge for
// the operand refresh
__global__ void set_potentials_kernel(const float* values, int64_t ld, const int32_t* dlist, int32_t i0,
                                      const DEdgeD* dedges, const NodeD* nodes, const ProbD* probs, const double* Z,
                                      double* f, DEdgeD* picked, int32_t* bad, int32_t write) {
  const int i = i0 + blockIdx.y;
  const DEdgeD d = dedges[dlist[i]];
  const int n = nodes[d.owner].n;
  const double ez = probs[d.prob].eps * Z[d.owner];
  if (write && blockIdx.x == 0 && threadIdx.x == 0) picked[i] = d;
  int local = 0;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
    const float v = values[(int64_t)i * ld + x];
    if (!isfinite(v)) local = 1;
    if (write) f[d.off + x] = (double)v + ez;
  }
  if (__syncthreads_or(local) && threadIdx.x == 0) atomicOr(bad, 1);
}

// batched potential read: one CTA per item, f = f' - eps Z_owner in FP32,
// optionally centred (mean over x subtracted, the mean taken in FP64)
__global__ void get_potentials_kernel(const int32_t* dlist, int32_t i0, const DEdgeD* dedges, const NodeD* nodes,
                                      const ProbD* probs, const double* Z, const double* f, float* values,
                                      int64_t ld, int32_t centred) {
  __shared__ double red[8];
  const int i = i0 + blockIdx.x;
  const DEdgeD d = dedges[dlist[i]];
  const int n = nodes[d.owner].n;
  const double ez = probs[d.prob].eps * Z[d.owner];
  double mean = 0.0;
  if (centred) {
    double acc = 0.0;
    for (int x = threadIdx.x; x < n; x += blockDim.x) acc += f[d.off + x] - ez;
    acc = warp_sum_d(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    double tot = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
    mean = tot / n;
  }
  for (int x = threadIdx.x; x < n; x += blockDim.x) values[(int64_t)i * ld + x] = (float)(f[d.off + x] - ez - mean);
}

// per problem: max |coordinate| (as the bits of a non-negative float)
__global__ void coord_absmax_kernel(const float* coords, const NodeD* nodes, int32_t nnodes, const ProbD* probs,
                                    uint32_t* cmax) {
  for (int j = blockIdx.x; j < nnodes; j += gridDim.x) {
    const NodeD nd = nodes[j];
    if (nd.coord_off < 0) continue;
    const int64_t cnt = (int64_t)nd.n * probs[nd.prob].dim;
    float m = 0.f;
    for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x) m = fmaxf(m, fabsf(coords[nd.coord_off + i]));
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0) atomicMax(&cmax[nd.prob], __float_as_uint(m));
  }
}

// coordinates split c = hi + lo, hi on the grid of unit = 2^-10 sigma, sigma the
// power of two >= the problem's max |coordinate| (the scalings are exact)
__global__ void split_coords_kernel(const float* coords, const NodeD* nodes, int32_t nnodes, const ProbD* probs,
                                    const uint32_t* cmax, float* hi, float* lo) {
  for (int j = blockIdx.x; j < nnodes; j += gridDim.x) {
    const NodeD nd = nodes[j];
    if (nd.coord_off < 0) continue;
    const float m = __uint_as_float(cmax[nd.prob]);
    int e = 0;
    if (m > 0.f) (void)frexpf(m, &e);  // m = f 2^e, f in [0.5, 1): sigma = 2^e >= m
    const int64_t cnt = (int64_t)nd.n * probs[nd.prob].dim;
    for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x) {
      const float c = coords[nd.coord_off + i];
      const float h = ldexpf(rintf(ldexpf(c, 10 - e)), e - 10);
      hi[nd.coord_off + i] = h;
      lo[nd.coord_off + i] = c - h;  // exact: c and h share the grid above unit / 2
    }
  }
}

// counts NaN and -inf entries of a padded dense cost (+inf is allowed)
__global__ void scan_cost_kernel(const float* C, int64_t ld, int32_t rows, int32_t cols, int32_t* bad) {
  int local = 0;
  const int64_t total = (int64_t)rows * cols;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const float v = C[(i / cols) * ld + (i % cols)];
    if (v != v || v == -INFINITY) local = 1;
  }
  if (__syncthreads_or(local) && threadIdx.x == 0) atomicOr(bad, 1);
}

__global__ void fill_kernel(float* p, int64_t n, float v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

__global__ void pad_copy_kernel(const float* src, int64_t src_ld, float* dst, int64_t dst_ld, int32_t rows,
                                int32_t cols) {
  const int r = blockIdx.y;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < dst_ld; c += (int64_t)gridDim.x * blockDim.x)
    dst[(int64_t)r * dst_ld + c] = c < cols ? src[(int64_t)r * src_ld + c] : INFINITY;
}

// 32 x 32 tiles through shared memory: reads and writes both coalesced
// src rows r < rows (of this launch's slice), columns c < cols; dst row c, columns
// r < dst_cols of the slice (rows <= r < dst_cols are the +inf pads)
__global__ void transpose_pad_kernel(const float* src, int64_t src_ld, int64_t rows, int32_t cols, float* dst,
                                     int64_t dst_ld, int64_t dst_cols) {
  __shared__ float tile[32][33];
  const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t r = r0 + i, c = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (r < rows && c < cols) ? src[r * src_ld + c] : INFINITY;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t c = c0 + i, r = r0 + threadIdx.x;
    if (c < cols && r < dst_cols) dst[c * dst_ld + r] = tile[threadIdx.x][i];
  }
}

}  // namespace

cudaError_t launch_transpose_pad(const float* src, int64_t src_ld, int32_t rows, int32_t cols, float* dst,
                                 int64_t dst_ld, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  // dst columns run to dst_ld (>= rows): the tiles past rows write the +inf pads
  const int64_t gy = (dst_ld + 31) / 32, gx = ((int64_t)cols + 31) / 32;
  for (int64_t y0 = 0; y0 < gy; y0 += 65535) {
    const int64_t ny = gy - y0 < 65535 ? gy - y0 : 65535;
    const int64_t first = y0 * 32;  // first source row / destination column of this slice
    dim3 grid((unsigned)gx, (unsigned)ny);
    transpose_pad_kernel<<<grid, dim3(32, 8), 0, s>>>(src + (first < rows ? first : 0) * src_ld, src_ld,
                                                       (int64_t)rows - first, cols, dst + first, dst_ld,
                                                       dst_ld - first);
  }
  return cudaGetLastError();
}

cudaError_t launch_check64(const CheckArgs& a, cudaStream_t s) {
  if (a.ntasks <= 0) return cudaSuccess;
  check64_kernel<<<a.ntasks < 1024 ? a.ntasks : 1024, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_check(const CheckArgs& a, cudaStream_t s) {
  if (a.ntasks <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = a.ntasks < sms * 4 ? a.ntasks : sms * 4;
  check_kernel<<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_operand(const double* f, const double* Z, const double* logg, const DEdgeD* dedges,
                           const NodeD* nodes, const ProbD* probs, int32_t ndedges, double scale, bool quantize,
                           float* vh, float* vl, cudaStream_t s) {
  for (int32_t d0 = 0; d0 < ndedges; d0 += 65535) {
    const int32_t cnt = ndedges - d0 < 65535 ? ndedges - d0 : 65535;
    dim3 grid(4, cnt);
    operand_kernel<<<grid, 256, 0, s>>>(f, Z, logg, dedges, nodes, probs, d0, ndedges, scale, quantize, vh, vl);
  }
  return cudaGetLastError();
}

cudaError_t launch_set_potentials(const float* values, int64_t ld, const int32_t* dlist, int32_t count,
                                  const DEdgeD* dedges, const NodeD* nodes, const ProbD* probs, const double* Z,
                                  double* f, DEdgeD* picked, int32_t* bad, bool write, cudaStream_t s) {
  for (int32_t i0 = 0; i0 < count; i0 += 65535) {
    const int32_t cnt = count - i0 < 65535 ? count - i0 : 65535;
    dim3 grid(4, cnt);
    set_potentials_kernel<<<grid, 256, 0, s>>>(values, ld, dlist, i0, dedges, nodes, probs, Z, f, picked, bad,
                                               write ? 1 : 0);
  }
  return cudaGetLastError();
}

cudaError_t launch_get_potentials(const int32_t* dlist, int32_t count, const DEdgeD* dedges, const NodeD* nodes,
                                  const ProbD* probs, const double* Z, const double* f, float* values, int64_t ld,
                                  bool centred, cudaStream_t s) {
  for (int32_t i0 = 0; i0 < count; i0 += 65535) {
    const int32_t cnt = count - i0 < 65535 ? count - i0 : 65535;
    get_potentials_kernel<<<cnt, 256, 0, s>>>(dlist, i0, dedges, nodes, probs, Z, f, values, ld, centred ? 1 : 0);
  }
  return cudaGetLastError();
}

cudaError_t launch_split_coords(const float* coords, const NodeD* nodes, int32_t nnodes, const ProbD* probs,
                                uint32_t* cmax, int32_t nprob, float* hi, float* lo, cudaStream_t s) {
  if (nnodes <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(cmax, 0, sizeof(uint32_t) * nprob, s);
  if (e != cudaSuccess) return e;
  const int grid = nnodes < 4096 ? nnodes : 4096;
  coord_absmax_kernel<<<grid, 256, 0, s>>>(coords, nodes, nnodes, probs, cmax);
  split_coords_kernel<<<grid, 256, 0, s>>>(coords, nodes, nnodes, probs, cmax, hi, lo);
  return cudaGetLastError();
}

cudaError_t launch_scan_cost(const float* C, int64_t ld, int32_t rows, int32_t cols, int32_t* bad, cudaStream_t s) {
  if ((int64_t)rows * cols <= 0) return cudaSuccess;
  scan_cost_kernel<<<1024, 256, 0, s>>>(C, ld, rows, cols, bad);
  return cudaGetLastError();
}

cudaError_t launch_fill_f32(float* p, int64_t n, float v, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  fill_kernel<<<(int)blocks, 256, 0, s>>>(p, n, v);
  return cudaGetLastError();
}

cudaError_t launch_pad_copy(const float* src, int64_t src_ld, float* dst, int64_t dst_ld, int32_t rows,
                            int32_t cols, cudaStream_t s) {
  for (int32_t r0 = 0; r0 < rows; r0 += 65535) {
    const int32_t cnt = rows - r0 < 65535 ? rows - r0 : 65535;
    dim3 grid(4, cnt);
    pad_copy_kernel<<<grid, 256, 0, s>>>(src + (int64_t)r0 * src_ld, src_ld, dst + (int64_t)r0 * dst_ld, dst_ld, cnt,
                                         cols);
  }
  return cudaGetLastError();
}

}  // namespace treeot
