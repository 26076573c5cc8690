// C ABI of the warm-start MLP (tree_ot_mlp_*): parameter storage, forward,
// backward and Adam, all on the device through the kernels of mlp.cu.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/tree_ot.h"
#include "internal.h"

using namespace treeot;

struct tree_ot_mlp {
  int32_t in = 0, hid = 0, out = 0, max_batch = 0;
  int64_t nparam = 0;
  int64_t off[6] = {};   // W1, b1, W2, b2, W3, b3 in the FP32 parameter vector
  int64_t len[6] = {};
  float *w = nullptr, *g = nullptr, *m1 = nullptr, *m2 = nullptr;  // FP32 master, gradients, Adam moments
  void* w16 = nullptr;                                             // BF16 copy of the whole vector
  void *x16 = nullptr, *a1 = nullptr, *a2 = nullptr, *dy16 = nullptr, *dz2_16 = nullptr, *dz1_16 = nullptr;
  float *z1 = nullptr, *z2 = nullptr, *y = nullptr, *dy32 = nullptr, *da2 = nullptr, *dz2_32 = nullptr;
  float *da1 = nullptr, *dz1_32 = nullptr;
  double* loss = nullptr;
  int64_t step = 0;
  int32_t nlog = 0;          // input transform: first nlog features -> log(max(x, floor)) * scale
  float log_floor = 1e-30f, log_scale = 1.f;
  std::vector<void*> owned;
};

namespace {
thread_local std::string g_mlp_err;
int mfail(int code, const std::string& m) {
  g_mlp_err = m;
  return code;
}
#define MCUDA(call)                                                                                  \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess)                                                                           \
      return mfail(e_ == cudaErrorMemoryAllocation ? TREE_OT_ERR_OOM : TREE_OT_ERR_CUDA,             \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                              \
  } while (0)

template <class T>
int dalloc(tree_ot_mlp* m, T** p, int64_t count, size_t elem = sizeof(T)) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, elem * (size_t)(count > 0 ? count : 1));
  if (e != cudaSuccess) return mfail(TREE_OT_ERR_OOM, "cudaMalloc (mlp)");
  m->owned.push_back(q);
  *p = static_cast<T*>(q);
  return TREE_OT_OK;
}

uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// bf16 pointer arithmetic on the weight copy
void* w16_at(tree_ot_mlp* m, int t) { return static_cast<char*>(m->w16) + 2 * m->off[t]; }

int forward(tree_ot_mlp* m, const float* x, int32_t B, cudaStream_t s) {
  MCUDA(mlp_input(x, m->x16, B, m->in, m->nlog, m->log_floor, m->log_scale, s));
  MCUDA(mlp_gemm(m->x16, m->in, 0, w16_at(m, 0), m->in, 1, m->z1, m->hid, B, m->hid, m->in, m->w + m->off[1], 0, s));
  MCUDA(mlp_gelu_fwd(m->z1, m->a1, (int64_t)B * m->hid, s));
  MCUDA(mlp_gemm(m->a1, m->hid, 0, w16_at(m, 2), m->hid, 1, m->z2, m->hid, B, m->hid, m->hid, m->w + m->off[3], 0, s));
  MCUDA(mlp_gelu_fwd(m->z2, m->a2, (int64_t)B * m->hid, s));
  MCUDA(mlp_gemm(m->a2, m->hid, 0, w16_at(m, 4), m->hid, 1, m->y, m->out, B, m->out, m->hid, m->w + m->off[5], 0, s));
  return TREE_OT_OK;
}

int backward(tree_ot_mlp* m, const float* t, int32_t B, cudaStream_t s) {
  MCUDA(cudaMemsetAsync(m->loss, 0, sizeof(double), s));
  MCUDA(mlp_mse(m->y, t, m->dy32, m->dy16, (int64_t)B * m->out, m->loss, s));
  // layer 3: dW3 = dy^T a2, db3 = sum dy, da2 = dy W3
  MCUDA(mlp_gemm(m->dy16, m->out, 1, m->a2, m->hid, 0, m->g + m->off[4], m->hid, m->out, m->hid, B, nullptr, 0, s));
  MCUDA(mlp_colsum(m->dy32, B, m->out, m->g + m->off[5], s));
  MCUDA(mlp_gemm(m->dy16, m->out, 0, w16_at(m, 4), m->hid, 0, m->da2, m->hid, B, m->hid, m->out, nullptr, 0, s));
  MCUDA(mlp_gelu_bwd(m->da2, m->z2, m->dz2_16, m->dz2_32, (int64_t)B * m->hid, s));
  // layer 2
  MCUDA(mlp_gemm(m->dz2_16, m->hid, 1, m->a1, m->hid, 0, m->g + m->off[2], m->hid, m->hid, m->hid, B, nullptr, 0, s));
  MCUDA(mlp_colsum(m->dz2_32, B, m->hid, m->g + m->off[3], s));
  MCUDA(mlp_gemm(m->dz2_16, m->hid, 0, w16_at(m, 2), m->hid, 0, m->da1, m->hid, B, m->hid, m->hid, nullptr, 0, s));
  MCUDA(mlp_gelu_bwd(m->da1, m->z1, m->dz1_16, m->dz1_32, (int64_t)B * m->hid, s));
  // layer 1
  MCUDA(mlp_gemm(m->dz1_16, m->hid, 1, m->x16, m->in, 0, m->g + m->off[0], m->in, m->hid, m->in, B, nullptr, 0, s));
  MCUDA(mlp_colsum(m->dz1_32, B, m->hid, m->g + m->off[1], s));
  return TREE_OT_OK;
}

int check_batch(tree_ot_mlp* m, const void* x, int32_t B) {
  if (!m || !x) return mfail(TREE_OT_ERR_ARG, "NULL mlp or input");
  if (B < 1 || B > m->max_batch) return mfail(TREE_OT_ERR_ARG, "batch must be 1..max_batch");
  return TREE_OT_OK;
}
}  // namespace

extern "C" {

const char* tree_ot_mlp_last_error(void) { return g_mlp_err.c_str(); }

int tree_ot_mlp_create(int32_t in_dim, int32_t hidden, int32_t out_dim, int32_t max_batch, uint64_t seed,
                       tree_ot_mlp** out) {
  g_mlp_err.clear();
  if (!out || in_dim < 1 || hidden < 1 || out_dim < 1 || max_batch < 1)
    return mfail(TREE_OT_ERR_ARG, "dimensions and max_batch must be >= 1");
  *out = nullptr;
  tree_ot_mlp* m = new tree_ot_mlp();
  m->in = in_dim;
  m->hid = hidden;
  m->out = out_dim;
  m->max_batch = max_batch;
  const int64_t lens[6] = {(int64_t)hidden * in_dim, hidden, (int64_t)hidden * hidden, hidden,
                           (int64_t)out_dim * hidden, out_dim};
  int64_t o = 0;
  for (int t = 0; t < 6; ++t) {
    m->off[t] = o;
    m->len[t] = lens[t];
    o += (lens[t] + 7) / 8 * 8;  // keep every tensor 16-byte aligned in the BF16 copy
  }
  m->nparam = o;
  const int64_t B = max_batch;
  int rc = 0;
  if ((rc = dalloc(m, &m->w, o)) || (rc = dalloc(m, &m->g, o)) || (rc = dalloc(m, &m->m1, o)) ||
      (rc = dalloc(m, &m->m2, o)) || (rc = dalloc(m, &m->w16, o, 2)) || (rc = dalloc(m, &m->x16, B * in_dim, 2)) ||
      (rc = dalloc(m, &m->a1, B * hidden, 2)) || (rc = dalloc(m, &m->a2, B * hidden, 2)) ||
      (rc = dalloc(m, &m->dy16, B * out_dim, 2)) || (rc = dalloc(m, &m->dz2_16, B * hidden, 2)) ||
      (rc = dalloc(m, &m->dz1_16, B * hidden, 2)) || (rc = dalloc(m, &m->z1, B * hidden)) ||
      (rc = dalloc(m, &m->z2, B * hidden)) || (rc = dalloc(m, &m->y, B * out_dim)) ||
      (rc = dalloc(m, &m->dy32, B * out_dim)) || (rc = dalloc(m, &m->da2, B * hidden)) ||
      (rc = dalloc(m, &m->dz2_32, B * hidden)) || (rc = dalloc(m, &m->da1, B * hidden)) ||
      (rc = dalloc(m, &m->dz1_32, B * hidden)) || (rc = dalloc(m, &m->loss, 1))) {
    tree_ot_mlp_destroy(m);
    return rc;
  }
  // uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases (SplitMix64 stream from seed)
  std::vector<float> h(o, 0.f);
  uint64_t st = seed;
  const int64_t fan[3] = {in_dim, hidden, hidden};
  for (int layer = 0; layer < 3; ++layer) {
    const double a = 1.0 / std::sqrt((double)fan[layer]);
    for (int64_t i = 0; i < m->len[2 * layer]; ++i) {
      const double u = (double)(splitmix64(st) >> 11) * (1.0 / 9007199254740992.0);
      h[m->off[2 * layer] + i] = (float)((2.0 * u - 1.0) * a);
    }
  }
  rc = tree_ot_mlp_set_params(m, h.data());
  if (rc) {
    tree_ot_mlp_destroy(m);
    return rc;
  }
  *out = m;
  return TREE_OT_OK;
}

int tree_ot_mlp_destroy(tree_ot_mlp* m) {
  if (!m) return TREE_OT_OK;
  for (void* p : m->owned) cudaFree(p);
  delete m;
  return TREE_OT_OK;
}

int tree_ot_mlp_num_params(tree_ot_mlp* m, int64_t* n, int64_t* offsets) {
  if (!m || !n) return mfail(TREE_OT_ERR_ARG, "NULL argument");
  *n = m->nparam;
  if (offsets)
    for (int t = 0; t < 6; ++t) offsets[t] = m->off[t];
  return TREE_OT_OK;
}

int tree_ot_mlp_get_params(tree_ot_mlp* m, float* host_out) {
  if (!m || !host_out) return mfail(TREE_OT_ERR_ARG, "NULL argument");
  MCUDA(cudaMemcpy(host_out, m->w, sizeof(float) * m->nparam, cudaMemcpyDeviceToHost));
  return TREE_OT_OK;
}

int tree_ot_mlp_set_params(tree_ot_mlp* m, const float* host_in) {
  if (!m || !host_in) return mfail(TREE_OT_ERR_ARG, "NULL argument");
  MCUDA(cudaMemcpy(m->w, host_in, sizeof(float) * m->nparam, cudaMemcpyHostToDevice));
  MCUDA(cudaMemset(m->m1, 0, sizeof(float) * m->nparam));
  MCUDA(cudaMemset(m->m2, 0, sizeof(float) * m->nparam));
  MCUDA(mlp_to_bf16(m->w, m->w16, m->nparam, 0));
  MCUDA(cudaDeviceSynchronize());
  m->step = 0;
  return TREE_OT_OK;
}

int tree_ot_mlp_set_input_log(tree_ot_mlp* m, int32_t count, double floor_value, double scale) {
  g_mlp_err.clear();
  if (!m || count < 0 || count > m->in || !(floor_value > 0.0)) return mfail(TREE_OT_ERR_ARG, "bad input transform");
  m->nlog = count;
  m->log_floor = (float)floor_value;
  m->log_scale = (float)scale;
  return TREE_OT_OK;
}

int tree_ot_mlp_forward(tree_ot_mlp* m, void* stream, const float* x, int32_t batch, float* y) {
  g_mlp_err.clear();
  int rc = check_batch(m, x, batch);
  if (rc) return rc;
  if (!y) return mfail(TREE_OT_ERR_ARG, "NULL output");
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = forward(m, x, batch, s))) return rc;
  MCUDA(cudaMemcpyAsync(y, m->y, sizeof(float) * (size_t)batch * m->out, cudaMemcpyDeviceToDevice, s));
  return TREE_OT_OK;
}

int tree_ot_mlp_backward(tree_ot_mlp* m, void* stream, const float* x, const float* target, int32_t batch,
                         float* grads, double* loss) {
  g_mlp_err.clear();
  int rc = check_batch(m, x, batch);
  if (rc) return rc;
  if (!target) return mfail(TREE_OT_ERR_ARG, "NULL target");
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = forward(m, x, batch, s)) || (rc = backward(m, target, batch, s))) return rc;
  if (grads) MCUDA(cudaMemcpyAsync(grads, m->g, sizeof(float) * m->nparam, cudaMemcpyDeviceToDevice, s));
  if (loss) {
    MCUDA(cudaMemcpyAsync(loss, m->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
    MCUDA(cudaStreamSynchronize(s));
  }
  return TREE_OT_OK;
}

int tree_ot_mlp_train_step(tree_ot_mlp* m, void* stream, const float* x, const float* target, int32_t batch,
                           double lr, double* loss) {
  g_mlp_err.clear();
  int rc = check_batch(m, x, batch);
  if (rc) return rc;
  if (!target || !(lr > 0.0)) return mfail(TREE_OT_ERR_ARG, "NULL target or lr <= 0");
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = forward(m, x, batch, s)) || (rc = backward(m, target, batch, s))) return rc;
  m->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)m->step), c2 = 1.f - std::pow(b2, (float)m->step);
  MCUDA(mlp_adam(m->w, m->g, m->m1, m->m2, m->w16, m->nparam, (float)lr, b1, b2, 1e-8f, c1, c2, s));
  if (loss) {
    MCUDA(cudaMemcpyAsync(loss, m->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
    MCUDA(cudaStreamSynchronize(s));
  }
  return TREE_OT_OK;
}

}  // extern "C"
