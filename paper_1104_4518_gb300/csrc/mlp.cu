// The per-level variant selector network: forward pass, mean-squared-error
// gradient and Adam, on the device.  The network is 12 -> 64 -> 64 -> 4 with
// ReLU, float32 (layout in mlp_device.cuh).  Gradients are summed in a fixed
// order (per-tile partial sums, then a serial sum over tiles per parameter),
// so a training run is bit-reproducible.
#include <cmath>
#include <mutex>
#include <vector>

#include "internal.h"
#include "nvtx_range.h"
#include "mlp_device.cuh"

namespace bfsint {
namespace {

using namespace bfsdev;

constexpr int kFwdThreads = 128;
constexpr int kTS = 32;           // samples per gradient tile
constexpr int kGradThreads = 256;

__global__ void __launch_bounds__(kFwdThreads) mlp_forward_kernel(const float* __restrict__ params,
                                                                  const float* __restrict__ X, int B,
                                                                  float* __restrict__ Y) {
  extern __shared__ float s_w[];
  for (int i = threadIdx.x; i < BFS_MLP_PARAMS; i += kFwdThreads) s_w[i] = params[i];
  __syncthreads();
  const int s = blockIdx.x * kFwdThreads + threadIdx.x;
  if (s >= B) return;
  float x[12], h1[64], h2[64];
#pragma unroll
  for (int k = 0; k < 12; ++k) x[k] = X[(long long)s * 12 + k];
  for (int t = 0; t < 64; ++t) h1[t] = mlp_h1(s_w, x, t);
  for (int t = 0; t < 64; ++t) h2[t] = mlp_h2(s_w, h1, t);
#pragma unroll
  for (int o = 0; o < 4; ++o) Y[(long long)s * 4 + o] = mlp_out(s_w, h2, o);
}

struct GradSmem {
  float x[kTS][12];
  float h1[kTS][64];
  float h2[kTS][64];
  float dz1[kTS][64];
  float dz2[kTS][64];
  float dy[kTS][4];
  float sq[kGradThreads];
};

// Partial gradient and squared error of one tile of kTS samples.
__global__ void __launch_bounds__(kGradThreads) mlp_grad_tile_kernel(const float* __restrict__ params,
                                                                     const float* __restrict__ X,
                                                                     const float* __restrict__ T, int B,
                                                                     float* __restrict__ partial,
                                                                     float* __restrict__ partial_loss) {
  extern __shared__ float smem[];
  float* s_w = smem;
  GradSmem& g = *reinterpret_cast<GradSmem*>(smem + BFS_MLP_PARAMS);
  const int tid = threadIdx.x;
  for (int i = tid; i < BFS_MLP_PARAMS; i += kGradThreads) s_w[i] = params[i];
  const long long s0 = (long long)blockIdx.x * kTS;
  for (int i = tid; i < kTS * 12; i += kGradThreads) {
    const int s = i / 12, k = i % 12;
    g.x[s][k] = (s0 + s < B) ? X[(s0 + s) * 12 + k] : 0.0f;
  }
  __syncthreads();
  for (int i = tid; i < kTS * 64; i += kGradThreads) {
    const int s = i / 64, t = i % 64;
    g.h1[s][t] = mlp_h1(s_w, g.x[s], t);
  }
  __syncthreads();
  for (int i = tid; i < kTS * 64; i += kGradThreads) {
    const int s = i / 64, t = i % 64;
    g.h2[s][t] = mlp_h2(s_w, g.h1[s], t);
  }
  __syncthreads();
  const float scale = 2.0f / (4.0f * (float)B);
  float sq = 0.0f;
  for (int i = tid; i < kTS * 4; i += kGradThreads) {
    const int s = i / 4, o = i % 4;
    float d = 0.0f;
    if (s0 + s < B) {
      const float y = mlp_out(s_w, g.h2[s], o);
      const float diff = y - T[(s0 + s) * 4 + o];
      sq += diff * diff;
      d = scale * diff;
    }
    g.dy[s][o] = d;
  }
  g.sq[tid] = sq;
  __syncthreads();
  for (int i = tid; i < kTS * 64; i += kGradThreads) {  // dz2 = (dy W3^T) * [h2 > 0]
    const int s = i / 64, j = i % 64;
    float a = 0.0f;
#pragma unroll
    for (int o = 0; o < 4; ++o) a = fmaf(g.dy[s][o], s_w[kW3 + j * 4 + o], a);
    g.dz2[s][j] = g.h2[s][j] > 0.0f ? a : 0.0f;
  }
  __syncthreads();
  for (int i = tid; i < kTS * 64; i += kGradThreads) {  // dz1 = (dz2 W2^T) * [h1 > 0]
    const int s = i / 64, t = i % 64;
    float a = 0.0f;
    for (int j = 0; j < 64; ++j) a = fmaf(g.dz2[s][j], s_w[kW2 + t * 64 + j], a);
    g.dz1[s][t] = g.h1[s][t] > 0.0f ? a : 0.0f;
  }
  __syncthreads();
  float* out = partial + (long long)blockIdx.x * BFS_MLP_PARAMS;
  for (int pidx = tid; pidx < BFS_MLP_PARAMS; pidx += kGradThreads) {
    float a = 0.0f;
    if (pidx < kB1) {
      const int k = pidx / 64, t = pidx % 64;
      for (int s = 0; s < kTS; ++s) a = fmaf(g.x[s][k], g.dz1[s][t], a);
    } else if (pidx < kW2) {
      const int t = pidx - kB1;
      for (int s = 0; s < kTS; ++s) a += g.dz1[s][t];
    } else if (pidx < kB2) {
      const int q = pidx - kW2, i = q / 64, t = q % 64;
      for (int s = 0; s < kTS; ++s) a = fmaf(g.h1[s][i], g.dz2[s][t], a);
    } else if (pidx < kW3) {
      const int t = pidx - kB2;
      for (int s = 0; s < kTS; ++s) a += g.dz2[s][t];
    } else if (pidx < kB3) {
      const int q = pidx - kW3, j = q / 4, o = q % 4;
      for (int s = 0; s < kTS; ++s) a = fmaf(g.h2[s][j], g.dy[s][o], a);
    } else {
      const int o = pidx - kB3;
      for (int s = 0; s < kTS; ++s) a += g.dy[s][o];
    }
    out[pidx] = a;
  }
  if (tid == 0) {
    float tot = 0.0f;
    for (int i = 0; i < kGradThreads; ++i) tot += g.sq[i];
    partial_loss[blockIdx.x] = tot;
  }
}

__global__ void mlp_reduce_kernel(const float* __restrict__ partial, const float* __restrict__ partial_loss,
                                  int ntiles, int B, float* __restrict__ grad, float* __restrict__ loss) {
  const int pidx = blockIdx.x * blockDim.x + threadIdx.x;
  if (pidx < BFS_MLP_PARAMS) {
    float a = 0.0f;
    for (int b = 0; b < ntiles; ++b) a += partial[(long long)b * BFS_MLP_PARAMS + pidx];
    grad[pidx] = a;
  }
  if (pidx == 0 && loss) {
    float a = 0.0f;
    for (int b = 0; b < ntiles; ++b) a += partial_loss[b];
    *loss = a / (4.0f * (float)B);
  }
}

__global__ void adam_kernel(float* __restrict__ params, const float* __restrict__ grad, float* __restrict__ m,
                            float* __restrict__ v, float lr, float beta1, float beta2, float eps, float bc1,
                            float bc2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= BFS_MLP_PARAMS) return;
  const float gi = grad[i];
  const float mi = beta1 * m[i] + (1.0f - beta1) * gi;
  const float vi = beta2 * v[i] + (1.0f - beta2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float mhat = mi / bc1;
  const float vhat = vi / bc2;
  params[i] -= lr * mhat / (sqrtf(vhat) + eps);
}

size_t grad_smem_bytes() { return sizeof(float) * BFS_MLP_PARAMS + sizeof(GradSmem); }

int grad_impl(const float* params, const float* X, const float* T, int B, float* grad, float* loss,
              float* partial, float* partial_loss, cudaStream_t s) {
  const int ntiles = (B + kTS - 1) / kTS;
  static bool configured = false;
  if (!configured) {
    BFS_CUDA_TRY(cudaFuncSetAttribute(mlp_grad_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)grad_smem_bytes()));
    configured = true;
  }
  mlp_grad_tile_kernel<<<ntiles, kGradThreads, grad_smem_bytes(), s>>>(params, X, T, B, partial, partial_loss);
  mlp_reduce_kernel<<<(BFS_MLP_PARAMS + 255) / 256, 256, 0, s>>>(partial, partial_loss, ntiles, B, grad, loss);
  BFS_CUDA_TRY(cudaGetLastError());
  return BFS_OK;
}

// ---------------- selector parameters of this process ----------------
std::mutex g_sel_mu;
std::vector<float> g_sel_host;
std::vector<float*> g_sel_dev;  // per device ordinal

}  // namespace

const float* learned_params_device() {
  std::lock_guard<std::mutex> lk(g_sel_mu);
  if (g_sel_host.empty()) return nullptr;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  if ((int)g_sel_dev.size() <= dev) g_sel_dev.resize(dev + 1, nullptr);
  if (!g_sel_dev[dev]) {
    float* p = nullptr;
    if (cudaMalloc(&p, sizeof(float) * BFS_MLP_PARAMS) != cudaSuccess) return nullptr;
    if (cudaMemcpy(p, g_sel_host.data(), sizeof(float) * BFS_MLP_PARAMS, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaFree(p);
      return nullptr;
    }
    g_sel_dev[dev] = p;
  }
  return g_sel_dev[dev];
}

void graph_feature_constants(int32_t n, int64_t nnz, float* log_n, float* log_nnz, float* inv_n, float* inv_nnz) {
  const float fn = (float)(n > 1 ? n : 1);
  const float fe = (float)(nnz > 1 ? nnz : 1);
  *log_n = log2f(fn) * 0.03125f;
  *log_nnz = log2f(fe) * 0.03125f;
  *inv_n = 1.0f / fn;
  *inv_nnz = 1.0f / fe;
}

}  // namespace bfsint

using namespace bfsint;

extern "C" {

int bfs_mlp_forward(const float* params, const float* X, int32_t B, float* Y, void* stream) {
  if (!params || !X || !Y || B < 0) return fail(BFS_ERR_INVALID_ARG, "bfs_mlp_forward: bad argument");
  if (B == 0) return BFS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  static bool configured = false;
  if (!configured) {
    BFS_CUDA_TRY(cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(sizeof(float) * BFS_MLP_PARAMS)));
    configured = true;
  }
  mlp_forward_kernel<<<(B + kFwdThreads - 1) / kFwdThreads, kFwdThreads, sizeof(float) * BFS_MLP_PARAMS, s>>>(
      params, X, B, Y);
  BFS_CUDA_TRY(cudaGetLastError());
  return BFS_OK;
}

int bfs_mlp_loss_grad(const float* params, const float* X, const float* T, int32_t B, float* grad, float* loss,
                      void* stream) {
  if (!params || !X || !T || !grad || B < 1) return fail(BFS_ERR_INVALID_ARG, "bfs_mlp_loss_grad: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  const int ntiles = (B + kTS - 1) / kTS;
  float* partial = nullptr;
  if (int e = dev_alloc((void**)&partial, sizeof(float) * ((size_t)ntiles * BFS_MLP_PARAMS + ntiles), "MLP partials"))
    return e;
  int rc = grad_impl(params, X, T, B, grad, loss, partial, partial + (size_t)ntiles * BFS_MLP_PARAMS, s);
  cudaError_t err = cudaStreamSynchronize(s);
  cudaFree(partial);
  if (rc) return rc;
  if (err != cudaSuccess) return cuda_fail(err, "bfs_mlp_loss_grad");
  return BFS_OK;
}

int bfs_mlp_adam(float* params, const float* grad, float* m, float* v, int32_t t, float lr, float beta1, float beta2,
                 float eps, void* stream) {
  if (!params || !grad || !m || !v || t < 1) return fail(BFS_ERR_INVALID_ARG, "bfs_mlp_adam: bad argument");
  const float bc1 = (float)(1.0 - std::pow((double)beta1, (double)t));
  const float bc2 = (float)(1.0 - std::pow((double)beta2, (double)t));
  adam_kernel<<<(BFS_MLP_PARAMS + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, grad, m, v, lr, beta1, beta2,
                                                                              eps, bc1, bc2);
  BFS_CUDA_TRY(cudaGetLastError());
  return BFS_OK;
}

int bfs_selector_train(float* params, const float* X, const float* T, int32_t B, int32_t steps, float lr,
                       float* loss_history, void* stream) {
  NvtxRange nvtx_range("bfs_selector_train");
  if (!params || !X || !T || B < 1 || steps < 0) return fail(BFS_ERR_INVALID_ARG, "bfs_selector_train: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  const int ntiles = (B + kTS - 1) / kTS;
  float* buf = nullptr;
  const size_t nfl = (size_t)ntiles * BFS_MLP_PARAMS + ntiles + 3 * (size_t)BFS_MLP_PARAMS;
  if (int e = dev_alloc((void**)&buf, sizeof(float) * nfl, "training buffers")) return e;
  float* partial = buf;
  float* ploss = partial + (size_t)ntiles * BFS_MLP_PARAMS;
  float* grad = ploss + ntiles;
  float* m = grad + BFS_MLP_PARAMS;
  float* v = m + BFS_MLP_PARAMS;
  int rc = BFS_OK;
  cudaError_t err = cudaMemsetAsync(m, 0, sizeof(float) * 2 * BFS_MLP_PARAMS, s);
  if (err != cudaSuccess) rc = cuda_fail(err, "memset");
  for (int t = 1; rc == BFS_OK && t <= steps; ++t) {
    rc = grad_impl(params, X, T, B, grad, loss_history ? loss_history + (t - 1) : nullptr, partial, ploss, s);
    if (rc == BFS_OK) rc = bfs_mlp_adam(params, grad, m, v, t, lr, 0.9f, 0.999f, 1e-8f, stream);
  }
  err = cudaStreamSynchronize(s);
  cudaFree(buf);
  if (rc) return rc;
  if (err != cudaSuccess) return cuda_fail(err, "bfs_selector_train");
  return BFS_OK;
}

int bfs_selector_set_params(const float* params) {
  std::lock_guard<std::mutex> lk(g_sel_mu);
  for (float* p : g_sel_dev)
    if (p) cudaFree(p);
  g_sel_dev.clear();
  if (!params) {
    g_sel_host.clear();
    return BFS_OK;
  }
  g_sel_host.assign(params, params + BFS_MLP_PARAMS);
  return BFS_OK;
}

int bfs_selector_load(const char* path) {
  if (!path) return fail(BFS_ERR_INVALID_ARG, "bfs_selector_load: NULL path");
  FILE* f = fopen(path, "rb");
  if (!f) return fail(BFS_ERR_INVALID_ARG, std::string("bfs_selector_load: cannot open ") + path);
  std::vector<float> w(BFS_MLP_PARAMS);
  const size_t got = fread(w.data(), sizeof(float), BFS_MLP_PARAMS, f);
  fclose(f);
  if (got != (size_t)BFS_MLP_PARAMS) return fail(BFS_ERR_INVALID_ARG, "bfs_selector_load: short file");
  return bfs_selector_set_params(w.data());
}

int bfs_selector_save(const char* path) {
  if (!path) return fail(BFS_ERR_INVALID_ARG, "bfs_selector_save: NULL path");
  std::vector<float> w;
  {
    std::lock_guard<std::mutex> lk(g_sel_mu);
    w = g_sel_host;
  }
  if (w.empty()) return fail(BFS_ERR_INVALID_ARG, "bfs_selector_save: no network set");
  FILE* f = fopen(path, "wb");
  if (!f) return fail(BFS_ERR_INVALID_ARG, std::string("bfs_selector_save: cannot open ") + path);
  const size_t put = fwrite(w.data(), sizeof(float), BFS_MLP_PARAMS, f);
  fclose(f);
  if (put != (size_t)BFS_MLP_PARAMS) return fail(BFS_ERR_INVALID_ARG, "bfs_selector_save: write failed");
  return BFS_OK;
}

int bfs_level_features(int32_t n, int64_t nnz, int32_t k, int64_t frontier_count, int64_t frontier_edges,
                       int64_t unvisited_count, int64_t unvisited_edges, const int64_t* bin_count, float* out12) {
  if (!bin_count || !out12) return fail(BFS_ERR_INVALID_ARG, "bfs_level_features: NULL pointer");
  // the float32 expressions of the in-loop selector (bfsdev::level_features)
  float rn = 0.0f, re = 0.0f;
  bfsint::graph_feature_constants(n, nnz, &out12[0], &out12[1], &rn, &re);
  const float c = (float)frontier_count, d = (float)frontier_edges;
  const float rc = 1.0f / (frontier_count > 1 ? c : 1.0f);
  out12[2] = log2f(1.0f + (float)k) * 0.1f;
  out12[3] = log2f(1.0f + c) * 0.03125f;
  out12[4] = log2f(1.0f + d) * 0.03125f;
  out12[5] = c * rn;
  out12[6] = d * re;
  out12[7] = (float)unvisited_count * rn;
  out12[8] = (float)unvisited_edges * re;
  out12[9] = (float)bin_count[0] * rc;
  out12[10] = (float)bin_count[1] * rc;
  out12[11] = (float)bin_count[2] * rc;
  return BFS_OK;
}

}  // extern "C"
