// The selector network's forward pass.  The in-loop selector evaluates it with
// a whole CTA (hidden layer 2 as 8 partial sums per unit combined by a
// butterfly of shuffles, the output layer as 32 partial sums per output); the
// stand-alone kernels evaluate the same sums in the same association order,
// one thread per row, so both give bit-identical scores.
#pragma once

#include "bfs.h"

namespace bfsdev {

// Offsets of the parameter blocks in the flat vector:
// W1[12][64], b1[64], W2[64][64], b2[64], W3[64][4], b3[4].
constexpr int kW1 = 0;
constexpr int kB1 = kW1 + 12 * 64;
constexpr int kW2 = kB1 + 64;
constexpr int kB2 = kW2 + 64 * 64;
constexpr int kW3 = kB2 + 64;
constexpr int kB3 = kW3 + 64 * 4;
static_assert(kB3 + 4 == BFS_MLP_PARAMS, "parameter layout");

// Hidden unit t (< 64) of layer 1 for input x[12].
__device__ __forceinline__ float mlp_h1(const float* w, const float* x, int t) {
  float a = w[kB1 + t];
#pragma unroll
  for (int k = 0; k < 12; ++k) a = fmaf(x[k], w[kW1 + k * 64 + t], a);
  return fmaxf(a, 0.0f);
}

// Partial sum j (< 8) of hidden unit t of layer 2: inputs 8j .. 8j+7.
__device__ __forceinline__ float mlp_h2_part(const float* w, const float* h1, int t, int j) {
  float a = 0.0f;
#pragma unroll
  for (int i = 8 * j; i < 8 * j + 8; ++i) a = fmaf(h1[i], w[kW2 + i * 64 + t], a);
  return a;
}

// Partial sum j (< 32) of output o: inputs j and j + 32.
__device__ __forceinline__ float mlp_out_part(const float* w, const float* h2, int o, int j) {
  return fmaf(h2[j + 32], w[kW3 + (j + 32) * 4 + o], h2[j] * w[kW3 + j * 4 + o]);
}

// Hidden unit t of layer 2, one thread: the 8 partial sums combined pairwise at
// distance 4, 2, 1 (the order of a shuffle butterfly over 8 lanes).
__device__ __forceinline__ float mlp_h2(const float* w, const float* h1, int t) {
  float p[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) p[j] = mlp_h2_part(w, h1, t, j);
#pragma unroll
  for (int m = 4; m >= 1; m >>= 1)
#pragma unroll
    for (int j = 0; j < m; ++j) p[j] = p[j] + p[j + m];
  return fmaxf(p[0] + w[kB2 + t], 0.0f);
}

// Output o, one thread: the 32 partial sums combined pairwise at distance 16 .. 1.
__device__ __forceinline__ float mlp_out(const float* w, const float* h2, int o) {
  float p[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) p[j] = mlp_out_part(w, h2, o, j);
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1)
#pragma unroll
    for (int j = 0; j < m; ++j) p[j] = p[j] + p[j + m];
  return p[0] + w[kB3 + o];
}

// Feature i (< 12) of a level (see bfs_level_features in bfs.h).
__device__ __forceinline__ float level_feature(int i, int n, long long nnz, int k, long long count, long long edges,
                                               long long unvisited, long long unvisited_edges,
                                               const long long* bins) {
  const float fn = (float)(n > 1 ? n : 1);
  const float fe = (float)(nnz > 1 ? nnz : 1);
  const float fc = (float)(count > 1 ? count : 1);
  switch (i) {
    case 0: return log2f(fn) / 32.0f;
    case 1: return log2f(fe) / 32.0f;
    case 2: return log2f(1.0f + (float)k) / 10.0f;
    case 3: return log2f(1.0f + (float)count) / 32.0f;
    case 4: return log2f(1.0f + (float)edges) / 32.0f;
    case 5: return (float)count / fn;
    case 6: return (float)edges / fe;
    case 7: return (float)unvisited / fn;
    case 8: return (float)unvisited_edges / fe;
    case 9: return (float)bins[0] / fc;
    case 10: return (float)bins[1] / fc;
    default: return (float)bins[2] / fc;
  }
}

// The 12 level features (see bfs_level_features in bfs.h).
__device__ __forceinline__ void level_features(int n, long long nnz, int k, long long count,
                                               long long edges, long long unvisited,
                                               long long unvisited_edges, const long long* bins,
                                               float* f) {
  const float fn = (float)(n > 1 ? n : 1);
  const float fe = (float)(nnz > 1 ? nnz : 1);
  const float fc = (float)(count > 1 ? count : 1);
  f[0] = log2f(fn) / 32.0f;
  f[1] = log2f(fe) / 32.0f;
  f[2] = log2f(1.0f + (float)k) / 10.0f;
  f[3] = log2f(1.0f + (float)count) / 32.0f;
  f[4] = log2f(1.0f + (float)edges) / 32.0f;
  f[5] = (float)count / fn;
  f[6] = (float)edges / fe;
  f[7] = (float)unvisited / fn;
  f[8] = (float)unvisited_edges / fe;
  f[9] = (float)bins[0] / fc;
  f[10] = (float)bins[1] / fc;
  f[11] = (float)bins[2] / fc;
}

}  // namespace bfsdev
