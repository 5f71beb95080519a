// The selector network's forward pass for one input row, computed by a whole
// CTA from shared memory.  Used by both the stand-alone forward kernel and the
// in-loop variant selector, so that the two give bit-identical scores.
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

__device__ __forceinline__ float mlp_h2(const float* w, const float* h1, int t) {
  float a = w[kB2 + t];
#pragma unroll 8
  for (int i = 0; i < 64; ++i) a = fmaf(h1[i], w[kW2 + i * 64 + t], a);
  return fmaxf(a, 0.0f);
}

__device__ __forceinline__ float mlp_out(const float* w, const float* h2, int o) {
  float a = w[kB3 + o];
#pragma unroll 8
  for (int j = 0; j < 64; ++j) a = fmaf(h2[j], w[kW3 + j * 4 + o], a);
  return a;
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
