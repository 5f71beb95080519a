// The selector network's forward pass.  The in-loop selector evaluates it with
// one warp (lane l computes hidden units l and l + 32 of each layer, the output
// layer as 32 partial sums combined by a butterfly of shuffles); the
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

// Hidden unit t (< 64) of layer 2: four partial dot products over inputs
// 16r .. 16r+15 (r < 4), added as (p0 + p1) + (p2 + p3), then the bias.
__device__ __forceinline__ float mlp_h2(const float* w, const float* h1, int t) {
  float a[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    a[r] = 0.0f;
#pragma unroll
    for (int i = 16 * r; i < 16 * r + 16; ++i) a[r] = fmaf(h1[i], w[kW2 + i * 64 + t], a[r]);
  }
  return fmaxf(((a[0] + a[1]) + (a[2] + a[3])) + w[kB2 + t], 0.0f);
}

// Partial sum j (< 32) of output o: inputs j (value hj) and j + 32 (value hj32).
__device__ __forceinline__ float mlp_out_part(const float* w, float hj, float hj32, int o, int j) {
  return fmaf(hj32, w[kW3 + (j + 32) * 4 + o], hj * w[kW3 + j * 4 + o]);
}

// Output o, one thread: the 32 partial sums combined pairwise at distance
// 16 .. 1 (the order of a shuffle butterfly over 32 lanes), then the bias.
__device__ __forceinline__ float mlp_out(const float* w, const float* h2, int o) {
  float p[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) p[j] = mlp_out_part(w, h2[j], h2[j + 32], o, j);
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1)
#pragma unroll
    for (int j = 0; j < m; ++j) p[j] = p[j] + p[j + m];
  return p[0] + w[kB3 + o];
}

// Exact float of a nonnegative 64-bit count.  Values below 2^32 go through the
// 32-bit conversion, which gives the same float and pipelines far better than
// the 64-bit one; the branch is uniform when every lane converts the same value.
__device__ __forceinline__ float count_to_float(long long v) {
  return ((unsigned long long)v >> 32) ? (float)v : (float)(unsigned)v;
}

// The 12 level features (see bfs_level_features in bfs.h), the same float32
// expressions as the host function.  f0 = log2(n) / 32, f1 = log2(nnz) / 32,
// rn = 1 / n and re = 1 / nnz are constants of the graph, passed in.
__device__ __forceinline__ void level_features(float f0, float f1, float rn, float re, int k, long long count,
                                               long long edges, long long unvisited, long long unvisited_edges,
                                               long long bin0, long long bin1, long long bin2, float* x) {
  const float c = count_to_float(count), d = count_to_float(edges);
  const float rc = 1.0f / (count > 1 ? c : 1.0f);
  x[0] = f0;
  x[1] = f1;
  x[2] = log2f(1.0f + (float)k) * 0.1f;
  x[3] = log2f(1.0f + c) * 0.03125f;
  x[4] = log2f(1.0f + d) * 0.03125f;
  x[5] = c * rn;
  x[6] = d * re;
  x[7] = count_to_float(unvisited) * rn;
  x[8] = count_to_float(unvisited_edges) * re;
  x[9] = count_to_float(bin0) * rc;
  x[10] = count_to_float(bin1) * rc;
  x[11] = count_to_float(bin2) * rc;
}

// ---- the network on one warp ----
// The in-loop selector keeps the parameters in shared memory in a layout for a
// warp: in the blocks W1, b1, W2, b2 (each made of rows of 64), entry t of a
// row moves to position 2 (t mod 32) + t / 32, so lane l reads the weights of
// its units l and l + 32 as one float2.  W3 and b3 keep their places (lane j
// reads W3 rows j and j + 32 as float4).  The arithmetic is that of mlp_h1,
// mlp_h2 and mlp_out, in the same order.
__device__ __forceinline__ int warp_layout_index(int i) {
  if (i >= kW3) return i;
  const int t = i & 63;
  return (i - t) + 2 * (t & 31) + (t >> 5);
}

// Returns the index of the smallest of the 4 outputs on every lane of the
// calling warp.  x: the 12 features (the same values in every lane); h1: 64
// floats of 16-byte aligned shared scratch; w: parameters in the warp layout.
// Each group of shared-memory loads is issued before the multiply-adds that
// use it, so their latencies overlap.
__device__ __forceinline__ int warp_mlp_argmin(const float* __restrict__ w, const float* x, float* h1, int lane) {
  {
    const float2 bias1 = reinterpret_cast<const float2*>(w + kB1)[lane];
    float2 w1[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) w1[k] = reinterpret_cast<const float2*>(w + kW1 + k * 64)[lane];
    float a = bias1.x, c = bias1.y;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      a = fmaf(x[k], w1[k].x, a);
      c = fmaf(x[k], w1[k].y, c);
    }
    h1[lane] = fmaxf(a, 0.0f);
    h1[lane + 32] = fmaxf(c, 0.0f);
  }
  __syncwarp();
  float pa[4], pc[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    float2 wv[16];
    float hs[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) wv[e] = reinterpret_cast<const float2*>(w + kW2 + (16 * r + e) * 64)[lane];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 hv = reinterpret_cast<const float4*>(h1)[4 * r + q];
      hs[4 * q] = hv.x;
      hs[4 * q + 1] = hv.y;
      hs[4 * q + 2] = hv.z;
      hs[4 * q + 3] = hv.w;
    }
    pa[r] = 0.0f;
    pc[r] = 0.0f;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      pa[r] = fmaf(hs[e], wv[e].x, pa[r]);
      pc[r] = fmaf(hs[e], wv[e].y, pc[r]);
    }
  }
  const float2 bias2 = reinterpret_cast<const float2*>(w + kB2)[lane];
  const float h2a = fmaxf(((pa[0] + pa[1]) + (pa[2] + pa[3])) + bias2.x, 0.0f);
  const float h2c = fmaxf(((pc[0] + pc[1]) + (pc[2] + pc[3])) + bias2.y, 0.0f);
  const float4 w3a = reinterpret_cast<const float4*>(w + kW3)[lane];
  const float4 w3c = reinterpret_cast<const float4*>(w + kW3)[lane + 32];
  const float4 b3 = *reinterpret_cast<const float4*>(w + kB3);
  float y[4] = {fmaf(h2c, w3c.x, h2a * w3a.x), fmaf(h2c, w3c.y, h2a * w3a.y), fmaf(h2c, w3c.z, h2a * w3a.z),
                fmaf(h2c, w3c.w, h2a * w3a.w)};
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1)
#pragma unroll
    for (int o = 0; o < 4; ++o) y[o] = y[o] + __shfl_xor_sync(0xffffffffu, y[o], m);
  y[0] += b3.x;
  y[1] += b3.y;
  y[2] += b3.z;
  y[3] += b3.w;
  int best = 0;
  float yb = y[0];
#pragma unroll
  for (int o = 1; o < 4; ++o)
    if (y[o] < yb) {
      best = o;
      yb = y[o];
    }
  return best;
}

}  // namespace bfsdev
