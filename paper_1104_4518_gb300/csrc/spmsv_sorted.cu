// Sorted-output SpMSV over the (select2nd, max) semiring, and the BFS of
// Algorithm 3 with one process built from it (Sec. 4.2).
//
// Sec. 4.2 forms the union of the adjacency columns that the frontier's
// nonzeros select in one of two ways: a sparse accumulator (a dense value
// vector, occupancy flags and a list of the occupied indices, which must be
// sorted afterwards) or a priority-queue multiway merge of the columns, which
// yields the output already sorted.  The level-loop kernel is an accumulator
// on the device (the parent array and the next bitmap; its queue is
// unsorted).  This file is the merge, done the way a GPU merges many lists:
// every entry (w, u) of a selected column u whose row w is not masked becomes
// one 64-bit key w << b | u (b bits hold any vertex id), a stable radix sort on
// the 2b key bits merges the columns, and the last key of each row's run holds
// the row's largest frontier id, which is the semiring's sum.  The output
// comes out with ascending indices.
#include <algorithm>
#include <string>

#include "device_common.cuh"
#include "internal.h"
#include "nvtx_range.h"

namespace bfsint {
namespace {

constexpr int kThreads = 256;

int id_bits(int32_t n) {  // bits that hold every id in [0, n)
  int b = 1;
  while (b < 31 && ((int64_t)1 << b) < (int64_t)n) ++b;
  return b;
}

unsigned blocks_for(long long work) {
  return (unsigned)std::max(1ll, std::min((work + kThreads - 1) / kThreads, 1ll << 20));
}

// Sum of the frontier's column lengths (an upper bound on the keys); a
// frontier id outside [0, n) sets bad[0] and is recorded in bad[1].
__global__ void frontier_degree_kernel(const int64_t* __restrict__ off, int32_t n, const int32_t* __restrict__ f,
                                       long long nf, unsigned long long* sum, long long* bad) {
  unsigned long long acc = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += (long long)gridDim.x * blockDim.x) {
    const int u = f[i];
    if (u < 0 || u >= n) {
      if (atomicCAS(reinterpret_cast<unsigned long long*>(bad), 0ull, 1ull) == 0ull) bad[1] = u;
      continue;
    }
    acc += (unsigned long long)(off[u + 1] - off[u]);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(bfsdev::kFull, acc, o);
  if ((threadIdx.x & 31) == 0 && acc) atomicAdd(sum, acc);
}

// One warp per frontier entry u: the keys w << b | u of u's column entries w
// that the mask leaves (visited == nullptr: no mask), appended with one atomic
// per warp step.  An entry outside [0, n) (a malformed graph) sets bad[2] and
// is recorded in bad[3].
__global__ void expand_kernel(const int64_t* __restrict__ off, const int32_t* __restrict__ adj, int32_t n,
                              const int32_t* __restrict__ f, long long nf, const uint32_t* __restrict__ visited,
                              int b, uint64_t* __restrict__ keys, unsigned long long* count, long long* bad) {
  const int lane = threadIdx.x & 31;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long i = gw; i < nf; i += nw) {
    const int u = f[i];  // checked by frontier_degree_kernel
    const long long rb = off[u], re = off[u + 1];
    for (long long j0 = rb; j0 < re; j0 += 32) {
      const long long j = j0 + lane;
      bool keep = false;
      int w = 0;
      if (j < re) {
        w = adj[j];
        if (w < 0 || w >= n) {
          if (atomicCAS(reinterpret_cast<unsigned long long*>(bad + 2), 0ull, 1ull) == 0ull) bad[3] = w;
        } else {
          keep = visited == nullptr || !((visited[w >> 5] >> (w & 31)) & 1u);
        }
      }
      const unsigned m = __ballot_sync(bfsdev::kFull, keep);
      if (!m) continue;
      unsigned long long base = 0;
      if (lane == 0) base = atomicAdd(count, (unsigned long long)__popc(m));
      base = __shfl_sync(bfsdev::kFull, base, 0);
      if (keep) keys[base + __popc(m & bfsdev::lanemask_lt())] = ((uint64_t)w << b) | (uint64_t)u;
    }
  }
}

// flag[i] = 1 where key i ends its row's run (the row's largest frontier id).
__global__ void run_end_kernel(const uint64_t* __restrict__ keys, long long N, int b, uint32_t* __restrict__ flag) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    flag[i] = (i + 1 == N || (keys[i] >> b) != (keys[i + 1] >> b)) ? 1u : 0u;
}

__global__ void compress_kernel(const uint64_t* __restrict__ keys, long long N, int b,
                                const uint32_t* __restrict__ flag, const int64_t* __restrict__ pos,
                                int32_t* __restrict__ out_idx, int32_t* __restrict__ out_val) {
  const uint64_t low = ((uint64_t)1 << b) - 1;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    if (flag[i]) {
      out_idx[pos[i]] = (int32_t)(keys[i] >> b);
      out_val[pos[i]] = (int32_t)(keys[i] & low);
    }
}

// BFS state of bfs_run_sorted: outputs -1, the source at level 0, its bit visited.
__global__ void sorted_init_kernel(int32_t n, int32_t s, int32_t* __restrict__ parent, int32_t* __restrict__ level,
                                   uint32_t* __restrict__ visited, long long nwords) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    parent[v] = v == s ? s : -1;
    level[v] = v == s ? 0 : -1;
  }
  for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < nwords; w += stride)
    visited[w] = w == (s >> 5) ? 1u << (s & 31) : 0u;
}

// pi <- pi + t (a masked assignment: t holds unvisited rows only), levels, and
// the visited bits of the new frontier.
__global__ void sorted_apply_kernel(const int32_t* __restrict__ idx, const int32_t* __restrict__ val, long long cnt,
                                    int32_t lev, int32_t* __restrict__ parent, int32_t* __restrict__ level,
                                    uint32_t* __restrict__ visited) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (long long)gridDim.x * blockDim.x) {
    const int v = idx[i];
    parent[v] = val[i];
    level[v] = lev;
    atomicOr(&visited[v >> 5], 1u << (v & 31));
  }
}

}  // namespace

// t = A (x) f masked by not(visited), sorted by index (see the file comment).
// Synchronises s.
int spmsv_sorted(const bfs_graph* g, const int32_t* f, long long nf, const uint32_t* visited, int32_t* out_idx,
                 int32_t* out_val, long long* out_count, cudaStream_t s) {
  *out_count = 0;
  if (nf == 0 || g->n == 0) return BFS_OK;
  const int b = id_bits(g->n);
  unsigned long long* d_ctr = nullptr;  // [0] degree sum, [1] key count
  long long* d_bad = nullptr;
  uint64_t* keys = nullptr;
  uint64_t* alt = nullptr;
  uint32_t* flag = nullptr;
  int64_t* pos = nullptr;
  auto cleanup = [&]() {
    for (void* p : {(void*)d_ctr, (void*)d_bad, (void*)keys, (void*)alt, (void*)flag, (void*)pos})
      if (p) cudaFree(p);
  };
  int rc = dev_alloc((void**)&d_ctr, 2 * sizeof(unsigned long long), "SpMSV counters");
  if (!rc) rc = dev_alloc((void**)&d_bad, 4 * sizeof(long long), "SpMSV flags");
  if (rc) return cleanup(), rc;
  cudaError_t err = cudaMemsetAsync(d_ctr, 0, 2 * sizeof(unsigned long long), s);
  if (err == cudaSuccess) err = cudaMemsetAsync(d_bad, 0, 4 * sizeof(long long), s);
  if (err != cudaSuccess) return cleanup(), cuda_fail(err, "SpMSV state");
  frontier_degree_kernel<<<blocks_for(nf), kThreads, 0, s>>>(g->d_off, g->n, f, nf, d_ctr, d_bad);
  unsigned long long h_ctr[2] = {0, 0};
  long long h_bad[4] = {0, 0, 0, 0};
  err = cudaGetLastError();
  if (err == cudaSuccess) err = cudaMemcpyAsync(h_ctr, d_ctr, sizeof(h_ctr), cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess) err = cudaMemcpyAsync(h_bad, d_bad, sizeof(h_bad), cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  if (err != cudaSuccess) return cleanup(), cuda_fail(err, "SpMSV frontier degrees");
  if (h_bad[0])
    return cleanup(), fail(BFS_ERR_INVALID_ARG, "bfs_spmsv_sorted: frontier id " + std::to_string(h_bad[1]) +
                                                    " outside [0, n)");
  const long long cap = (long long)h_ctr[0];
  if (cap == 0) return cleanup(), BFS_OK;
  rc = dev_alloc((void**)&keys, sizeof(uint64_t) * cap, "SpMSV keys");
  if (!rc) rc = dev_alloc((void**)&alt, sizeof(uint64_t) * cap, "SpMSV sort scratch");
  if (rc) return cleanup(), rc;
  expand_kernel<<<blocks_for(nf * 32), kThreads, 0, s>>>(g->d_off, g->d_adj, g->n, f, nf, visited, b, keys,
                                                          d_ctr + 1, d_bad);
  err = cudaGetLastError();
  if (err == cudaSuccess) err = cudaMemcpyAsync(h_ctr, d_ctr, sizeof(h_ctr), cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess) err = cudaMemcpyAsync(h_bad, d_bad, sizeof(h_bad), cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  if (err != cudaSuccess) return cleanup(), cuda_fail(err, "SpMSV expansion");
  if (h_bad[2])
    return cleanup(), fail(BFS_ERR_INVALID_GRAPH, "bfs_spmsv_sorted: adjacency id " + std::to_string(h_bad[3]) +
                                                      " outside [0, n)");
  const long long N = (long long)h_ctr[1];
  if (N == 0) return cleanup(), BFS_OK;
  uint64_t* sorted = nullptr;
  if ((rc = radix_sort_u64(keys, alt, N, 0, 2 * b, s, &sorted))) return cleanup(), rc;
  rc = dev_alloc((void**)&flag, sizeof(uint32_t) * N, "SpMSV run ends");
  if (!rc) rc = dev_alloc((void**)&pos, sizeof(int64_t) * N, "SpMSV output slots");
  if (rc) return cleanup(), rc;
  run_end_kernel<<<blocks_for(N), kThreads, 0, s>>>(sorted, N, b, flag);
  if ((err = cudaGetLastError()) != cudaSuccess) return cleanup(), cuda_fail(err, "SpMSV run ends");
  long long total = 0;
  if ((rc = exclusive_scan_u32(flag, N, pos, s, &total))) return cleanup(), rc;
  compress_kernel<<<blocks_for(N), kThreads, 0, s>>>(sorted, N, b, flag, pos, out_idx, out_val);
  err = cudaGetLastError();
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  cleanup();
  if (err != cudaSuccess) return cuda_fail(err, "SpMSV compression");
  *out_count = total;
  return BFS_OK;
}

}  // namespace bfsint

using namespace bfsint;

extern "C" {

int bfs_spmsv_sorted(bfs_graph* g, const int32_t* frontier, int32_t nf, const uint32_t* visited, int32_t* out_idx,
                     int32_t* out_val, int32_t* out_count, void* stream) {
  NvtxRange nvtx_range("bfs_spmsv_sorted");
  if (!g) return fail(BFS_ERR_INVALID_ARG, "NULL graph");
  if (!out_count) return fail(BFS_ERR_INVALID_ARG, "bfs_spmsv_sorted: NULL out_count");
  *out_count = 0;
  if (nf < 0) return fail(BFS_ERR_INVALID_ARG, "bfs_spmsv_sorted: negative frontier size");
  if (nf > 0 && (!frontier || !out_idx || !out_val)) return fail(BFS_ERR_INVALID_ARG, "bfs_spmsv_sorted: NULL array");
  long long cnt = 0;
  if (int e = spmsv_sorted(g, frontier, nf, visited, out_idx, out_val, &cnt, (cudaStream_t)stream)) return e;
  *out_count = (int32_t)cnt;
  return BFS_OK;
}

int bfs_run_sorted(bfs_graph* g, int32_t source, int32_t* parent_out, int32_t* level_out, void* stream) {
  NvtxRange nvtx_range("bfs_run_sorted");
  if (!g) return fail(BFS_ERR_INVALID_ARG, "NULL graph");
  if (source < 0 || source >= g->n) return fail(BFS_ERR_INVALID_ARG, "bfs_run_sorted: source outside [0, n)");
  if (!parent_out || !level_out) return fail(BFS_ERR_INVALID_ARG, "bfs_run_sorted: NULL output");
  cudaStream_t s = (cudaStream_t)stream;
  const int32_t n = g->n;
  const long long nwords = ((long long)n + 31) / 32;
  uint32_t* visited = nullptr;
  int32_t* fa = nullptr;  // frontier of the level
  int32_t* fb = nullptr;  // indices of t
  int32_t* tv = nullptr;  // values of t
  auto cleanup = [&]() {
    for (void* p : {(void*)visited, (void*)fa, (void*)fb, (void*)tv})
      if (p) cudaFree(p);
  };
  int rc = dev_alloc((void**)&visited, sizeof(uint32_t) * nwords, "visited bitmap");
  if (!rc) rc = dev_alloc((void**)&fa, sizeof(int32_t) * n, "frontier");
  if (!rc) rc = dev_alloc((void**)&fb, sizeof(int32_t) * n, "SpMSV indices");
  if (!rc) rc = dev_alloc((void**)&tv, sizeof(int32_t) * n, "SpMSV values");
  if (rc) return cleanup(), rc;
  sorted_init_kernel<<<blocks_for(n), kThreads, 0, s>>>(n, source, parent_out, level_out, visited, nwords);
  cudaError_t err = cudaGetLastError();
  if (err == cudaSuccess) err = cudaMemcpyAsync(fa, &source, sizeof(int32_t), cudaMemcpyHostToDevice, s);
  if (err != cudaSuccess) return cleanup(), cuda_fail(err, "sorted BFS init");
  long long nf = 1;
  for (int32_t k = 0; nf > 0; ++k) {  // f <- t while t is not empty
    long long cnt = 0;
    if ((rc = spmsv_sorted(g, fa, nf, visited, fb, tv, &cnt, s))) return cleanup(), rc;
    if (cnt > 0) {
      sorted_apply_kernel<<<blocks_for(cnt), kThreads, 0, s>>>(fb, tv, cnt, k + 1, parent_out, level_out, visited);
      if ((err = cudaGetLastError()) != cudaSuccess) return cleanup(), cuda_fail(err, "sorted BFS update");
    }
    std::swap(fa, fb);
    nf = cnt;
  }
  err = cudaStreamSynchronize(s);
  cleanup();
  if (err != cudaSuccess) return cuda_fail(err, "sorted BFS");
  return BFS_OK;
}

}  // extern "C"
