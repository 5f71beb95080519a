// Symmetric half storage of an undirected graph and a BFS over it.
//
// The paper's closing notes point out that an undirected graph's adjacency
// matrix is symmetric, so one triangle holds it whole at half the memory.
// Here the kept triangle U has, in row v, the entries w > v of v's row (rows
// stay sorted).  A vertex's neighbours above its own id are then in its own U
// row and those below it in theirs (w with v in U row w), so a level of the
// BFS takes two passes over U, in separate launches:
// 1. pull: each unvisited v scans its U row from the top; the first frontier
//    entry is v's largest frontier neighbour above v, hence its parent (it is
//    larger than any neighbour below v);
// 2. push: each frontier vertex u offers itself with atomicMax to the entries
//    w of its U row that are unvisited and that pass 1 left unreached; the
//    largest offer, all from neighbours below w, is w's parent.
// The two passes reach disjoint sets whose union is the next frontier, so
// levels and parents are those of bfs_run.  Both passes take a 32-vertex
// bitmap word per warp and walk a row with the whole warp.
#include <algorithm>
#include <mutex>
#include <string>
#include <unordered_map>

#include "device_common.cuh"
#include "internal.h"
#include "nvtx_range.h"

namespace bfsint {
namespace {

constexpr int kThreads = 256;

// U of each graph that has one, owned by this file (the graph struct that the
// kernels share stays as it is); freed with the graph.
struct HalfSet {
  int64_t* off = nullptr;
  int32_t* adj = nullptr;
  int64_t nnz = 0;
};
std::mutex g_half_mu;
std::unordered_map<const bfs_graph*, HalfSet> g_half;

unsigned blocks_for(long long work) {
  return (unsigned)std::max(1ll, std::min((work + kThreads - 1) / kThreads, 1ll << 20));
}

// cnt[v] = entries of row v above v (rows ascending: the row's length minus
// the position of its first entry > v).
__global__ void half_count_kernel(const int64_t* __restrict__ off, const int32_t* __restrict__ adj, int32_t n,
                                  uint32_t* __restrict__ cnt) {
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
    long long lo = off[v], hi = off[v + 1];
    const long long end = hi;
    while (lo < hi) {  // first position with adj > v
      const long long mid = (lo + hi) >> 1;
      if (adj[mid] > v) hi = mid;
      else lo = mid + 1;
    }
    cnt[v] = (uint32_t)(end - lo);
  }
}

// U row v = the last hoff[v+1] - hoff[v] entries of row v; one warp per row.
__global__ void half_copy_kernel(const int64_t* __restrict__ off, const int32_t* __restrict__ adj, int32_t n,
                                 const int64_t* __restrict__ hoff, int32_t* __restrict__ hadj) {
  const int lane = threadIdx.x & 31;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long v = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += nw) {
    const long long len = hoff[v + 1] - hoff[v];
    const long long src = off[v + 1] - len;
    for (long long i = lane; i < len; i += 32) hadj[hoff[v] + i] = adj[src + i];
  }
}

__global__ void half_init_kernel(int32_t n, int32_t s, int32_t* __restrict__ parent, int32_t* __restrict__ level,
                                 uint32_t* __restrict__ vis, uint32_t* __restrict__ cur, uint32_t* __restrict__ na,
                                 uint32_t* __restrict__ nb, long long nwords) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    parent[v] = v == s ? s : -1;
    level[v] = v == s ? 0 : -1;
  }
  for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < nwords; w += stride) {
    const uint32_t sb = w == (s >> 5) ? 1u << (s & 31) : 0u;
    vis[w] = sb;
    cur[w] = sb;
    na[w] = 0u;
    nb[w] = 0u;
  }
}

// Pass 1: warp per word of 32 vertices; each unvisited vertex's U row is
// scanned by the warp, 32 entries per step from the top; the lowest lane with
// a frontier entry holds the row's largest one.  The warp owns its word of na.
__global__ void half_pull_kernel(const int64_t* __restrict__ hoff, const int32_t* __restrict__ hadj, int32_t n,
                                 int32_t lev, const uint32_t* __restrict__ vis, const uint32_t* __restrict__ cur,
                                 uint32_t* __restrict__ na, int32_t* __restrict__ parent, int32_t* __restrict__ level,
                                 long long nwords) {
  const int lane = threadIdx.x & 31;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long wi = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; wi < nwords; wi += nw) {
    const long long v0 = wi * 32;
    const uint32_t valid = n - v0 >= 32 ? 0xffffffffu : ((1u << (n - v0)) - 1u);
    uint32_t open = ~vis[wi] & valid;
    uint32_t found = 0u;
    while (open) {
      const int bit = __ffs(open) - 1;
      open &= open - 1u;
      const int v = (int)(v0 + bit);
      const long long b = hoff[v];
      for (long long hi = hoff[v + 1]; hi > b; hi -= 32) {
        const long long j = hi - 1 - lane;
        const int u = j >= b ? hadj[j] : -1;
        const bool hit = u >= 0 && ((cur[u >> 5] >> (u & 31)) & 1u);
        const unsigned m = __ballot_sync(bfsdev::kFull, hit);
        if (m) {
          if (lane == __ffs(m) - 1) {
            parent[v] = u;
            level[v] = lev;
          }
          found |= 1u << bit;
          break;
        }
      }
    }
    if (lane == 0 && found) na[wi] = found;
  }
}

// Pass 2: warp per word of the frontier; each frontier vertex u's U row is
// walked by the warp, offering u to every entry w not visited and not reached
// by pass 1.
__global__ void half_push_kernel(const int64_t* __restrict__ hoff, const int32_t* __restrict__ hadj, int32_t lev,
                                 const uint32_t* __restrict__ vis, const uint32_t* __restrict__ cur,
                                 const uint32_t* __restrict__ na, uint32_t* __restrict__ nb,
                                 int32_t* __restrict__ parent, int32_t* __restrict__ level, long long nwords) {
  const int lane = threadIdx.x & 31;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long wi = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; wi < nwords; wi += nw) {
    uint32_t f = cur[wi];
    while (f) {
      const int bit = __ffs(f) - 1;
      f &= f - 1u;
      const int u = (int)(wi * 32 + bit);
      for (long long j = hoff[u] + lane; j < hoff[u + 1]; j += 32) {
        const int w = hadj[j];
        const uint32_t m = 1u << (w & 31);
        if ((vis[w >> 5] | na[w >> 5]) & m) continue;
        atomicMax(&parent[w], u);
        level[w] = lev;
        atomicOr(&nb[w >> 5], m);
      }
    }
  }
}

// The next frontier (na | nb) becomes cur and joins vis; na, nb cleared; its size counted.
__global__ void half_finish_kernel(uint32_t* __restrict__ vis, uint32_t* __restrict__ cur, uint32_t* __restrict__ na,
                                   uint32_t* __restrict__ nb, long long nwords, unsigned long long* count) {
  unsigned long long c = 0;
  for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < nwords; w += (long long)gridDim.x * blockDim.x) {
    const uint32_t f = na[w] | nb[w];
    cur[w] = f;
    vis[w] |= f;
    na[w] = 0u;
    nb[w] = 0u;
    c += (unsigned long long)__popc(f);
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(bfsdev::kFull, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

// U of g, built on first use (caller holds g->mu).  Synchronises s.
int ensure_half(bfs_graph* g, cudaStream_t s, HalfSet* out) {
  {
    std::lock_guard<std::mutex> lk(g_half_mu);
    auto it = g_half.find(g);
    if (it != g_half.end()) {
      *out = it->second;
      return BFS_OK;
    }
  }
  if (g->directed) return fail(BFS_ERR_UNSUPPORTED, "half storage needs an undirected graph");
  const int32_t n = g->n;
  uint32_t* cnt = nullptr;
  int64_t* hoff = nullptr;
  int32_t* hadj = nullptr;
  int rc = dev_alloc((void**)&cnt, sizeof(uint32_t) * std::max(1, n), "half-row counts");
  if (!rc) rc = dev_alloc((void**)&hoff, sizeof(int64_t) * ((size_t)n + 1), "half offsets");
  if (rc) {
    if (cnt) cudaFree(cnt);
    return rc;
  }
  half_count_kernel<<<blocks_for(n), kThreads, 0, s>>>(g->d_off, g->d_adj, n, cnt);
  long long total = 0;
  cudaError_t err = cudaGetLastError();
  if (err == cudaSuccess) rc = exclusive_scan_u32(cnt, n, hoff, s, &total);
  if (err == cudaSuccess && !rc) err = cudaMemcpyAsync(hoff + n, &total, sizeof(int64_t), cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess && !rc) err = cudaStreamSynchronize(s);
  cudaFree(cnt);
  if (!rc && err == cudaSuccess) rc = dev_alloc((void**)&hadj, sizeof(int32_t) * std::max(1ll, total), "half adjacency");
  if (!rc && err == cudaSuccess) {
    half_copy_kernel<<<blocks_for((long long)n * 32), kThreads, 0, s>>>(g->d_off, g->d_adj, n, hoff, hadj);
    err = cudaGetLastError();
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  }
  if (rc || err != cudaSuccess) {
    cudaFree(hoff);
    if (hadj) cudaFree(hadj);
    return rc ? rc : cuda_fail(err, "half storage");
  }
  HalfSet h;
  h.off = hoff;
  h.adj = hadj;
  h.nnz = total;
  std::lock_guard<std::mutex> lk(g_half_mu);
  g_half[g] = h;
  *out = h;
  return BFS_OK;
}

}  // namespace

void free_half(const bfs_graph* g) {
  std::lock_guard<std::mutex> lk(g_half_mu);
  auto it = g_half.find(g);
  if (it == g_half.end()) return;
  cudaFree(it->second.off);
  cudaFree(it->second.adj);
  g_half.erase(it);
}

}  // namespace bfsint

using namespace bfsint;

extern "C" {

int bfs_graph_half(bfs_graph* g, bfs_half_info* info, void* stream) {
  NvtxRange nvtx_range("bfs_graph_half");
  if (!g) return fail(BFS_ERR_INVALID_ARG, "NULL graph");
  if (!info) return fail(BFS_ERR_INVALID_ARG, "bfs_graph_half: NULL info");
  std::lock_guard<std::mutex> lk(g->mu);
  HalfSet h;
  if (int e = ensure_half(g, (cudaStream_t)stream, &h)) return e;
  info->nnz = h.nnz;
  info->offsets = h.off;
  info->adj = h.adj;
  return BFS_OK;
}

int bfs_run_half(bfs_graph* g, int32_t source, int32_t* parent_out, int32_t* level_out, void* stream) {
  NvtxRange nvtx_range("bfs_run_half");
  if (!g) return fail(BFS_ERR_INVALID_ARG, "NULL graph");
  if (source < 0 || source >= g->n) return fail(BFS_ERR_INVALID_ARG, "bfs_run_half: source outside [0, n)");
  if (!parent_out || !level_out) return fail(BFS_ERR_INVALID_ARG, "bfs_run_half: NULL output");
  cudaStream_t s = (cudaStream_t)stream;
  HalfSet h;
  {
    std::lock_guard<std::mutex> lk(g->mu);
    if (int e = ensure_half(g, s, &h)) return e;
  }
  const int32_t n = g->n;
  const long long nwords = ((long long)n + 31) / 32;
  uint32_t* bits = nullptr;  // vis, cur, na, nb
  unsigned long long* count = nullptr;
  int rc = dev_alloc((void**)&bits, sizeof(uint32_t) * 4 * nwords, "half BFS bitmaps");
  if (!rc) rc = dev_alloc((void**)&count, sizeof(unsigned long long), "half BFS count");
  auto cleanup = [&]() {
    if (bits) cudaFree(bits);
    if (count) cudaFree(count);
  };
  if (rc) return cleanup(), rc;
  uint32_t *vis = bits, *cur = bits + nwords, *na = bits + 2 * nwords, *nb = bits + 3 * nwords;
  half_init_kernel<<<blocks_for(std::max((long long)n, nwords)), kThreads, 0, s>>>(n, source, parent_out, level_out,
                                                                                   vis, cur, na, nb, nwords);
  cudaError_t err = cudaGetLastError();
  const unsigned wblocks = blocks_for(nwords * 32);
  for (int32_t lev = 1; err == cudaSuccess; ++lev) {
    half_pull_kernel<<<wblocks, kThreads, 0, s>>>(h.off, h.adj, n, lev, vis, cur, na, parent_out,
                                                  level_out, nwords);
    half_push_kernel<<<wblocks, kThreads, 0, s>>>(h.off, h.adj, lev, vis, cur, na, nb, parent_out,
                                                  level_out, nwords);
    unsigned long long h = 0;
    err = cudaMemsetAsync(count, 0, sizeof(unsigned long long), s);
    if (err == cudaSuccess) {
      half_finish_kernel<<<blocks_for(nwords), kThreads, 0, s>>>(vis, cur, na, nb, nwords, count);
      err = cudaGetLastError();
    }
    if (err == cudaSuccess) err = cudaMemcpyAsync(&h, count, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if (h == 0) break;
  }
  cleanup();
  if (err != cudaSuccess) return cuda_fail(err, "half-storage BFS");
  return BFS_OK;
}

}  // extern "C"
