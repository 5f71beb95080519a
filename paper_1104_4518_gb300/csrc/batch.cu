// Batched BFS: up to 64 roots in one persistent traversal.
//
// Every vertex carries three 64-bit words: F_k[v] (bit r set when v is in the
// frontier of root r at level k), V[v] (bit r set when root r has reached v)
// and F_{k+1}[v].  One level is the boolean sparse matrix-dense matrix product
// F_{k+1} = (A (x) F_k) AND NOT V, i.e. the SpMSV of Sec. 3.2 for 64 vectors at
// once.  Parents follow the same max-id rule as the single-root traversal: for
// a vertex v newly reached by root r, parent_r[v] is the largest neighbour u
// with bit r in F_k[u], found by scanning v's sorted row from the largest id
// down and masking off the bits already resolved.
//
// Two ways to expand a level (identical results):
//   pull      : every vertex not reached by all roots scans its row (one phase);
//   top-down  : vertices of the frontier queue OR their bits into F_{k+1} of
//               their neighbours (first writer enqueues), then every queued
//               vertex resolves its parents with the same descending scan
//               (two phases).
// Output rows are root-major: level[r * n + v], parent[r * n + v].
#include "device_common.cuh"
#include "internal.h"

namespace bfsint {
namespace {

using bfsdev::kFull;

constexpr int kBBlock = 512;

struct BatchParams {
  const int64_t* __restrict__ off;
  const int32_t* __restrict__ adj;
  int32_t n;
  long long nnz;
  int32_t k;  // roots in this traversal (<= 64)
  uint64_t mask;
  int32_t src[64];
  int32_t* level;   // [k][n]
  int32_t* parent;  // [k][n]
  uint64_t* F[3];
  uint64_t* V;
  int32_t* queue[3];
  LevelCtr* ctr;
  bfsdev::GridBarrier* bar;
  int* status;
  int32_t* misc;
  unsigned spin_limit;
  long long td_limit;
};

// Writes level / parent of the roots in `bits` for vertex v.
__device__ __forceinline__ void write_hits(const BatchParams& p, uint64_t bits, int v, int u, int lvl) {
  while (bits) {
    const int r = __ffsll((long long)bits) - 1;
    bits &= bits - 1;
    const long long o = (long long)r * p.n + v;
    p.level[o] = lvl;
    p.parent[o] = u;
  }
}

// Descending scan of v's row: resolves the parents of the roots in `need`
// whose frontier (F) contains a neighbour; returns the bits found.
__device__ __forceinline__ uint64_t resolve_row(const BatchParams& p, const uint64_t* F, int v, uint64_t need,
                                                int lvl) {
  const long long b = __ldg(&p.off[v]);
  uint64_t found = 0;
  for (long long j = __ldg(&p.off[v + 1]) - 1; j >= b && need; --j) {
    const int u = __ldg(&p.adj[j]);
    const uint64_t h = F[u] & need;
    if (h) {
      write_hits(p, h, v, u, lvl);
      need &= ~h;
      found |= h;
    }
  }
  return found;
}

__device__ __forceinline__ void enqueue_warp(const BatchParams& p, int knext, int v, bool pred) {
  const unsigned m = __ballot_sync(kFull, pred);
  if (!m) return;
  const int lane = threadIdx.x & 31;
  unsigned base = 0;
  if (lane == 0) base = atomicAdd(&p.ctr[knext % kCtrRing].count, (unsigned)__popc(m));
  base = __shfl_sync(kFull, base, 0);
  if (pred) p.queue[knext % 3][base + __popc(m & bfsdev::lanemask_lt())] = v;
}

__global__ void __launch_bounds__(kBBlock) batch_kernel(BatchParams p) {
  const int tid = threadIdx.x;
  unsigned epoch = 0;
  if (tid == 0) epoch = bfsdev::ld_acquire_u32(&p.bar->epoch);
  const long long gtid = (long long)blockIdx.x * kBBlock + tid;
  const long long gthreads = (long long)gridDim.x * kBBlock;
  const unsigned nblocks = gridDim.x;

  // init: outputs to -1, bitsets to 0, counters to 0
  const long long total = (long long)p.k * p.n;
  for (long long i = gtid; i < total; i += gthreads) {
    p.level[i] = -1;
    p.parent[i] = -1;
  }
  for (long long v = gtid; v < p.n; v += gthreads) {
    p.F[0][v] = 0;
    p.F[1][v] = 0;
    p.F[2][v] = 0;
    p.V[v] = 0;
  }
  if (blockIdx.x == 0 && tid < kCtrRing * (int)(sizeof(LevelCtr) / 8))
    reinterpret_cast<unsigned long long*>(p.ctr)[tid] = 0ull;
  if (!bfsdev::grid_barrier(p.bar, nblocks, epoch, p.spin_limit, p.status)) return;

  // seed: root r sets bit r of its own vertex (roots may repeat)
  if (blockIdx.x == 0 && tid < p.k) {
    const int s = p.src[tid];
    const uint64_t bit = 1ull << tid;
    const long long o = (long long)tid * p.n + s;
    p.level[o] = 0;
    p.parent[o] = s;
    atomicOr((unsigned long long*)&p.V[s], (unsigned long long)bit);
    const unsigned long long old = atomicOr((unsigned long long*)&p.F[0][s], (unsigned long long)bit);
    if (old == 0) {
      const unsigned pos = atomicAdd(&p.ctr[0].count, 1u);
      p.queue[0][pos] = s;
    }
  }
  if (!bfsdev::grid_barrier(p.bar, nblocks, epoch, p.spin_limit, p.status)) return;

  int k = 0;
  for (;; ++k) {
    const unsigned count = __ldcg(&p.ctr[k % kCtrRing].count);
    if (count == 0) break;
    const uint64_t* Fc = p.F[k % 3];
    uint64_t* Fn = p.F[(k + 1) % 3];
    const int32_t* Q = p.queue[k % 3];
    const int knext = k + 1;
    if (blockIdx.x == 0 && tid < (int)(sizeof(LevelCtr) / 8))
      reinterpret_cast<unsigned long long*>(&p.ctr[(k + 4) % kCtrRing])[tid] = 0ull;
    if (k >= 1) {  // clear F_{k-1} for reuse as F_{k+2}
      uint64_t* clr = p.F[(k + 2) % 3];
      const unsigned pc = __ldcg(&p.ctr[(k + kCtrRing - 1) % kCtrRing].count);
      if ((long long)pc * 8 < p.n) {
        const int32_t* PQ = p.queue[(k + 2) % 3];
        for (long long i = gtid; i < pc; i += gthreads) clr[PQ[i]] = 0;
      } else {
        for (long long v = gtid; v < p.n; v += gthreads) clr[v] = 0;
      }
    }

    if ((long long)count <= p.td_limit) {
      // top-down discover: OR frontier bits into unreached neighbours
      for (long long i = gtid; i < count; i += gthreads) {
        const int u = Q[i];
        const uint64_t f = Fc[u];
        const long long b = __ldg(&p.off[u]), e = __ldg(&p.off[u + 1]);
        for (long long j = b; j < e; ++j) {
          const int w = __ldg(&p.adj[j]);
          const uint64_t nb = f & ~p.V[w];
          if (!nb || (Fn[w] & nb) == nb) continue;
          const unsigned long long old = atomicOr((unsigned long long*)&Fn[w], (unsigned long long)nb);
          if (old == 0) {
            const unsigned pos = atomicAdd(&p.ctr[knext % kCtrRing].count, 1u);
            p.queue[knext % 3][pos] = w;
          }
        }
      }
      if (!bfsdev::grid_barrier(p.bar, nblocks, epoch, p.spin_limit, p.status)) return;
      // resolve parents of the newly reached (vertex, root) pairs
      const unsigned ncount = __ldcg(&p.ctr[knext % kCtrRing].count);
      const int32_t* NQ = p.queue[knext % 3];
      for (long long i = gtid; i < ncount; i += gthreads) {
        const int w = NQ[i];
        const uint64_t need = Fn[w];
        resolve_row(p, Fc, w, need, knext);
        p.V[w] |= need;
      }
    } else {
      // pull: every vertex with unreached roots scans its row
      const long long nw = ((long long)p.n + 31) / 32 * 32;
      for (long long v0 = gtid; v0 < nw; v0 += gthreads) {
        const int v = (int)v0;
        uint64_t found = 0;
        if (v0 < p.n) {
          const uint64_t need = ~p.V[v] & p.mask;
          if (need) found = resolve_row(p, Fc, v, need, knext);
          if (found) {
            Fn[v] = found;
            p.V[v] |= found;
          }
        }
        enqueue_warp(p, knext, v, found != 0);
      }
    }
    if (!bfsdev::grid_barrier(p.bar, nblocks, epoch, p.spin_limit, p.status)) return;
  }
  if (gtid == 0) p.misc[1] = k;
}

}  // namespace

int launch_batch(const BatchRequest& r, cudaStream_t s) {
  bfs_graph* g = r.g;
  Workspace* w = r.w;
  DeviceInfo di;
  if (int e = current_device_info(&di)) return e;
  if (r.k < 1 || r.k > 64) return fail(BFS_ERR_INVALID_ARG, "batch of 1..64 roots expected");
  if (int e = ensure_batch_state(g, w)) return e;
  const bfs_tuning t = effective_tuning(g);
  BatchParams p{};
  p.off = g->d_off;
  p.adj = g->d_adj;
  p.n = g->n;
  p.nnz = g->nnz;
  p.k = r.k;
  p.mask = r.k == 64 ? ~0ull : ((1ull << r.k) - 1ull);
  for (int i = 0; i < r.k; ++i) p.src[i] = r.h_sources[i];
  p.level = r.level;
  p.parent = r.parent;
  for (int i = 0; i < 3; ++i) {
    p.F[i] = w->bset[i];
    p.queue[i] = w->queue[i];
  }
  p.V = w->bvis;
  p.ctr = w->ctr;
  p.bar = reinterpret_cast<bfsdev::GridBarrier*>(w->barrier);
  p.status = w->status;
  p.misc = w->misc;
  p.spin_limit = r.spin_limit ? r.spin_limit : (1u << 25);
  p.td_limit = t.batch_topdown_limit;
  int per_sm = 0;
  BFS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel, kBBlock, 0));
  if (per_sm < 1) return fail(BFS_ERR_CUDA, "batch kernel cannot be resident");
  void* args[] = {&p};
  BFS_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)batch_kernel, dim3(per_sm * di.sm_count), dim3(kBBlock),
                                           args, 0, s));
  return BFS_OK;
}

}  // namespace bfsint
