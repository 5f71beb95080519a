// Level-synchronous BFS as one persistent cooperative kernel per traversal.
//
// Each level k is one sparse matrix-sparse vector product over the
// (select2nd, max) semiring followed by the mask with the visited set, the
// parent update and the frontier replacement (Sec. 3.2, Algorithm 3 on one
// device).  A level is one phase of the kernel; phases are separated by a
// grid-wide barrier, and the loop's control (frontier size, variant choice,
// termination) lives on the device, so a whole traversal is a single launch.
//
// State of a phase k (all in HBM, the bitmaps stay resident in L2):
//   cur  = bits[k % 3]        frontier f_k as a bitmap (read only)
//   nxt  = bits[(k + 1) % 3]  f_{k+1} being built (claims by atomicOr / owner stores)
//   clr  = bits[(k + 2) % 3]  f_{k-1}, cleared during the phase for reuse as nxt
//   vis  = visited bitmap; during phase k it holds levels <= k-1 (and possibly k),
//          so "reached" is tested as (vis | cur)
//   queue[k % 3]              f_k as a list; queue[(k + 1) % 3] receives f_{k+1}
//   ctr[k % 8]                counters of f_k (size, degree sum, degree bins)
//
// Variants (identical results):
//   top-down (thread / warp / degree-binned): for u in f_k and every neighbour w
//     not yet reached, atomicMax(parent[w], u) -- every frontier neighbour of w
//     contributes, so parent[w] ends as the largest-id one -- and the first
//     atomicOr on nxt claims w (level, queue, counters).  Frontier entries are
//     dealt round-robin over the CTAs so that small frontiers use every SM, and
//     vertices above the chunk degree are split into grid-wide chunk items of
//     kChunkEdges edges, one CTA each.
//   pull: for every vertex v not yet reached, scan its sorted row from the
//     largest id down; the first neighbour in f_k is the max-id parent.  One
//     warp owns a chunk of 32 bitmap words (1,024 vertices) at a time, so nxt /
//     vis words are written by their owner lane without atomics; the chunk's
//     live rows are dealt to the lanes, two per lane.  Each lane first probes
//     the top entries of its rows; rows still open are then scanned by the
//     whole warp, 32 entries per step, packed across rows by a warp prefix sum
//     (per-row early exit is kept).  Vertices without edges are marked visited
//     at init, so pull levels never touch them.
#include <cooperative_groups.h>
#include <cooperative_groups/scan.h>

#include <algorithm>
#include <mutex>
#include <climits>
#include <cstdio>

#include "device_common.cuh"
#include "internal.h"
#include "claims.cuh"
#include "mlp_device.cuh"

namespace cg = cooperative_groups;

namespace bfsint {
namespace {

using bfsdev::kFull;

constexpr int kBlock = 512;
constexpr int kWarps = kBlock / 32;

#ifdef BFS_PHASE_TIMING
// Diagnostic build only: global-timer stamps of the first 4096 levels.
// [0] CTA 0 at level start, [1] after recycling, [2] after selection,
// [3] after expansion, [4] after counter flush, [5] latest barrier arrival
// of any CTA, [6] CTA 0 after the barrier.
__device__ unsigned long long g_phase_ts[4096][8];
#define PHASE_TS(k, slot)                                                             \
  do {                                                                                \
    if (blockIdx.x == 0 && threadIdx.x == 0 && (k) < 4096) g_phase_ts[k][slot] = bfsdev::global_timer_ns(); \
  } while (0)
#define PHASE_ARRIVAL(k)                                                              \
  do {                                                                                \
    __syncthreads();                                                                  \
    if (threadIdx.x == 0 && (k) < 4096) atomicMax(&g_phase_ts[k][5], (unsigned long long)bfsdev::global_timer_ns()); \
  } while (0)
#else
#define PHASE_TS(k, slot) \
  do {                    \
  } while (0)
#define PHASE_ARRIVAL(k) \
  do {                   \
  } while (0)
#endif

struct LoopParams {
  const int64_t* __restrict__ off;    // out-rows: top-down expansion
  const int32_t* __restrict__ adj;
  const int64_t* __restrict__ toff;   // in-rows: pull scans (the same arrays when undirected)
  const int32_t* __restrict__ tadj;
  int32_t directed;
  const uint32_t* __restrict__ dead;  // vertices no arc enters (and the tail), or null
  int32_t n;
  int32_t nwords;
  long long nnz;
  int32_t* level;
  int32_t* parent;
  int32_t* queue[3];
  uint32_t* bits[3];
  uint32_t* vis;
  int64_t* chunks[2];
  long long chunk_cap;  // entries of each chunk list
  LevelCtr* ctr;
  bfsdev::GridBarrier* bar;
  int* status;
  bfs_level_stat* stats;
  int32_t* misc;
  long long* edges_out;
  const int32_t* sources;  // device list when nsources > 1
  int32_t src0;            // the source when nsources == 1
  int32_t nsources;
  int32_t selector;
  int32_t forced;
  const int32_t* schedule;
  int32_t schedule_len;
  const float* mlp;
  float feat_log_n, feat_log_nnz, feat_inv_n, feat_inv_nnz;  // graph constants of the selector's features
  int32_t want_stats;
  unsigned spin_limit;
  int32_t warp_deg, cta_deg, pull_thread_deg, chunk_deg;
  float alpha, beta;
  long long small_frontier;  // TD_WARP for top-down levels up to this many vertices, all of degree <= 32
  long long narrow_edges;    // levels whose frontier has at most this many edges run on half the CTAs
  int32_t parts;
  const int64_t* part_base;
  int32_t** part_out;  // [2 * parts]: level outputs then parent outputs
  // 2D tiles of the in-adjacency for the tiled variant (t_jc null when absent)
  const uint16_t* __restrict__ t_jc;
  const uint32_t* __restrict__ t_cp;
  const uint16_t* __restrict__ t_ir;
  const int64_t* __restrict__ t_dir_jc;
  const int64_t* __restrict__ t_dir_ir;
  int32_t t_rb_bits, t_cb_bits, t_nrb, t_ncb;
  int32_t tile_smem_off;  // byte offset of the tiled phase's slices in dynamic shared memory
};

// Per-thread accumulation of the next frontier's counters.
struct Acc {
  unsigned long long edges = 0, b0 = 0, b1 = 0, b2 = 0;
};

__device__ __forceinline__ void acc_vertex(Acc& a, long long deg) {
  a.edges += (unsigned long long)deg;
  if (deg <= 32) a.b0 += 1;
  else if (deg <= 1024) a.b1 += 1;
  else a.b2 += 1;
}

// Bookkeeping of a vertex claimed for level knext (the caller already set nxt).
__device__ __forceinline__ void claim_topdown(const LoopParams& p, int knext, int w, long long deg, Acc& acc,
                                              Claims& cl) {
  p.level[w] = knext;
  cta_enqueue(p, knext, cl, w);
  acc_vertex(acc, deg);
  if (deg > p.chunk_deg) push_chunks_cta(p, knext, cl, w, deg);
}

// Top-down visit of edge (u -> w) in phase k.
__device__ __forceinline__ void td_visit(const LoopParams& p, const uint32_t* cur, uint32_t* nxt, int k,
                                         int u, int w, Acc& acc, Claims& cl) {
  if (!bfsdev::in_range(p.status, bfsdev::kSiteTopDown, w, p.n)) return;
  const int ww = w >> 5;
  const uint32_t m = 1u << (w & 31);
  const uint32_t vw = p.vis[ww], cw = cur[ww], nw = nxt[ww];  // independent loads, one round trip
  if ((vw | cw) & m) return;
  atomicMax(&p.parent[w], u);
  if (nw & m) return;
  const long long wb = __ldg(&p.off[w]), we = __ldg(&p.off[w + 1]);  // speculative: the claim needs the degree
  const uint32_t old = atomicOr(&nxt[ww], m);
  if (old & m) return;
  claim_topdown(p, k + 1, w, we - wb, acc, cl);
}

// Warp-cooperative descending scan of the rows still open in a warp: lane r
// owns row r with entries [b, t) not yet examined (t exclusive, scanned from
// t-1 down).  Every step the open rows' next entries (at most kCoopRow per
// row) are packed into kCoopSteps x 32 slots by a prefix sum; slot g is
// examined by lane g % 32 in sub-step g / 32, so every lane has kCoopSteps
// adjacency loads and bitmap loads in flight.  A row whose slots hold a hit
// takes the hit in its lowest slot (its highest position, i.e. its largest
// id) and closes.  All lanes call it; returns the row's hit or -1.  status and
// n serve the bounds-checking build's check of every id the scan loads.
#ifndef BFS_COOP_STEPS
#define BFS_COOP_STEPS 1
#endif
constexpr int kCoopSteps = BFS_COOP_STEPS;
constexpr int kCoopRow = 32 * kCoopSteps;

__device__ __forceinline__ int scan_desc_coop(const int32_t* __restrict__ adj, const uint32_t* bm, long long b,
                                              long long t, bool open, int hit, int lane, int* status, int n) {
  unsigned pm = __ballot_sync(kFull, open);
  while (pm) {
    const int rc = open ? (int)min(t - b, (long long)kCoopRow) : 0;
    int incl = rc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    const int excl = incl - rc;
    const int total = __shfl_sync(kFull, incl, 31);
    int u[kCoopSteps];
    bool h[kCoopSteps];
#pragma unroll
    for (int sstep = 0; sstep < kCoopSteps; ++sstep) {
      const int slot = sstep * 32 + lane;
      // owner row of this slot: the last row whose prefix is <= slot
      int r = 0;
#pragma unroll
      for (int st = 16; st >= 1; st >>= 1) {
        const int c = r + st;
        const int ec = __shfl_sync(kFull, excl, c & 31);
        if (c < 32 && ec <= slot) r = c;
      }
      const long long tr = __shfl_sync(kFull, t, r);
      const int er = __shfl_sync(kFull, excl, r);
      u[sstep] = slot < total ? __ldg(&adj[tr - 1 - (slot - er)]) : -1;
    }
#pragma unroll
    for (int sstep = 0; sstep < kCoopSteps; ++sstep) {
      const bool live = bfsdev::kBoundsCheck
                            ? sstep * 32 + lane < total && bfsdev::in_range(status, bfsdev::kSitePull, u[sstep], n)
                            : u[sstep] >= 0;
      h[sstep] = live && ((bm[u[sstep] >> 5] >> (u[sstep] & 31)) & 1u);
    }
    // this lane's row takes slots [excl, excl + cons) of the kCoopRow slots
    const int cons = max(0, min(rc, kCoopRow - excl));
    int found = -1;
#pragma unroll
    for (int sstep = 0; sstep < kCoopSteps; ++sstep) {
      const unsigned hm = __ballot_sync(kFull, h[sstep]);
      const int lo = max(excl - sstep * 32, 0), hi = min(excl + cons - sstep * 32, 32);
      unsigned seg = 0u;
      if (hi > lo) seg = (hi - lo == 32 ? kFull : ((1u << (hi - lo)) - 1u)) << lo;
      const unsigned mine = hm & seg;
      const int hv = __shfl_sync(kFull, u[sstep], mine ? __ffs(mine) - 1 : 0);
      if (found < 0 && mine) found = hv;
    }
    if (open) {
      if (found >= 0) {
        hit = found;
        open = false;
      } else {
        t -= cons;
        if (t <= b) open = false;
      }
    }
    pm = __ballot_sync(kFull, open);
  }
  return hit;
}

// 64-bit warp sum.
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// End of a phase for one CTA: adds its counters into level knext's slot and
// moves its buffered next-frontier vertices to the global queue with a single
// atomic.  CTAs that claimed nothing skip all of it.
// End of a phase: the CTA's counter contributions, its buffered queue entries
// and its buffered chunk items go to level knext with one atomic each.
template <typename S>
__device__ __forceinline__ void end_phase(const LoopParams& p, int knext, Acc& acc, S& sm) {
  const bool mine = (acc.edges | acc.b0 | acc.b1 | acc.b2) != 0;
  if (__syncthreads_or(mine)) {
    const unsigned long long e = warp_sum_u64(acc.edges), b0 = warp_sum_u64(acc.b0), b1 = warp_sum_u64(acc.b1),
                             b2 = warp_sum_u64(acc.b2);
    if ((threadIdx.x & 31) == 0 && (e | b0 | b1 | b2)) {
      atomicAdd(&sm.acc[0], e);
      atomicAdd(&sm.acc[1], b0);
      atomicAdd(&sm.acc[2], b1);
      atomicAdd(&sm.acc[3], b2);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      LevelCtr* c = &p.ctr[knext % kCtrRing];
      if (sm.acc[0]) atomicAdd(&c->edges, sm.acc[0]);
      if (sm.acc[1]) atomicAdd(&c->bins[0], sm.acc[1]);
      if (sm.acc[2]) atomicAdd(&c->bins[1], sm.acc[2]);
      if (sm.acc[3]) atomicAdd(&c->bins[2], sm.acc[3]);
      sm.acc[0] = sm.acc[1] = sm.acc[2] = sm.acc[3] = 0;
    }
  }
  flush_claims(p, knext, sm.cl);
  acc = Acc{};
}

struct Smem {
  int owner;
  int cu;
  long long cb, ce;
  int warp_tmp[kWarps + 1];
  unsigned long long acc[4];
  int tu[kBlock];
  long long tb[kBlock];
  int tpref[kBlock + 1];
  Claims cl;
  uint32_t pull_hits[kWarps][32];  // pull: hit bits of each warp's 32 bitmap words
  __align__(16) float h1[64];  // selector network: hidden layer 1, choice
  int choice;
  unsigned long long next_item;  // top-down: the next chunk item of this CTA
};

// ---------------- top-down phase ----------------
__device__ void topdown_phase(const LoopParams& p, int k, int variant, unsigned count, unsigned nchunks, Smem& sm,
                              Acc& acc, unsigned G) {
  const uint32_t* cur = p.bits[k % 3];
  uint32_t* nxt = p.bits[(k + 1) % 3];
  const int32_t* Q = p.queue[k % 3];
  const int tid = threadIdx.x, lane = tid & 31;

  // chunk items of high-degree frontier vertices: one CTA per item; before each
  // item the CTA makes room in its buffers for the item's claims
  const int64_t* items = p.chunks[k & 1];
  for (unsigned ci = blockIdx.x; ci < nchunks; ci += G) {
    flush_claims_if_full(p, k + 1, sm.cl, kChunkEdges, kBigBuf / 2);
    const int64_t it = items[ci];
    const int v = (int)(it >> 32);
    const long long c = it & 0xffffffffll;
    const long long rb = __ldg(&p.off[v]), re = __ldg(&p.off[v + 1]);
    const long long b = rb + c * kChunkEdges;
    const long long e = min(b + (long long)kChunkEdges, re);
    for (long long j = b + tid; j < e; j += kBlock) td_visit(p, cur, nxt, k, v, __ldg(&p.adj[j]), acc, sm.cl);
  }

  // frontier entry i goes to CTA i % G, so that small frontiers spread over the SMs
  const long long gthreads = (long long)G * kBlock;
  if (variant == BFS_VARIANT_TD_THREAD) {
    for (long long i = blockIdx.x + (long long)tid * G; i < count; i += gthreads) {
      const int u = Q[i];
      atomicOr(&p.vis[u >> 5], 1u << (u & 31));
      const long long b = __ldg(&p.off[u]), e = __ldg(&p.off[u + 1]);
      if (e - b > p.chunk_deg) continue;
      for (long long j = b; j < e; ++j) td_visit(p, cur, nxt, k, u, __ldg(&p.adj[j]), acc, sm.cl);
    }
  } else if (variant == BFS_VARIANT_TD_WARP) {
    const long long gwarps = gthreads / 32;
    for (long long i = blockIdx.x + (long long)(tid >> 5) * G; i < count; i += gwarps) {
      const int u = Q[i];
      if (lane == 0) atomicOr(&p.vis[u >> 5], 1u << (u & 31));
      const long long b = __ldg(&p.off[u]), e = __ldg(&p.off[u + 1]);
      if (e - b > p.chunk_deg) continue;
      for (long long j = b + lane; j < e; j += 32) td_visit(p, cur, nxt, k, u, __ldg(&p.adj[j]), acc, sm.cl);
    }
  } else {  // BFS_VARIANT_TD_BINNED
    for (long long tile = 0; tile < count; tile += gthreads) {
      flush_claims_if_full(p, k + 1, sm.cl, kQBuf / 2, kBigBuf / 2);
      const long long i = tile + blockIdx.x + (long long)tid * G;
      int u = -1;
      long long b = 0, e = 0;
      if (i < count) {
        u = Q[i];
        atomicOr(&p.vis[u >> 5], 1u << (u & 31));
        b = __ldg(&p.off[u]);
        e = __ldg(&p.off[u + 1]);
        if (e - b > p.chunk_deg) u = -1;
      }
      const long long deg = u >= 0 ? e - b : 0;
      // CTA bin: the whole CTA walks one row at a time
      for (;;) {
        if (u >= 0 && deg >= p.cta_deg) sm.owner = tid;
        __syncthreads();
        const int owner = sm.owner;
        if (owner < 0) break;
        if (tid == owner) {
          sm.cu = u;
          sm.cb = b;
          sm.ce = e;
          u = -1;
        }
        __syncthreads();
        const int cu = sm.cu;
        const long long cb = sm.cb, ce = sm.ce;
        for (long long j = cb + tid; j < ce; j += kBlock) td_visit(p, cur, nxt, k, cu, __ldg(&p.adj[j]), acc, sm.cl);
        __syncthreads();
        if (tid == 0) sm.owner = -1;
        __syncthreads();
      }
      // warp bin: a warp walks one row at a time
      for (;;) {
        const unsigned wm = __ballot_sync(kFull, u >= 0 && deg >= p.warp_deg);
        if (!wm) break;
        const int l = __ffs(wm) - 1;
        const int cu = __shfl_sync(kFull, u, l);
        const long long cb = __shfl_sync(kFull, b, l), ce = __shfl_sync(kFull, e, l);
        if (lane == l) u = -1;
        for (long long j = cb + lane; j < ce; j += 32) td_visit(p, cur, nxt, k, cu, __ldg(&p.adj[j]), acc, sm.cl);
      }
      // thread bin: the CTA gathers the remaining short rows edge by edge
      const int sdeg = u >= 0 ? (int)deg : 0;
      int excl = 0;
      const int total = block_exclusive_scan(sdeg, sm.warp_tmp, excl);
      sm.tu[tid] = u;
      sm.tb[tid] = b;
      sm.tpref[tid] = excl;
      if (tid == 0) sm.tpref[kBlock] = total;
      __syncthreads();
      for (int base = 0; base < total; base += kBlock) {
        const int idx = base + tid;
        if (idx < total) {
          int lo = 0, hi = kBlock;  // largest slot with tpref <= idx (and a non-empty row)
          while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (sm.tpref[mid] <= idx) lo = mid;
            else hi = mid;
          }
          const int ou = sm.tu[lo];
          td_visit(p, cur, nxt, k, ou, __ldg(&p.adj[sm.tb[lo] + (idx - sm.tpref[lo])]), acc, sm.cl);
        }
      }
      __syncthreads();
    }
  }
}

// ---------------- pull phase ----------------
constexpr int kPullRows = 2;    // live rows per lane in flight
constexpr int kPullProbes = 4;  // at most this many top entries of each row are probed before the warp scan
// Position of the r-th (0-based) set bit of m; r < popc(m).
__device__ __forceinline__ int select_bit(uint32_t m, int r) {
  int pos = 0;
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const int c = __popc(m & ((1u << s) - 1u));  // set bits in the low s bits
    if (r >= c) {
      r -= c;
      m >>= s;
      pos += s;
    }
  }
  return pos;
}

// The idx-th live vertex of a warp's chunk of 32 bitmap words (all lanes call
// it; lane l holds word l's live bits `live` and the inclusive prefix `incl` of
// their counts).  Returns the vertex, the owner lane of its word and its bit.
__device__ __forceinline__ int live_vertex(long long chunk, uint32_t live, int incl, int idx, int& owner,
                                           uint32_t& bit) {
  int o = 0;  // number of lanes whose inclusive prefix is <= idx: the owner
#pragma unroll
  for (int st = 16; st >= 1; st >>= 1) {
    const int c = __shfl_sync(kFull, incl, o + st - 1);
    if (c <= idx) o += st;
  }
  o = min(o, 31);
  const uint32_t lo = __shfl_sync(kFull, live, o);
  const int excl_o = __shfl_sync(kFull, incl, o) - __popc(lo);
  const int b = select_bit(lo, max(idx - excl_o, 0));
  owner = o;
  bit = 1u << b;
  return (int)((chunk * 32 + o) * 32 + b);
}

// The max-id frontier neighbour of R rows per lane (v[r] < 0: no row): the
// rows' bounds, then a probe of the top `probe` (<= P) entries of every row with all their
// adjacency loads and then all their frontier-word loads in flight together,
// then the warp's cooperative descending scan of the rows still open.  R = 2,
// P = 4 is what the 64-register budget holds without spills (R = 3 or 4 with
// P = 2 spilled and ran 5 % and 16 % slower on R-MAT scale 26).
template <int R, int P>
__device__ __forceinline__ void pull_rows(const LoopParams& p, const uint32_t* cur, int lane, int probe,
                                          const int (&v)[R], int (&h)[R], long long (&d)[R]) {
  long long b[R], e[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    b[r] = e[r] = 0;
    if (v[r] >= 0) {
      b[r] = __ldg(&p.toff[v[r]]);
      e[r] = __ldg(&p.toff[v[r] + 1]);
    }
  }
  int np[R];
  int u[R][P];
  uint32_t x[R][P];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    np[r] = v[r] >= 0 ? (int)min((long long)probe, e[r] - b[r]) : 0;
#pragma unroll
    for (int q = 0; q < P; ++q) u[r][q] = q < np[r] ? __ldg(&p.tadj[e[r] - 1 - q]) : 0;
  }
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int q = 0; q < P; ++q)
      x[r][q] = q < np[r] && bfsdev::in_range(p.status, bfsdev::kSitePull, u[r][q], p.n) ? cur[u[r][q] >> 5] : 0u;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    h[r] = -1;
#pragma unroll
    for (int q = 0; q < P; ++q)
      if (q < np[r] && h[r] < 0 && ((x[r][q] >> (u[r][q] & 31)) & 1u)) h[r] = u[r][q];
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const long long t = e[r] - np[r];
    h[r] = scan_desc_coop(p.tadj, cur, b[r], t, v[r] >= 0 && h[r] < 0 && t > b[r], h[r], lane, p.status, p.n);
    d[r] = e[r] - b[r];
  }
}

// Bookkeeping of a vertex v reached by the pull (hit = its parent): outputs,
// counters, chunk items, the owner word's hit bit and the warp's queue buffer.
__device__ __forceinline__ void pull_claim(const LoopParams& p, int knext, int v, int hit, long long deg_in,
                                           uint32_t* hitw, int owner, uint32_t bit, Acc& acc, Claims& cl, int* wq,
                                           int& nbuf, int lane) {
  if (hit >= 0) {
    p.parent[v] = hit;
    p.level[v] = knext;
    atomicOr(&hitw[owner], bit);
    // out-degree: the next level expands v's out-row (the row scanned here when undirected)
    const long long deg = p.directed ? __ldg(&p.off[v + 1]) - __ldg(&p.off[v]) : deg_in;
    acc_vertex(acc, deg);
    if (deg > p.chunk_deg) push_chunks_cta(p, knext, cl, v, deg);
  }
  warp_enqueue(p, knext, wq, nbuf, hit >= 0, v, lane, false);
}

// Dense-frontier SpMV over the unvisited rows.  A warp takes a chunk of 32
// bitmap words (1,024 vertices) at a time: lane l loads word l of `vis` and of
// `cur`, and the chunk's live vertices (not reached, not edgeless) are dealt to
// the lanes 64 at a time, two rows per lane, so that every lane carries an open
// row however sparse the live vertices are (in the last pull levels of a
// scale-26 R-MAT graph most words hold one live vertex).  Each word's hits are
// gathered in shared memory and its owner lane writes the word's `nxt` and
// `vis` (no global atomics on the bitmaps).  Rows without a frontier
// neighbour near their top make some chunks far dearer than others, so the
// second half of a large level's chunks is handed out dynamically: with an
// all-static deal the level waited on its slowest warps (R-MAT scale 26: 126.4
// ms for the 64 bench roots, 121.8 with the dynamic tail), and with an
// all-dynamic one the cursor's atomics, all at once at the start of every
// level, made the 2^27-edge edgefactor-16 and -64 graphs 11 % and 15 % slower.
__device__ void pull_phase(const LoopParams& p, int k, Smem& sm, Acc& acc, unsigned G) {
  const uint32_t* cur = p.bits[k % 3];
  uint32_t* nxt = p.bits[(k + 1) % 3];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long gwarps = (long long)G * kWarps;
  const int knext = k + 1;
  const int probe = min(p.pull_thread_deg, kPullProbes);  // the tuning knob, at most kPullProbes
  int* wq = sm.cl.wq[wid];
  uint32_t* hitw = sm.pull_hits[wid];
  int nbuf = 0;
  // chunk indices fit 32 bits: nwords < 2^26
  const int nchunks = (p.nwords + 31) / 32, gw = (int)gwarps;
  // Chunks [0, S) are dealt statically (warp i takes i, i + gw, ...), the
  // rest from the level's cursor, each fetch issued one chunk ahead.  With
  // fewer than two chunks per warp the level is all static (S past every chunk).
  const int S = nchunks > 2 * gw ? gw * max(1, (nchunks / 2) / gw) : INT_MAX;
  for (int c = wid * (int)G + (int)blockIdx.x; c < nchunks;) {
    unsigned taken = 0;
    if (c + gw >= S && lane == 0) taken = (unsigned)atomicAdd(&p.ctr[k % kCtrRing].pad, 1ull);  // used after the chunk
    const int w = c * 32 + lane;
    const bool has = w < p.nwords;
    const uint32_t vw = has ? p.vis[w] : 0xffffffffu;
    const uint32_t cw = has ? cur[w] : 0u;
    const uint32_t visw = vw | cw;
    const uint32_t live = ~visw;
    const int cnt = __popc(live);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(kFull, incl, 31);
    hitw[lane] = 0u;
    __syncwarp();
    for (int base = 0; base < total; base += 32 * kPullRows) {
      int v[kPullRows], o[kPullRows], h[kPullRows];
      uint32_t bit[kPullRows];
      long long d[kPullRows];
#pragma unroll
      for (int r = 0; r < kPullRows; ++r) {
        const int i = base + r * 32 + lane;
        const int lv = live_vertex(c, live, incl, min(i, total - 1), o[r], bit[r]);
        v[r] = i < total ? lv : -1;
      }
      pull_rows<kPullRows, kPullProbes>(p, cur, lane, probe, v, h, d);
#pragma unroll
      for (int r = 0; r < kPullRows; ++r)
        pull_claim(p, knext, v[r], v[r] >= 0 ? h[r] : -1, d[r], hitw, o[r], bit[r], acc, sm.cl, wq, nbuf, lane);
    }
    __syncwarp();
    const uint32_t hits = hitw[lane];
    if (has) {
      if (hits) nxt[w] = hits;
      if ((visw | hits) != vw) p.vis[w] = visw | hits;
    }
    __syncwarp();
    c = c + gw >= S ? S + (int)__shfl_sync(kFull, taken, 0) : c + gw;
  }
  warp_enqueue(p, knext, wq, nbuf, false, 0, lane, true);
}

// ---------------- tiled phase ----------------
// Dense-frontier SpMV over the 2D tiles of the in-adjacency (Sec. 3.2's 2D
// blocks, each in the DCSC form of Sec. 4.1).  A CTA owns a row block at a
// time and keeps two tile-local slices in shared memory: `done`, the row
// block's reached rows (vis | cur at level start, plus the rows found in the
// tiles already walked), and `slice`, the frontier bits of the current column
// block.  It walks the row block's tiles from the highest column block down;
// in each tile the non-empty columns that are in the frontier expand their
// rows (flattened over the CTA by a prefix sum, like the thread bin of the
// top-down phase), and every row not yet done takes the column as a parent
// candidate with atomicMax.  A row's candidates all come from the first tile
// (in that order) that holds a frontier neighbour, since `done` only changes
// between tiles, so the largest candidate is its max-id parent.  The row
// block's found rows then go out as in the pull: owner-written nxt / vis
// words, levels, counters and the warp queue buffers.
constexpr int kTileWordsMax = 2048;  // 2^16 rows or columns per tile

__device__ void tiled_phase(const LoopParams& p, int k, Smem& sm, uint32_t* tsm, Acc& acc, unsigned G) {
  const uint32_t* cur = p.bits[k % 3];
  uint32_t* nxt = p.bits[(k + 1) % 3];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int knext = k + 1;
  uint32_t* done = tsm;
  uint32_t* newf = tsm + kTileWordsMax;
  uint32_t* slice = tsm + 2 * kTileWordsMax;
  const int rbw = 1 << (p.t_rb_bits - 5), cbw = 1 << (p.t_cb_bits - 5);
  int* wq = sm.cl.wq[wid];
  int nbuf = 0;
  for (int rb = blockIdx.x; rb < p.t_nrb; rb += G) {
    const long long w0 = (long long)rb * rbw;
    bool live = false;
    for (int i = tid; i < rbw; i += kBlock) {
      const long long w = w0 + i;
      const uint32_t d = w < p.nwords ? (p.vis[w] | cur[w]) : 0xffffffffu;
      done[i] = d;
      newf[i] = 0u;
      live |= d != 0xffffffffu;
    }
    // a block whose rows are all reached walks no tile, but still folds cur into vis below
    const int first_cb = __syncthreads_or(live) ? p.t_ncb - 1 : -1;
    for (int cb = first_cb; cb >= 0; --cb) {
      const long long t = (long long)rb * p.t_ncb + cb;
      const long long j0 = p.t_dir_jc[t], j1 = p.t_dir_jc[t + 1];
      if (j0 == j1) continue;  // empty tile (the same on every thread)
      const long long ibase = p.t_dir_ir[t], iend = p.t_dir_ir[t + 1];
      const long long s0 = (long long)cb * cbw;
      for (int i = tid; i < cbw; i += kBlock) slice[i] = s0 + i < p.nwords ? cur[s0 + i] : 0u;
      __syncthreads();
      bool tile_hit = false;
      for (long long jb = j0; jb < j1; jb += kBlock) {
        const long long j = jb + tid;
        int ul = -1;
        long long rbeg = 0, rlen = 0;
        if (j < j1) {
          const int c = p.t_jc[j];
          if ((slice[c >> 5] >> (c & 31)) & 1u) {
            ul = c;
            rbeg = ibase + p.t_cp[j];
            rlen = (j + 1 < j1 ? ibase + p.t_cp[j + 1] : iend) - rbeg;
          }
        }
        int excl = 0;
        const int total = block_exclusive_scan((int)rlen, sm.warp_tmp, excl);
        sm.tu[tid] = ul;
        sm.tb[tid] = rbeg;
        sm.tpref[tid] = excl;
        if (tid == 0) sm.tpref[kBlock] = total;
        __syncthreads();
        for (int base = 0; base < total; base += kBlock) {
          const int idx = base + tid;
          if (idx < total) {
            int lo = 0, hi = kBlock;  // largest slot with tpref <= idx (a frontier column with rows)
            while (hi - lo > 1) {
              const int mid = (lo + hi) >> 1;
              if (sm.tpref[mid] <= idx) lo = mid;
              else hi = mid;
            }
            const int r = p.t_ir[sm.tb[lo] + (idx - sm.tpref[lo])];
            if (!((done[r >> 5] >> (r & 31)) & 1u)) {
              atomicMax(&p.parent[(rb << p.t_rb_bits) + r], (cb << p.t_cb_bits) + sm.tu[lo]);
              atomicOr(&newf[r >> 5], 1u << (r & 31));
              tile_hit = true;
            }
          }
        }
        __syncthreads();
      }
      // the tile's rows are done from here on; stop once every row of the block is
      if (__syncthreads_or(tile_hit)) {
        live = false;
        for (int i = tid; i < rbw; i += kBlock) {
          const uint32_t d = done[i] | newf[i];
          done[i] = d;
          newf[i] = 0u;
          live |= d != 0xffffffffu;
        }
        if (!__syncthreads_or(live)) break;
      }
    }
    // rows found in this row block: done now minus reached at level start; every
    // word of the block gets vis |= cur | found, as in the pull phase, so that
    // f_k stays reached after its bitmap is recycled
    for (int i = wid; i < rbw; i += kWarps) {
      const long long w = w0 + i;
      if (w >= p.nwords) break;
      const uint32_t vw = p.vis[w], cw = cur[w];
      const uint32_t visw = vw | cw;
      const uint32_t f = done[i] & ~visw;
      if (lane == 0) {
        if (f) nxt[w] = f;
        if ((visw | f) != vw) p.vis[w] = visw | f;
      }
      const bool hit = (f >> lane) & 1u;
      const int v = (int)(w * 32 + lane);
      if (hit) {
        p.level[v] = knext;
        const long long deg = __ldg(&p.off[v + 1]) - __ldg(&p.off[v]);
        acc_vertex(acc, deg);
        if (deg > p.chunk_deg) push_chunks_cta(p, knext, sm.cl, v, deg);
      }
      warp_enqueue(p, knext, wq, nbuf, hit, v, lane, false);
    }
    __syncthreads();
  }
  warp_enqueue(p, knext, wq, nbuf, false, 0, lane, true);
}

// The selector network on one warp: every lane computes the 12 level features
// in registers (lane j < 3 brings bin count j), then the warp evaluates the
// network on the parameters in the warp layout; returns the chosen variant on
// every lane.  Kept out of line so that its registers do not crowd the phases.
__device__ __noinline__ int learned_choice(const LoopParams& p, const float* w, float* h1, int lane, int k,
                                           long long count, long long edges, long long unvisited,
                                           long long unvisited_edges, long long binv) {
  float x[12];
  bfsdev::level_features(p.feat_log_n, p.feat_log_nnz, p.feat_inv_n, p.feat_inv_nnz, k, count, edges, unvisited,
                         unvisited_edges, __shfl_sync(kFull, binv, 0), __shfl_sync(kFull, binv, 1),
                         __shfl_sync(kFull, binv, 2), x);
  return bfsdev::warp_mlp_argmin(w, x, h1, lane);
}

// Direction choice in the manner of direction-optimising BFS: go pull when the
// frontier's edges exceed the unvisited edges / alpha while the frontier is
// growing, leave pull when the frontier falls below n / beta.  (p.alpha is the
// tuned alpha scaled by 1 + 4 n / L2 bytes at launch.)
__device__ __forceinline__ int heuristic_variant(const LoopParams& p, int prev_variant, long long count,
                                                 long long prev_count, long long edges,
                                                 long long unvisited_edges, bool small_rows) {
  bool pull;
  if (prev_variant == BFS_VARIANT_PULL) pull = (float)count * p.beta >= (float)p.n;
  else pull = (float)edges * p.alpha > (float)unvisited_edges && count >= prev_count;
  if (pull) return BFS_VARIANT_PULL;
  // a small frontier of short rows: one warp per vertex beats the binning's scan
  return (count <= p.small_frontier && small_rows) ? BFS_VARIANT_TD_WARP : BFS_VARIANT_TD_BINNED;
}

// kTiles: the kernel can run the tiled phase.  Runs that cannot pick the tiled
// variant launch the instance without it: on R-MAT scale 26 the tiled phase's
// code alone made the other phases 5 % slower.
template <bool kTiles>
__global__ void __launch_bounds__(kBlock, 2) level_loop_kernel(LoopParams p) {
  __shared__ Smem sm;
  // dynamic shared memory: the selector network's parameters (BFS_MLP_PARAMS
  // floats) when the learned selector is on, then the tiled phase's slices
  // (3 * kTileWordsMax words) when tiles are present
  extern __shared__ __align__(16) unsigned char s_dyn[];
  float* s_mlp = reinterpret_cast<float*>(s_dyn);
  uint32_t* s_tile = reinterpret_cast<uint32_t*>(s_dyn + p.tile_smem_off);
  const int tid = threadIdx.x;
  unsigned long long bar_target = 0;
  if (tid == 0) {
    bar_target = bfsdev::barrier_base(p.bar, gridDim.x);
    sm.owner = -1;
    claims_reset(sm.cl);
    sm.acc[0] = sm.acc[1] = sm.acc[2] = sm.acc[3] = 0;
  }
  const bool learned = p.selector == BFS_SELECT_LEARNED && p.mlp != nullptr;
  if (learned)
    for (int i = tid; i < BFS_MLP_PARAMS; i += kBlock) s_mlp[bfsdev::warp_layout_index(i)] = p.mlp[i];

  const long long gtid = (long long)blockIdx.x * kBlock + tid;
  const long long gthreads = (long long)gridDim.x * kBlock;
  const unsigned nblocks = gridDim.x;

  // ---- init: outputs to -1, bitmaps cleared, counters zeroed.  Vertices
  // without edges (and the tail beyond n) start as visited, since no traversal
  // can reach them.  A single source is seeded in the same phase; several
  // sources (ragged runs) get a seeding phase of their own.  The output fill
  // only stores and the bitmap loop's loads are independent, so neither waits
  // on a load per step.
  const bool single = p.nsources == 1;
  const int s0 = p.src0;
  // outputs: 4 vertices per thread and step, one 16-byte store each when aligned
  const bool vec = ((reinterpret_cast<uintptr_t>(p.level) | reinterpret_cast<uintptr_t>(p.parent)) & 15u) == 0;
  const long long n4 = ((long long)p.n + 3) / 4;
  for (long long q = gtid; q < n4; q += gthreads) {
    const long long v = 4 * q;
    int lv[4], pv[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const bool src = single && v + c == s0;
      lv[c] = src ? 0 : -1;
      pv[c] = src ? s0 : -1;
    }
    if (vec && v + 4 <= p.n) {
      *reinterpret_cast<int4*>(p.level + v) = make_int4(lv[0], lv[1], lv[2], lv[3]);
      *reinterpret_cast<int4*>(p.parent + v) = make_int4(pv[0], pv[1], pv[2], pv[3]);
    } else {
      for (int c = 0; c < 4 && v + c < p.n; ++c) {
        p.level[v + c] = lv[c];
        p.parent[v + c] = pv[c];
      }
    }
  }
  // bitmaps: vis starts as the edgeless vertices (and the tail beyond n) plus
  // the single source; one thread per word when the dead bits are precomputed
  const uint32_t srcbit = 1u << (s0 & 31);
  const long long sw = s0 >> 5;
  if (p.dead != nullptr) {
    for (long long w = gtid; w < p.nwords; w += gthreads) {
      const bool sword = single && w == sw;
      p.vis[w] = __ldg(&p.dead[w]) | (sword ? srcbit : 0u);
      p.bits[0][w] = sword ? srcbit : 0u;
      p.bits[1][w] = 0;
      p.bits[2][w] = 0;
    }
  } else {  // dead bits from the row offsets, one warp per word
    const long long nv32 = (long long)p.nwords * 32;
    for (long long v = gtid; v < nv32; v += gthreads) {
      const bool dead = v >= p.n || (single && v == s0) || __ldg(&p.toff[v + 1]) == __ldg(&p.toff[v]);
      const unsigned dm = __ballot_sync(kFull, dead);
      if ((tid & 31) == 0) {
        const long long w = v >> 5;
        const bool sword = single && w == sw;
        p.vis[w] = dm;
        p.bits[0][w] = sword ? srcbit : 0u;
        p.bits[1][w] = 0;
        p.bits[2][w] = 0;
      }
    }
  }
  if (blockIdx.x == 0) {
    if (tid < kCtrRing * (int)(sizeof(LevelCtr) / 8)) reinterpret_cast<unsigned long long*>(p.ctr)[tid] = 0ull;
    __syncthreads();
    if (single && tid == 0) {
      p.queue[0][0] = s0;
      const long long deg = __ldg(&p.off[s0 + 1]) - __ldg(&p.off[s0]);
      p.ctr[0].count = 1;
      p.ctr[0].edges = (unsigned long long)deg;
      p.ctr[0].bins[deg <= 32 ? 0 : (deg <= 1024 ? 1 : 2)] = 1;
      if (deg > p.chunk_deg) push_chunks(p, 0, s0, deg);
    }
  }
  if (!bfsdev::grid_barrier(p.bar, nblocks, bar_target, p.spin_limit, p.status)) return;

  if (!single) {  // seed level 0 with the sources (block 0)
    if (blockIdx.x == 0) {
      Acc acc;
      for (int i = tid; i < p.nsources; i += kBlock) {
        const int s = p.sources[i];
        p.level[s] = 0;
        p.parent[s] = s;
        atomicOr(&p.bits[0][s >> 5], 1u << (s & 31));
        p.queue[0][i] = s;
        const long long deg = __ldg(&p.off[s + 1]) - __ldg(&p.off[s]);
        acc_vertex(acc, deg);
        if (deg > p.chunk_deg) push_chunks(p, 0, s, deg);
      }
      if (tid == 0) p.ctr[0].count = (unsigned)p.nsources;
      end_phase(p, 0, acc, sm);
    }
    if (!bfsdev::grid_barrier(p.bar, nblocks, bar_target, p.spin_limit, p.status)) return;
  }

  // ---- level loop
  long long cum_count = 0, cum_edges = 0;
  int prev_variant = -1;
  unsigned prev_count = 0;
  uint64_t t_prev = 0;
  if (blockIdx.x == 0 && tid == 0) t_prev = bfsdev::global_timer_ns();
  int k = 0;
  Acc acc;
  for (;; ++k) {
    PHASE_TS(k, 0);
    // one round of loads: the counters of f_k and the first entry of f_{k-1} to recycle
    const LevelCtr* c = &p.ctr[k % kCtrRing];
    const unsigned count = __ldcg(&c->count);
    const unsigned nchunks = __ldcg(&c->chunks);
    const long long edges = (long long)__ldcg(&c->edges);
    const long long binv = (learned && tid < 3) ? (long long)__ldcg(&c->bins[tid]) : 0;
    const unsigned long long big_rows = __ldcg(&c->bins[1]) | __ldcg(&c->bins[2]);
    const bool sparse_clr = k >= 1 && (long long)prev_count * 4 < p.nwords;
    const int32_t* PQ = p.queue[(k + 2) % 3];
    const int clr0 = (sparse_clr && gtid < prev_count) ? PQ[gtid] : -1;
    if (count == 0) break;
    cum_count += count;
    cum_edges += edges;
    const long long unvisited = (long long)p.n - cum_count;
    const long long unvisited_edges = p.nnz - cum_edges;

    // A level whose frontier has few edges runs on the first half of the CTAs
    // (one per SM when two are resident): only they recycle, expand and arrive
    // at its barrier, which halves the barrier's arrivals and the CTAs that
    // contend for the level's few claims.  The other CTAs still choose the
    // variant (the next level's choice depends on it) and wait at the barrier.
    const unsigned G = (edges <= p.narrow_edges && nblocks >= 2) ? (nblocks + 1) / 2 : nblocks;
    const bool part = blockIdx.x < G;
    const long long pthreads = (long long)G * kBlock;

    // recycle: counters of level k+4, bitmap of level k-1 (stores only; they
    // drain while the selector runs)
    if (blockIdx.x == 0 && tid < (int)(sizeof(LevelCtr) / 8))
      reinterpret_cast<unsigned long long*>(&p.ctr[(k + 4) % kCtrRing])[tid] = 0ull;
    if (k >= 1 && part) {
      uint32_t* clr = p.bits[(k + 2) % 3];
      if (sparse_clr) {
        if (clr0 >= 0) clr[clr0 >> 5] = 0u;
        for (long long i = gtid + pthreads; i < prev_count; i += pthreads) clr[PQ[i] >> 5] = 0u;
      } else {
        for (long long w = gtid; w < p.nwords; w += pthreads) clr[w] = 0u;
      }
    }
    PHASE_TS(k, 1);

    int variant;
    if (p.selector == BFS_SELECT_FORCED) {
      variant = p.forced;
    } else if (p.selector == BFS_SELECT_SCHEDULE && k < p.schedule_len) {
      variant = p.schedule[k];
    } else if (learned) {
      // warp 0 of every CTA evaluates the network (all CTAs compute the same bits)
      if (tid < 32) {
        const int best = learned_choice(p, s_mlp, sm.h1, tid, k, count, edges, unvisited, unvisited_edges, binv);
        if (tid == 0) sm.choice = best;
      }
      __syncthreads();
      variant = sm.choice;
    } else {
      variant = heuristic_variant(p, prev_variant, count, prev_count, edges, unvisited_edges, big_rows == 0);
    }
    if (variant < 0 || variant >= BFS_NUM_VARIANTS) variant = BFS_VARIANT_TD_BINNED;
    if (variant == BFS_VARIANT_TILED && (!kTiles || p.t_jc == nullptr)) variant = BFS_VARIANT_PULL;  // the SpMV untiled
    PHASE_TS(k, 2);
    if (part) {
      if (variant == BFS_VARIANT_PULL) pull_phase(p, k, sm, acc, G);
      else if (kTiles && variant == BFS_VARIANT_TILED) tiled_phase(p, k, sm, s_tile, acc, G);
      else topdown_phase(p, k, variant, count, nchunks, sm, acc, G);
      PHASE_TS(k, 3);
      end_phase(p, k + 1, acc, sm);
    }
    PHASE_TS(k, 4);
    PHASE_ARRIVAL(k);
    if (!bfsdev::grid_barrier_partial(p.bar, G, bar_target, p.spin_limit, p.status)) return;
    PHASE_TS(k, 6);

    if (p.want_stats && blockIdx.x == 0 && tid == 0 && k < kMaxStatLevels) {
      const uint64_t t = bfsdev::global_timer_ns();
      bfs_level_stat st;
      st.frontier_count = count;
      st.frontier_edges = edges;
      st.bin_count[0] = (int64_t)__ldcg(&c->bins[0]);  // level k's slot is recycled only in phase k + 4
      st.bin_count[1] = (int64_t)__ldcg(&c->bins[1]);
      st.bin_count[2] = (int64_t)__ldcg(&c->bins[2]);
      st.unvisited_count = unvisited;
      st.unvisited_edges = unvisited_edges;
      st.time_ns = (int64_t)(t - t_prev);
      st.variant = variant;
      st.reserved = 0;
      p.stats[k] = st;
      t_prev = t;
    }
    prev_variant = variant;
    prev_count = count;
  }

  if (gtid == 0) {
    bfsdev::barrier_pad(p.bar, nblocks, bar_target);  // partial barriers: round the counter to the grid size
    p.misc[0] = k;
    *p.edges_out = p.directed ? cum_edges : cum_edges / 2;  // arcs, or undirected edges
  }
  // ragged: copy the union-space outputs into each part's arrays, local ids
  if (p.part_out != nullptr) {
    for (int q = 0; q < p.parts; ++q) {
      const long long base = p.part_base[q], size = p.part_base[q + 1] - base;
      int32_t* lo = p.part_out[q];
      int32_t* po = p.part_out[p.parts + q];
      for (long long v = gtid; v < size; v += gthreads) {
        lo[v] = p.level[base + v];
        const int par = p.parent[base + v];
        po[v] = par >= 0 ? (int)(par - base) : -1;
      }
    }
  }
}

}  // namespace

#ifdef BFS_PHASE_TIMING
extern "C" __attribute__((visibility("default"))) int bfs_debug_phase_times(unsigned long long* host, int levels) {
  if (levels > 4096) levels = 4096;
  cudaDeviceSynchronize();
  if (cudaMemcpyFromSymbol(host, g_phase_ts, sizeof(unsigned long long) * 8 * levels) != cudaSuccess) return 1;
  static unsigned long long zero[4096][8];
  cudaMemcpyToSymbol(g_phase_ts, zero, sizeof(zero));
  return 0;
}
#endif

int launch_level_loop(const RunRequest& r, cudaStream_t s) {
  bfs_graph* g = r.g;
  Workspace* w = r.w;
  DeviceInfo di;
  if (int e = current_device_info(&di)) return e;
  if (r.nsources < 1 || r.nsources > kMaxSources) return fail(BFS_ERR_INVALID_ARG, "number of sources out of range");
  int sched_len = 0;
  const bool need_sched = r.selector == BFS_SELECT_SCHEDULE && r.h_schedule && r.schedule_len > 0;
  if (r.nsources > 1 || need_sched) {  // stage through pinned memory (no pageable-copy synchronisation)
    if (int e = stage_wait(w)) return e;
    if (r.nsources > 1) {
      std::copy(r.h_sources, r.h_sources + r.nsources, w->h_stage + kMaxSchedule);
      BFS_CUDA_TRY(cudaMemcpyAsync(w->sources, w->h_stage + kMaxSchedule, sizeof(int32_t) * r.nsources,
                                   cudaMemcpyHostToDevice, s));
    }
    if (need_sched) {
      sched_len = r.schedule_len < kMaxSchedule ? r.schedule_len : kMaxSchedule;
      std::copy(r.h_schedule, r.h_schedule + sched_len, w->h_stage);
      BFS_CUDA_TRY(cudaMemcpyAsync(w->schedule, w->h_stage, sizeof(int32_t) * sched_len, cudaMemcpyHostToDevice, s));
    }
    BFS_CUDA_TRY(cudaEventRecord(w->stage_ev, s));
  }
  if (!g->d_off || !g->d_toff || (g->nnz > 0 && (!g->d_adj || !g->d_tadj)))
    return fail(BFS_ERR_INVALID_ARG, "graph without rows");
  const bfs_tuning t = effective_tuning(g);
  // the tiled variant needs the graph's tiles: built here the first time a run may use it
  bool may_tile = r.selector == BFS_SELECT_FORCED && r.forced == BFS_VARIANT_TILED;
  for (int i = 0; i < sched_len && !may_tile; ++i) may_tile = r.h_schedule[i] == BFS_VARIANT_TILED;
  const TileSet* tiles = r.tiles;
  if (may_tile && tiles == nullptr) {
    TileSet* ts = nullptr;
    if (int e = ensure_tiles(g, s, &ts)) return e;
    tiles = ts;
  }
  LoopParams p{};
  p.off = g->d_off;
  p.adj = g->d_adj;
  p.toff = g->d_toff;
  p.tadj = g->d_tadj;
  p.directed = g->directed ? 1 : 0;
  p.dead = g->d_dead;
  p.n = g->n;
  p.nwords = w->nwords;
  p.nnz = g->nnz;
  p.level = r.level;
  p.parent = r.parent;
  for (int i = 0; i < 3; ++i) {
    p.queue[i] = w->queue[i];
    p.bits[i] = w->bits[i];
  }
  p.vis = w->vis;
  p.chunks[0] = w->chunks[0];
  p.chunks[1] = w->chunks[1];
  p.chunk_cap = w->chunk_cap;
  p.ctr = w->ctr;
  p.status = w->status;
  p.stats = w->stats;
  p.misc = w->misc;
  p.edges_out = w->edges_out;
  p.sources = w->sources;
  p.src0 = r.h_sources[0];
  p.nsources = r.nsources;
  p.selector = r.selector;
  p.forced = r.forced;
  p.schedule = w->schedule;
  p.schedule_len = sched_len;
  p.mlp = r.selector == BFS_SELECT_LEARNED ? learned_params_device() : nullptr;
  graph_feature_constants(g->n, g->nnz, &p.feat_log_n, &p.feat_log_nnz, &p.feat_inv_n, &p.feat_inv_nnz);
  p.want_stats = r.want_stats ? 1 : 0;
  p.spin_limit = r.spin_limit ? r.spin_limit : (1u << 25);
  p.warp_deg = t.warp_degree;
  p.cta_deg = t.cta_degree;
  p.pull_thread_deg = t.pull_thread_degree;
  p.chunk_deg = t.chunk_degree;
  // top-down's atomics on the parent array get dearer once 4 bytes per vertex
  // no longer fit in L2, so the switch to pull comes earlier on large graphs
  p.alpha = (float)(t.alpha * (1.0 + 4.0 * (double)g->n / (double)(di.l2_bytes > 0 ? di.l2_bytes : (1ll << 27))));
  p.beta = t.beta;
  p.parts = g->parts;
  p.part_base = g->d_part_base;
  p.part_out = r.part_out;
  if (may_tile && tiles != nullptr) {
    const TileSet* ts = tiles;
    p.t_jc = ts->jc;
    p.t_cp = ts->cp;
    p.t_ir = ts->ir;
    p.t_dir_jc = ts->tdir_jc;
    p.t_dir_ir = ts->tdir_ir;
    p.t_rb_bits = ts->rb_bits;
    p.t_cb_bits = ts->cb_bits;
    p.t_nrb = ts->nrb;
    p.t_ncb = ts->ncb;
  }

  // the tiled variant's slices follow the network's parameters in dynamic shared memory
  const size_t mlp_bytes = p.mlp ? (sizeof(float) * BFS_MLP_PARAMS + 15) / 16 * 16 : 0;
  const size_t tile_bytes = p.t_jc ? sizeof(uint32_t) * 3 * kTileWordsMax : 0;
  p.tile_smem_off = (int32_t)mlp_bytes;
  const size_t dyn_smem = mlp_bytes + tile_bytes;
  const void* kernel = p.t_jc ? (const void*)level_loop_kernel<true> : (const void*)level_loop_kernel<false>;
  {  // the attribute belongs to the current device: set it once per device
    static std::mutex mu;
    static bool configured[64] = {};
    std::lock_guard<std::mutex> lk(mu);
    if (di.device < 0 || di.device >= 64) return fail(BFS_ERR_UNSUPPORTED, "device ordinal out of range");
    if (!configured[di.device]) {
      const int max_dyn = (int)((sizeof(float) * BFS_MLP_PARAMS + 15) / 16 * 16 + sizeof(uint32_t) * 3 * kTileWordsMax);
      BFS_CUDA_TRY(cudaFuncSetAttribute((const void*)level_loop_kernel<false>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn));
      BFS_CUDA_TRY(cudaFuncSetAttribute((const void*)level_loop_kernel<true>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn));
      configured[di.device] = true;
    }
  }
  int per_sm = 0;
  BFS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, dyn_smem));
  if (per_sm < 1) return fail(BFS_ERR_CUDA, "level loop kernel cannot be resident");
  const int grid = (t.ctas_per_sm > 0 ? std::min(per_sm, t.ctas_per_sm) : per_sm) * di.sm_count;
  if (int e = prepare_barrier(w, 0, grid, s, &p.bar)) return e;
  p.small_frontier = t.small_frontier > 0 ? t.small_frontier : (t.small_frontier == 0 ? (long long)grid * kWarps : 0);
  p.narrow_edges = t.narrow_edges > 0 ? t.narrow_edges : (t.narrow_edges == 0 ? (1ll << 14) : -1);
#ifdef BFS_PHASE_TIMING
  fprintf(stderr, "level loop: %d CTAs (%d per SM), %zu bytes dynamic shared memory\n", grid, per_sm, dyn_smem);
#endif
  void* args[] = {&p};
  BFS_CUDA_TRY(cudaLaunchCooperativeKernel(kernel, dim3(grid), dim3(kBlock), args, dyn_smem, s));
  return BFS_OK;
}

}  // namespace bfsint
