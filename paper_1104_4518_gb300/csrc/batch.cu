// Batched BFS: up to 64 roots in one persistent traversal.
//
// Every vertex carries 64-bit words: F_k[v] (bit r set when v is in the
// frontier of root r at level k), V[v] (bit r set when root r has reached v)
// and F_{k+1}[v].  One level is the boolean sparse matrix-dense matrix product
// F_{k+1} = (A (x) F_k) AND NOT V, i.e. the SpMSV of Sec. 3.2 for 64 vectors at
// once.  Parents follow the same max-id rule as the single-root traversal: for
// a vertex v newly reached by root r, parent_r[v] is the largest neighbour u
// with bit r in F_k[u], found by scanning v's sorted row from the largest id
// down and masking off the bits already resolved.
//
// "Reached before level k+1" is tested as V | F_k, so V only has to absorb a
// frontier's bits during the level that expands it, and every level is one
// phase.  Two ways to expand a level (identical results):
//   pull     : every vertex not yet reached by all roots scans its row; short
//              rows lane by lane, rows up to kChunkEdges entries by the whole
//              warp, longer rows in kChunkEdges-entry chunks (a static table
//              built with the graph), one CTA per chunk, the chunks combining
//              through atomicMax on the parents and atomicOr on F_{k+1};
//   top-down : every frontier row ORs its bits into F_{k+1} of unreached
//              neighbours and offers itself as their parent with atomicMax
//              for each new root bit (every frontier neighbour offers, so the
//              largest id wins); the first writer of a root bit writes the
//              level, the first writer of any bit enqueues the neighbour.
//              Rows above kChunkEdges entries are split into chunk items.
// Output rows are root-major: level[r * n + v], parent[r * n + v].  During
// the traversal the results go to vertex-major scratch (sl / sp [v][r], one
// row of `stride` ints per vertex), so that the results of one vertex share a
// few sectors instead of landing 4 * n bytes apart; a last phase transposes the
// scratch into the outputs through shared-memory tiles, coalesced both ways.
//
// The words are 8, 16, 32 or 64 bits wide (one bit per root of the
// traversal; bit arithmetic is done in 64-bit registers whatever the word).
// 64 is the default: a traversal's row scans cost about the same whatever
// the number of roots it carries, so fewer, wider traversals win even when
// the frontier array no longer fits in L2 (measured at scales 22 to 26).
#include <cooperative_groups.h>
#include <climits>

#include "claims.cuh"
#include "device_common.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace bfsint {
namespace {

using bfsdev::kFull;

constexpr int kBBlock = 512;
static_assert(kBBlock == kClaimBlock, "the claim buffers assume 512-thread CTAs");
constexpr int kBWarps = kBBlock / 32;
constexpr int kShortRow = 32;  // rows up to this length are scanned by one lane

struct BatchParams {
  const int64_t* __restrict__ off;   // out-rows: top-down
  const int32_t* __restrict__ adj;
  const int64_t* __restrict__ toff;  // in-rows: pull (the same arrays when undirected)
  const int32_t* __restrict__ tadj;
  int32_t directed;
  int32_t n;
  long long nnz;
  int32_t k;  // roots in this traversal (<= 64)
  uint64_t mask;
  int32_t src[64];
  int32_t* level;   // [k][n]
  int32_t* parent;  // [k][n]
  int32_t* sl;      // scratch levels [n][stride]
  int32_t* sp;      // scratch parents [n][stride]
  int32_t stride;   // roots per scratch row (the word width)
  void* F[3];  // Word[n] each
  void* V;     // Word[n]
  int32_t* queue[3];
  int64_t* chunks[2];
  long long chunk_cap;  // entries of each chunk list
  const int64_t* big;  // chunks of in-rows longer than kChunkEdges (static, per graph)
  long long nbig;
  LevelCtr* ctr;
  bfsdev::GridBarrier* bar;
  int* status;
  int32_t* misc;
  bfs_level_stat* stats;  // per-level statistics when non-null
  unsigned spin_limit;
  long long td_limit;
};

using Bits = unsigned long long;

// atomicOr of v into a word of an 8-, 16-, 32- or 64-bit array; returns the old word.
template <typename Word>
__device__ __forceinline__ Bits atomic_or_word(Word* a, Bits v) {
  if constexpr (sizeof(Word) == 8) {
    return atomicOr(reinterpret_cast<unsigned long long*>(a), v);
  } else if constexpr (sizeof(Word) == 4) {
    return atomicOr(reinterpret_cast<unsigned*>(a), (unsigned)v);
  } else {  // the aligned 32-bit word that holds *a
    const uintptr_t ad = reinterpret_cast<uintptr_t>(a);
    const int sh = (int)(ad & 3u) * 8;
    const unsigned old = atomicOr(reinterpret_cast<unsigned*>(ad & ~(uintptr_t)3), (unsigned)v << sh);
    return (Bits)((old >> sh) & ((1u << (8 * sizeof(Word))) - 1u));
  }
}

// OR of v over the warp (v has at most 8 * sizeof(Word) bits).
template <typename Word>
__device__ __forceinline__ Bits warp_or(Bits v) {
  const unsigned lo = __reduce_or_sync(kFull, (unsigned)v);
  if constexpr (sizeof(Word) == 8) {
    const unsigned hi = __reduce_or_sync(kFull, (unsigned)(v >> 32));
    return ((Bits)hi << 32) | lo;
  } else {
    return lo;
  }
}

// Writes level / parent of the roots in `bits` for vertex v.
__device__ __forceinline__ void write_hits(const BatchParams& p, uint64_t bits, int v, int u, int lvl) {
  while (bits) {
    const int r = __ffsll((long long)bits) - 1;
    bits &= bits - 1;
    const long long o = (long long)v * p.stride + r;
    p.sl[o] = lvl;
    p.sp[o] = u;
  }
}

// One lane scans rows [b, e) of v from the top, four loads at a time, and
// resolves the roots in `need`; returns the bits found.
template <typename Word>
__device__ __forceinline__ uint64_t resolve_lane(const BatchParams& p, const Word* F, int v, long long b,
                                                 long long e, uint64_t need, int lvl) {
  uint64_t found = 0;
  long long j = e - 1;
  while (j >= b && need) {
    int u[4];
    uint64_t f[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) u[q] = (j - q >= b) ? __ldg(&p.tadj[j - q]) : -1;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const bool live = bfsdev::kBoundsCheck
                            ? j - q >= b && bfsdev::in_range(p.status, bfsdev::kSiteBatchPull, u[q], p.n)
                            : u[q] >= 0;
      f[q] = live ? (Bits)F[u[q]] : 0ull;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint64_t h = f[q] & need;
      if (h) {
        write_hits(p, h, v, u[q], lvl);
        need &= ~h;
        found |= h;
      }
    }
    j -= 4;
  }
  return found;
}

// The whole warp scans entries [b, e) of v's row from the top, 128 entries per
// step (four loads per lane in flight, examined in descending position order);
// returns the bits found (same value in every lane).  kChunk: the range is one
// chunk of a longer row, so the first hit of a root is only this chunk's
// candidate: it is offered with atomicMax and the level is left to the claim.
template <typename Word, bool kChunk>
__device__ __forceinline__ uint64_t resolve_warp(const BatchParams& p, const Word* F, int v, long long b,
                                                 long long e, uint64_t need, int lvl, int lane) {
  uint64_t found = 0;
  for (long long top = e; top > b && need; top -= 128) {
    int u[4];
    uint64_t f[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const long long j = top - 1 - lane - 32 * q;
      u[q] = j >= b ? __ldg(&p.tadj[j]) : 0;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
      f[q] = (top - 1 - lane - 32 * q >= b && bfsdev::in_range(p.status, bfsdev::kSiteBatchPull, u[q], p.n))
                 ? ((Bits)F[u[q]] & need)
                 : 0ull;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint64_t nb = warp_or<Word>(f[q]) & need;
      found |= nb;
      need &= ~nb;
      while (nb) {  // each new root takes the lowest lane holding its bit (the highest position)
        const int r = __ffsll((long long)nb) - 1;
        nb &= nb - 1;
        const unsigned who = __ballot_sync(kFull, (f[q] >> r) & 1ull);
        const int pu = __shfl_sync(kFull, u[q], __ffs(who) - 1);
        if (lane == 0) {
          const long long o = (long long)v * p.stride + r;
          if (kChunk) {
            atomicMax(&p.sp[o], pu);
          } else {
            p.sl[o] = lvl;
            p.sp[o] = pu;
          }
        }
      }
    }
  }
  return found;
}

// Resolves the parents of 32 vertices (one per lane, need = roots to find)
// against frontier F; lanes with short rows scan alone, long rows get the warp.
template <typename Word>
__device__ __forceinline__ uint64_t resolve_group(const BatchParams& p, const Word* F, int v, long long b,
                                                  long long e, uint64_t need, int lvl, int lane) {
  uint64_t found = 0;
  const bool longrow = need && (e - b) > kShortRow;
  if (need && !longrow) found = resolve_lane(p, F, v, b, e, need, lvl);
  unsigned lm = __ballot_sync(kFull, longrow);
  while (lm) {
    const int l = __ffs(lm) - 1;
    lm &= lm - 1;
    const int lv = __shfl_sync(kFull, v, l);
    const long long lb = __shfl_sync(kFull, b, l), le = __shfl_sync(kFull, e, l);
    const uint64_t ln = __shfl_sync(kFull, need, l);
    const uint64_t fw = resolve_warp<Word, false>(p, F, lv, lb, le, ln, lvl, lane);
    if (lane == l) found = fw;
  }
  return found;
}

// Top-down visit of edge (u -> w) with frontier bits f of u at level knext - 1.
template <typename Word>
__device__ __forceinline__ void td_visit(const BatchParams& p, const Word* Fc, Word* Fn, const Word* V, int knext,
                                         uint64_t f, int u, int w, Claims& cl) {
  if (!bfsdev::in_range(p.status, bfsdev::kSiteBatchTopDown, w, p.n)) return;
  const uint64_t nb = f & ~((Bits)V[w] | (Bits)Fc[w]);
  if (!nb) return;
  // u is a parent candidate of w for every new root bit; an offer no larger than
  // the current one is dropped without an atomic (the row of w is one 256-byte
  // line, read once)
  for (uint64_t b = nb; b;) {
    const int r = __ffsll((long long)b) - 1;
    b &= b - 1;
    int32_t* o = &p.sp[(long long)w * p.stride + r];
    if (__ldcg(o) < u) atomicMax(o, u);
  }
  if (((Bits)Fn[w] & nb) == nb) return;
  const Bits old = atomic_or_word(&Fn[w], nb);
  for (uint64_t b = nb & ~old; b;) {
    const int r = __ffsll((long long)b) - 1;
    b &= b - 1;
    p.sl[(long long)w * p.stride + r] = knext;
  }
  if (old == 0) {
    cta_enqueue(p, knext, cl, w);
    const long long deg = __ldg(&p.off[w + 1]) - __ldg(&p.off[w]);
    if (deg > kChunkEdges) push_chunks_cta(p, knext, cl, w, deg);
  }
}

// Pull over one kChunkEdges-entry chunk [rb, re) of a long row of v by one warp;
// chunks of the same row combine through atomicMax on the parents and atomicOr
// on F_{k+1}, whose first setter of a root bit writes that root's level, and
// whose first setter of any bit claims v for the queue.
template <typename Word>
__device__ __forceinline__ void pull_chunk(const BatchParams& p, const Word* Fc, Word* Fn, int knext, int v,
                                           long long rb, long long re, uint64_t need, int lane, Claims& cl,
                                           int* wq, int& nbuf) {
  const uint64_t found = resolve_warp<Word, true>(p, Fc, v, rb, re, need, knext, lane);
  bool claimed = false;
  if (lane == 0 && found) {
    const Bits old = atomic_or_word(&Fn[v], found);
    for (uint64_t bb = found & ~old; bb;) {
      const int r = __ffsll((long long)bb) - 1;
      bb &= bb - 1;
      p.sl[(long long)v * p.stride + r] = knext;
    }
    if (old == 0) {
      claimed = true;
      push_chunks_cta(p, knext, cl, v, __ldg(&p.off[v + 1]) - __ldg(&p.off[v]));
    }
  }
  warp_enqueue(p, knext, wq, nbuf, claimed, v, lane, false);
}

template <typename Word>
__global__ void __launch_bounds__(kBBlock, 2) batch_kernel(BatchParams p) {
  Word* F[3] = {static_cast<Word*>(p.F[0]), static_cast<Word*>(p.F[1]), static_cast<Word*>(p.F[2])};
  Word* V = static_cast<Word*>(p.V);
  __shared__ Claims cl;
  const int tid = threadIdx.x, lane = tid & 31;
  unsigned long long bar_target = 0;
  if (tid == 0) {
    bar_target = bfsdev::barrier_base(p.bar, gridDim.x);
    claims_reset(cl);
  }
  const long long G = gridDim.x;
  const long long gtid = (long long)blockIdx.x * kBBlock + tid;
  const long long gthreads = G * kBBlock;
  const long long gwarps = G * kBWarps;
  const long long gwarp = blockIdx.x + (long long)(tid >> 5) * G;  // round-robin over CTAs
  const unsigned nblocks = gridDim.x;

  // init: scratch parents to -1 (atomicMax offers need a floor; scratch levels
  // are only read where V says the root reached the vertex), bitsets to 0,
  // counters to 0
  const long long total = (long long)p.n * p.stride;
  for (long long i = gtid; i < total; i += gthreads) p.sp[i] = -1;
  for (long long v = gtid; v < p.n; v += gthreads) {
    F[0][v] = 0;
    F[1][v] = 0;
    F[2][v] = 0;
    V[v] = 0;
  }
  if (blockIdx.x == 0 && tid < kCtrRing * (int)(sizeof(LevelCtr) / 8))
    reinterpret_cast<unsigned long long*>(p.ctr)[tid] = 0ull;
  if (!bfsdev::grid_barrier(p.bar, nblocks, bar_target, p.spin_limit, p.status)) return;

  // seed: root r sets bit r of its own vertex (roots may repeat)
  if (blockIdx.x == 0 && tid < p.k) {
    const int s = p.src[tid];
    const uint64_t bit = 1ull << tid;
    const long long o = (long long)s * p.stride + tid;
    p.sl[o] = 0;
    p.sp[o] = s;
    atomic_or_word(&V[s], bit);
    const Bits old = atomic_or_word(&F[0][s], bit);
    if (old == 0) {
      const unsigned pos = atomicAdd(&p.ctr[0].count, 1u);
      p.queue[0][pos] = s;
      const long long deg = __ldg(&p.off[s + 1]) - __ldg(&p.off[s]);
      if (deg > kChunkEdges) push_chunks(p, 0, s, deg);
    }
  }
  if (!bfsdev::grid_barrier(p.bar, nblocks, bar_target, p.spin_limit, p.status)) return;

  int k = 0;
  uint64_t t_prev = 0;
  if (p.stats && blockIdx.x == 0 && tid == 0) t_prev = bfsdev::global_timer_ns();
  for (;; ++k) {
    const unsigned count = __ldcg(&p.ctr[k % kCtrRing].count);
    if (count == 0) break;
    const unsigned nchunks = __ldcg(&p.ctr[k % kCtrRing].chunks);
    const Word* Fc = F[k % 3];
    Word* Fn = F[(k + 1) % 3];
    const int32_t* Q = p.queue[k % 3];
    const int knext = k + 1;
    if (blockIdx.x == 0 && tid < (int)(sizeof(LevelCtr) / 8))
      reinterpret_cast<unsigned long long*>(&p.ctr[(k + 4) % kCtrRing])[tid] = 0ull;
    if (k >= 1) {  // clear F_{k-1} for reuse as F_{k+2}
      Word* clr = F[(k + 2) % 3];
      const unsigned pc = __ldcg(&p.ctr[(k + kCtrRing - 1) % kCtrRing].count);
      if ((long long)pc * 8 < p.n) {
        const int32_t* PQ = p.queue[(k + 2) % 3];
        for (long long i = gtid; i < pc; i += gthreads) clr[PQ[i]] = 0;
      } else {
        for (long long v = gtid; v < p.n; v += gthreads) clr[v] = 0;
      }
    }

    const bool topdown = (long long)count <= p.td_limit;
    const int wid = tid >> 5;
    if (topdown) {
      // frontier rows above kChunkEdges: one CTA per chunk item, with room in the
      // CTA's buffers for the item's claims
      const int64_t* items = p.chunks[k & 1];
      for (long long ci = blockIdx.x; ci < nchunks; ci += G) {
        flush_claims_if_full(p, knext, cl, kChunkEdges, kBigBuf / 2);
        const int64_t it = items[ci];
        const int u = (int)(it >> 32);
        const long long rb = __ldg(&p.off[u]) + (it & 0xffffffffll) * kChunkEdges;
        const long long re = min(rb + (long long)kChunkEdges, (long long)__ldg(&p.off[u + 1]));
        const uint64_t f = (Bits)Fc[u];
        for (long long j = rb + tid; j < re; j += kBBlock) td_visit(p, Fc, Fn, V, knext, f, u, __ldg(&p.adj[j]), cl);
      }
      // other frontier rows: one warp each; every frontier vertex folds its bits into V
      for (long long i = gwarp; i < count; i += gwarps) {
        const int u = Q[i];
        const uint64_t f = (Bits)Fc[u];
        if (lane == 0) V[u] = (Word)((Bits)V[u] | f);
        const long long b = __ldg(&p.off[u]), e = __ldg(&p.off[u + 1]);
        if (e - b > kChunkEdges) continue;
        for (long long j = b + lane; j < e; j += 32) td_visit(p, Fc, Fn, V, knext, f, u, __ldg(&p.adj[j]), cl);
      }
    } else {
      int* wq = cl.wq[wid];
      int nbuf = 0;
      // long rows: one warp per chunk of the static table
      for (long long ci = gwarp; ci < p.nbig; ci += gwarps) {
        const int64_t it = p.big[ci];
        const int v = (int)(it >> 32);
        const uint64_t need = __shfl_sync(kFull, ~((Bits)V[v] | (Bits)Fc[v]) & p.mask, 0);
        if (!need) continue;
        const long long rb = __ldg(&p.toff[v]) + (it & 0xffffffffll) * kChunkEdges;
        const long long re = min(rb + (long long)kChunkEdges, (long long)__ldg(&p.toff[v + 1]));
        pull_chunk(p, Fc, Fn, knext, v, rb, re, need, lane, cl, wq, nbuf);
      }
      // other rows: 32 vertices per warp; the owner lane updates V and F_{k+1}
      // word indices fit 32 bits: n < 2^31
      const int nw = (int)(((long long)p.n + 31) / 32), gw = (int)gwarps;
      constexpr int kGroupWords = 16;
      // words [0, S) are dealt one at a time round robin (warp i takes i, i + gw, ...),
      // the rest in groups of kGroupWords words from the level's cursor, each fetch issued
      // one group ahead.  Full row scans make some words far dearer than others: with an
      // all-static deal a level waited on its slowest warps (64 roots at R-MAT scale 26:
      // 104.6 ms, 94.4 with the dynamic tail).  With few words per warp all are dealt
      // round robin: 16-word groups from the first word left warps idle on the 2^27-edge
      // edgefactor-16 and -64 graphs (16 roots: 3 % and 4 % slower).
      const int S = nw > 64 * gw ? gw * ((nw / 2) / gw) : nw;
      const int ngroups = (nw - S + kGroupWords - 1) / kGroupWords;
      auto pull_word = [&](int ww) {
        const long long v0 = (long long)ww * 32 + lane;
        const int v = (int)v0;
        uint64_t need = 0, vv = 0, fv = 0;
        long long b = 0, e = 0;
        if (v0 < p.n) {
          vv = (Bits)V[v];
          fv = (Bits)Fc[v];
          need = ~(vv | fv) & p.mask;
          if (need) {
            b = __ldg(&p.toff[v]);
            e = __ldg(&p.toff[v + 1]);
            if (e == b || e - b > kChunkEdges) need = 0;
          }
        }
        const uint64_t found = resolve_group(p, Fc, v, b, e, need, knext, lane);
        if (v0 < p.n) {
          const uint64_t nv = vv | fv | found;
          if (nv != vv) V[v] = (Word)nv;
          if (found) {
            Fn[v] = (Word)found;
            if (p.directed) {  // the next level's top-down expansion needs the chunks of a long out-row
              const long long deg = __ldg(&p.off[v + 1]) - __ldg(&p.off[v]);
              if (deg > kChunkEdges) push_chunks_cta(p, knext, cl, v, deg);
            }
          }
        }
        warp_enqueue(p, knext, wq, nbuf, found != 0, v, lane, false);
      };
      for (int ww = (int)gwarp; ww < S; ww += gw) pull_word(ww);
      if (ngroups > 0) {
        unsigned next = 0;
        if (lane == 0) next = (unsigned)atomicAdd(&p.ctr[k % kCtrRing].pad, 1ull);
        for (int grp = (int)__shfl_sync(kFull, next, 0); grp < ngroups; grp = (int)__shfl_sync(kFull, next, 0)) {
          if (lane == 0) next = (unsigned)atomicAdd(&p.ctr[k % kCtrRing].pad, 1ull);  // fetched one group ahead
          const int w0 = S + grp * kGroupWords, w1 = min(nw, w0 + kGroupWords);
          for (int ww = w0; ww < w1; ++ww) pull_word(ww);
        }
      }
      warp_enqueue(p, knext, wq, nbuf, false, 0, lane, true);
    }
    flush_claims(p, knext, cl);
    if (!bfsdev::grid_barrier(p.bar, nblocks, bar_target, p.spin_limit, p.status)) return;
    if (p.stats && blockIdx.x == 0 && tid == 0 && k < kMaxStatLevels) {
      const uint64_t t = bfsdev::global_timer_ns();
      bfs_level_stat st{};
      st.frontier_count = count;
      st.time_ns = (int64_t)(t - t_prev);
      st.variant = topdown ? BFS_VARIANT_TD_WARP : BFS_VARIANT_PULL;
      p.stats[k] = st;
      t_prev = t;
    }
  }
  if (gtid == 0) p.misc[1] = k;

  // transpose the scratch rows of 32 vertices into the root-major outputs
  // (the loop ended right after a grid barrier, so the scratch is final, and V
  // holds every root bit of every vertex reached).  Scratch rows are read as
  // int4 (S is a multiple of 4 and the scratch 16-byte aligned); output rows
  // are written as int4 when n is a multiple of 4 and both outputs start on a
  // 16-byte boundary (every row then does), else one int at a time.
  int* tl = cl.cq;            // [S][33] levels
  int* tp = cl.cq + 64 * 33;  // [S][33] parents
  const int S = p.stride, S4 = S / 4;
  const bool vec_out = (p.n & 3) == 0 &&
                       ((reinterpret_cast<uintptr_t>(p.level) | reinterpret_cast<uintptr_t>(p.parent)) & 15u) == 0;
  const long long ntiles = ((long long)p.n + 31) / 32;
  for (long long t = blockIdx.x; t < ntiles; t += G) {
    const long long v0 = t * 32;
    const int nv = (int)min(32ll, (long long)p.n - v0);
    for (int e = tid; e < 32 * S4; e += kBBlock) {
      const int i = e / S4, c = e - i * S4;
      if (i < nv) {
        const long long o = (v0 + i) * S + 4 * c;
        const int4 lv = *reinterpret_cast<const int4*>(p.sl + o);
        const int4 pv = *reinterpret_cast<const int4*>(p.sp + o);
        const Bits vv = (Bits)V[v0 + i] >> (4 * c);
        tl[(4 * c + 0) * 33 + i] = (vv & 1ull) ? lv.x : -1;
        tl[(4 * c + 1) * 33 + i] = (vv & 2ull) ? lv.y : -1;
        tl[(4 * c + 2) * 33 + i] = (vv & 4ull) ? lv.z : -1;
        tl[(4 * c + 3) * 33 + i] = (vv & 8ull) ? lv.w : -1;
        tp[(4 * c + 0) * 33 + i] = pv.x;
        tp[(4 * c + 1) * 33 + i] = pv.y;
        tp[(4 * c + 2) * 33 + i] = pv.z;
        tp[(4 * c + 3) * 33 + i] = pv.w;
      }
    }
    __syncthreads();
    for (int e = tid; e < 8 * p.k; e += kBBlock) {
      const int r = e >> 3, i = 4 * (e & 7);
      const long long o = (long long)r * p.n + v0 + i;
      const int* L = tl + r * 33 + i;
      const int* P = tp + r * 33 + i;
      if (vec_out && i + 4 <= nv) {
        *reinterpret_cast<int4*>(p.level + o) = make_int4(L[0], L[1], L[2], L[3]);
        *reinterpret_cast<int4*>(p.parent + o) = make_int4(P[0], P[1], P[2], P[3]);
      } else {
        for (int m = 0; m < 4 && i + m < nv; ++m) {
          p.level[o + m] = L[m];
          p.parent[o + m] = P[m];
        }
      }
    }
    __syncthreads();
  }
}

}  // namespace

int launch_batch(const BatchRequest& r, cudaStream_t s) {
  bfs_graph* g = r.g;
  Workspace* w = r.w;
  DeviceInfo di;
  if (int e = current_device_info(&di)) return e;
  if (r.width != 8 && r.width != 16 && r.width != 32 && r.width != 64)
    return fail(BFS_ERR_INVALID_ARG, "batch width must be 8, 16, 32 or 64");
  if (r.k < 1 || r.k > r.width) return fail(BFS_ERR_INVALID_ARG, "batch of 1..width roots expected");
  if (!g->d_off || !g->d_toff || (g->nnz > 0 && (!g->d_adj || !g->d_tadj)))
    return fail(BFS_ERR_INVALID_ARG, "graph without rows");
  if (int e = ensure_batch_state(g, w)) return e;
  const bfs_tuning t = effective_tuning(g);
  BatchParams p{};
  p.off = g->d_off;
  p.adj = g->d_adj;
  p.toff = g->d_toff;
  p.tadj = g->d_tadj;
  p.directed = g->directed ? 1 : 0;
  p.n = g->n;
  p.nnz = g->nnz;
  p.k = r.k;
  p.mask = r.k == 64 ? ~0ull : ((1ull << r.k) - 1ull);
  for (int i = 0; i < r.k; ++i) p.src[i] = r.h_sources[i];
  p.level = r.level;
  p.parent = r.parent;
  p.stride = r.width;
  p.sl = w->bscr;
  p.sp = w->bscr + (size_t)g->n * 64;
  for (int i = 0; i < 3; ++i) {
    p.F[i] = w->bset[i];
    p.queue[i] = w->queue[i];
  }
  p.V = w->bvis;
  p.chunks[0] = w->chunks[0];
  p.chunks[1] = w->chunks[1];
  p.chunk_cap = w->chunk_cap;
  p.big = g->d_big;
  p.nbig = g->nbig;
  p.ctr = w->ctr;
  p.status = w->status;
  p.misc = w->misc;
  p.stats = r.want_stats ? w->stats : nullptr;
  p.spin_limit = r.spin_limit ? r.spin_limit : (1u << 25);
  p.td_limit = t.batch_topdown_limit;
  const void* fn = r.width == 8    ? (const void*)batch_kernel<uint8_t>
                   : r.width == 16 ? (const void*)batch_kernel<uint16_t>
                   : r.width == 32 ? (const void*)batch_kernel<uint32_t>
                                   : (const void*)batch_kernel<uint64_t>;
  int per_sm = 0;
  BFS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBBlock, 0));
  if (per_sm < 1) return fail(BFS_ERR_CUDA, "batch kernel cannot be resident");
  const int grid = per_sm * di.sm_count;
  if (int e = prepare_barrier(w, 1, grid, s, &p.bar)) return e;
  void* args[] = {&p};
  BFS_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kBBlock), args, 0, s));
  return BFS_OK;
}

}  // namespace bfsint
