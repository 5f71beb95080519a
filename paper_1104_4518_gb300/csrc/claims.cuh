// Claims of one CTA in one phase of a persistent traversal: newly reached
// vertices bound for the next frontier queue, and vertices above the chunk
// degree whose rows must be split into chunk items for a top-down level.
// Top-down claims go to a CTA buffer, pull claims to per-warp buffers (the
// two never live in the same phase, so they share storage), chunk requests to
// a third buffer; flush_claims moves the CTA's buffers to the global queue and
// chunk list with one atomic each.  Without the buffers every claim would be
// an atomic on the same counter word, and at scale 26 those atomics, serialised
// in L2, cost more than the level's memory traffic.
//
// P is a kernel's parameter block with the fields ctr (LevelCtr ring), queue[3]
// (n entries each), chunks[2] (chunk_cap entries each), n and status; every
// function here expects 512-thread CTAs.  In the bounds-checking build every
// queue and chunk-list slot is checked against its capacity before the write.
#pragma once

#include <cooperative_groups.h>
#include <cooperative_groups/scan.h>

#include "device_common.cuh"
#include "internal.h"

namespace bfsint {

constexpr int kClaimBlock = 512;
constexpr int kClaimWarps = kClaimBlock / 32;
constexpr int kQBuf = 6144;               // per-CTA buffer of next-frontier vertices (top-down claims)
constexpr int kWQBuf = 256;               // per-warp buffer of next-frontier vertices (pull claims)
constexpr int kBigBuf = 2 * kClaimBlock;  // per-CTA buffer of claimed vertices above the chunk degree
static_assert(kQBuf >= 2 * 64 * 33, "the batched transpose tiles live in the CTA buffer");

struct Claims {
  int qn;    // entries in cq (may exceed kQBuf: the excess went straight to the queue)
  int nbig;  // entries in bigv (may exceed kBigBuf: the excess went straight to the chunk list)
  unsigned qbase, bbase;
  int scan_tmp[kClaimWarps + 1];
  int bigv[kBigBuf];
  int bign[kBigBuf];  // chunk counts, then their inclusive prefix sums
  union {
    int cq[kQBuf];
    int wq[kClaimWarps][kWQBuf];
  };
};

__device__ __forceinline__ void claims_reset(Claims& cl) {
  cl.qn = 0;
  cl.nbig = 0;
}

// Exclusive CTA-wide prefix sum of one int per thread; returns the total.
// s_warp holds kClaimWarps + 1 ints.
__device__ __forceinline__ int block_exclusive_scan(int x, int* s_warp, int& excl) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(bfsdev::kFull, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_warp[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    const int v = lane < kClaimWarps ? s_warp[lane] : 0;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(bfsdev::kFull, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane < kClaimWarps) s_warp[lane] = inc - v;
    if (lane == kClaimWarps - 1) s_warp[kClaimWarps] = inc;
  }
  __syncthreads();
  excl = s_warp[wid] + incl - x;
  const int total = s_warp[kClaimWarps];
  __syncthreads();
  return total;
}

__device__ __forceinline__ unsigned chunk_count(long long deg) {
  return (unsigned)((deg + kChunkEdges - 1) / kChunkEdges);
}

// Appends the chunk items of vertex v of level knext to the chunk list
// directly (one atomic per group of converged threads).
template <typename P>
__device__ __forceinline__ void push_chunks(const P& p, int knext, int v, long long deg) {
  namespace cg = cooperative_groups;
  const unsigned nch = chunk_count(deg);
  cg::coalesced_group g = cg::coalesced_threads();
  const unsigned incl = cg::inclusive_scan(g, nch);
  unsigned base = 0;
  if (g.thread_rank() == g.size() - 1) base = atomicAdd(&p.ctr[knext % kCtrRing].chunks, incl);
  const unsigned pos = g.shfl(base, g.size() - 1) + incl - nch;
  int64_t* dst = p.chunks[knext & 1];
  for (unsigned c = 0; c < nch; ++c)
    if (bfsdev::in_range(p.status, bfsdev::kSiteChunk, (long long)pos + c, p.chunk_cap))
      dst[pos + c] = ((int64_t)v << 32) | (int64_t)c;
}

// Records vertex v of level knext for chunking in the CTA's buffer; a full
// buffer sends it to the chunk list directly.
template <typename P>
__device__ __forceinline__ void push_chunks_cta(const P& p, int knext, Claims& cl, int v, long long deg) {
  const int pos = atomicAdd(&cl.nbig, 1);
  if (pos < kBigBuf) {
    cl.bigv[pos] = v;
    cl.bign[pos] = (int)chunk_count(deg);
  } else {
    push_chunks(p, knext, v, deg);
  }
}

// Appends w to the CTA's next-frontier buffer; when the buffer is full the
// vertex goes to the queue directly (one atomic per group of converged threads).
template <typename P>
__device__ __forceinline__ void cta_enqueue(const P& p, int knext, Claims& cl, int w) {
  namespace cg = cooperative_groups;
  const int pos = atomicAdd(&cl.qn, 1);
  if (pos < kQBuf) {
    cl.cq[pos] = w;
  } else {
    cg::coalesced_group g = cg::coalesced_threads();
    unsigned base = 0;
    if (g.thread_rank() == 0) base = atomicAdd(&p.ctr[knext % kCtrRing].count, (unsigned)g.size());
    base = g.shfl(base, 0);
    if (bfsdev::in_range(p.status, bfsdev::kSiteQueue, (long long)base + g.thread_rank(), p.n))
      p.queue[knext % 3][base + g.thread_rank()] = w;
  }
}

// Appends the claimed vertices of a converged warp (one per lane where
// `claimed`) to the warp's buffer wq; once it holds at least kWQBuf - 32
// vertices (or when `flush`) they move to the queue with one atomic.
template <typename P>
__device__ __forceinline__ void warp_enqueue(const P& p, int knext, int* wq, int& nbuf, bool claimed, int v,
                                             int lane, bool flush) {
  const unsigned hm = __ballot_sync(bfsdev::kFull, claimed);
  if (claimed) wq[nbuf + __popc(hm & bfsdev::lanemask_lt())] = v;
  nbuf += __popc(hm);
  if (nbuf == 0 || (!flush && nbuf < kWQBuf - 32)) return;
  __syncwarp();
  unsigned base = 0;
  if (lane == 0) base = atomicAdd(&p.ctr[knext % kCtrRing].count, (unsigned)nbuf);
  base = __shfl_sync(bfsdev::kFull, base, 0);
  for (int i = lane; i < nbuf; i += 32)
    if (bfsdev::in_range(p.status, bfsdev::kSiteQueue, (long long)base + i, p.n)) p.queue[knext % 3][base + i] = wq[i];
  __syncwarp();
  nbuf = 0;
}

// Moves the CTA's buffered queue entries and chunk items of level knext to
// global memory.  Called by every thread of the CTA (it synchronises); the
// buffers are empty on return.
template <typename P>
__device__ __forceinline__ void flush_claims(const P& p, int knext, Claims& cl) {
  __syncthreads();
  const int nbig = min(cl.nbig, kBigBuf);
  const int nq = min(cl.qn, kQBuf);
  if (nbig == 0 && nq == 0) return;  // nothing buffered (the counters are zero already)
  int nch_total = 0;
  if (nbig > 0) {  // inclusive prefix sums of the chunk counts, two entries per thread
    const int i0 = 2 * threadIdx.x, i1 = i0 + 1;
    const int c0 = i0 < nbig ? cl.bign[i0] : 0, c1 = i1 < nbig ? cl.bign[i1] : 0;
    int excl = 0;
    nch_total = block_exclusive_scan(c0 + c1, cl.scan_tmp, excl);
    if (i0 < nbig) cl.bign[i0] = excl + c0;
    if (i1 < nbig) cl.bign[i1] = excl + c0 + c1;
  }
  if (threadIdx.x == 0) {
    LevelCtr* c = &p.ctr[knext % kCtrRing];
    if (nq) cl.qbase = atomicAdd(&c->count, (unsigned)nq);
    if (nch_total) cl.bbase = atomicAdd(&c->chunks, (unsigned)nch_total);
  }
  __syncthreads();
  int32_t* Q = p.queue[knext % 3];
  for (int i = threadIdx.x; i < nq; i += kClaimBlock)
    if (bfsdev::in_range(p.status, bfsdev::kSiteQueue, (long long)cl.qbase + i, p.n)) Q[cl.qbase + i] = cl.cq[i];
  int64_t* dst = p.chunks[knext & 1];
  for (int it = threadIdx.x; it < nch_total; it += kClaimBlock) {
    int lo = 0, hi = nbig - 1;  // the first entry whose inclusive prefix exceeds it
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (cl.bign[mid] > it) hi = mid;
      else lo = mid + 1;
    }
    const int c = it - (lo ? cl.bign[lo - 1] : 0);
    if (bfsdev::in_range(p.status, bfsdev::kSiteChunk, (long long)cl.bbase + it, p.chunk_cap))
      dst[cl.bbase + it] = ((int64_t)cl.bigv[lo] << 32) | (int64_t)c;
  }
  __syncthreads();
  if (threadIdx.x == 0) claims_reset(cl);
}

// Flushes the CTA's buffers when fewer than qroom queue entries or bigroom
// chunk requests are left, so that the work that follows cannot overflow them.
// A claim that overflows the buffer costs a global atomic on the level's one
// queue counter, and at scale 26 a top-down level that claims 2.9 M vertices
// sent a million of those to one L2 slice, which the parent atomics of the
// same level also use: the level took 0.81 ms instead of 0.44 ms.  Called by
// every thread of the CTA at a point where the whole CTA is converged.
template <typename P>
__device__ __forceinline__ void flush_claims_if_full(const P& p, int knext, Claims& cl, int qroom, int bigroom) {
  __syncthreads();
  if (cl.qn > kQBuf - qroom || cl.nbig > kBigBuf - bigroom) {  // the same on every thread after the barrier
    flush_claims(p, knext, cl);
    __syncthreads();  // thread 0's reset of the counts lands before any thread claims again
  }
}

}  // namespace bfsint
