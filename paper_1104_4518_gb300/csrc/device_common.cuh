// Device helpers shared by the traversal kernels: grid barrier with a bounded
// wait, global timer, warp utilities.  sm_103a only.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "bfs.h"

namespace bfsdev {

constexpr unsigned kFull = 0xffffffffu;

// The bounds-checking build (-DBFS_BOUNDS_CHECK) checks every index that the
// traversal kernels take from the graph or from a counter before using it.
#ifdef BFS_BOUNDS_CHECK
constexpr bool kBoundsCheck = true;
#else
constexpr bool kBoundsCheck = false;
#endif

// Where an index was checked (status[1] of a bounds error).
enum BoundsSite : int {
  kSiteTopDown = 1,       // adjacency id of a top-down expansion (single-source kernel)
  kSitePull = 2,          // adjacency id of a pull scan (single-source kernel)
  kSiteQueue = 3,         // slot of the next frontier queue
  kSiteChunk = 4,         // slot of the chunk list
  kSiteBatchTopDown = 5,  // adjacency id of a top-down expansion (batched kernel)
  kSiteBatchPull = 6,     // adjacency id of a pull scan (batched kernel)
};

// True when 0 <= i < cap.  In the bounds-checking build an index outside that
// range makes the first such thread record BFS_ERR_BOUNDS in status[0], the
// site in status[1] and the index in status[2..3] (as one 64-bit word; status
// is 16-byte aligned), and returns false so that the caller skips the access.
// The other CTAs see the status at their next grid barrier and return.  In the
// normal build it is always true and costs nothing.
__device__ __forceinline__ bool in_range(int* status, BoundsSite site, long long i, long long cap) {
  if constexpr (!kBoundsCheck) {
    return true;
  } else {
    if (i >= 0 && i < cap) return true;
    if (atomicCAS(status, 0, (int)BFS_ERR_BOUNDS) == 0) {
      status[1] = (int)site;
      *reinterpret_cast<long long*>(status + 2) = i;
    }
    return false;
  }
}

// Barrier word in global memory: a 64-bit arrival counter that only grows
// (128-byte aligned, alone in its L2 line).
struct __align__(128) GridBarrier {
  unsigned long long count;
  unsigned pad[30];
};

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_relaxed_i32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned atom_add_acqrel_u32(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier for a cooperative launch (all CTAs co-resident).  Every
// CTA adds one to the arrival counter without waiting for the result and
// polls until the counter reaches its target, nblocks more than at the
// previous barrier: no CTA has to learn that it came last and publish a
// release, which saves a round trip to L2 per barrier.
// `target` is thread 0's copy of the count the barrier waits for; it starts
// at barrier_base().  Every wait is bounded: after `spin_limit` polls (or once
// another CTA has posted an error) the CTA records BFS_ERR_TIMEOUT in *status
// and the barrier returns false, so that the kernel can return instead of
// hanging.
// Ordering: __syncthreads + a gpu-scope fence and the release add by thread 0
// publish the CTA's writes before its arrival; the acquire load that sees the
// target, then __syncthreads, order the CTA's later reads after every CTA's
// writes.
__device__ __forceinline__ bool grid_barrier(GridBarrier* bar, unsigned nblocks, unsigned long long& target,
                                             unsigned spin_limit, int* status) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    target += nblocks;
    __threadfence();
    red_release_add_u64(&bar->count, 1ull);
    unsigned polls = 0;
    while (ld_acquire_u64(&bar->count) < target) {
      if (++polls > spin_limit || ld_relaxed_i32(status) != 0) {
        ok = 0;
        break;
      }
      __nanosleep(32);
    }
    if (!ok) atomicCAS(status, 0, (int)BFS_ERR_TIMEOUT);
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// The grid barrier of a level that only `arrivals` CTAs (those with
// blockIdx.x < arrivals) worked on: those CTAs arrive as in grid_barrier, the
// others only wait until the counter reaches the new target (polling less
// often, since nothing waits on them).  Every CTA must pass the same
// `arrivals`.  A launch that used such barriers must pad the counter to a
// multiple of its grid size before it ends (barrier_pad).
__device__ __forceinline__ bool grid_barrier_partial(GridBarrier* bar, unsigned arrivals, unsigned long long& target,
                                                     unsigned spin_limit, int* status) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const bool arrive = blockIdx.x < arrivals;
    target += arrivals;
    if (arrive) {
      __threadfence();
      red_release_add_u64(&bar->count, 1ull);
    }
    unsigned polls = 0;
    while (ld_acquire_u64(&bar->count) < target) {
      if (++polls > spin_limit || ld_relaxed_i32(status) != 0) {
        ok = 0;
        break;
      }
      __nanosleep(arrive ? 32 : 2048);
    }
    if (!ok) atomicCAS(status, 0, (int)BFS_ERR_TIMEOUT);
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Called by one thread of one CTA after the last barrier of a launch: adds
// the arrivals that round the counter up to a multiple of nblocks, so that
// the next launch's barrier_base finds its base.  `target` is that thread's
// copy of the last barrier's target.
__device__ __forceinline__ void barrier_pad(GridBarrier* bar, unsigned nblocks, unsigned long long target) {
  const unsigned long long r = target % nblocks;
  if (r) red_release_add_u64(&bar->count, nblocks - r);
}

// The count at which this launch's barriers start, read by thread 0 at kernel
// start.  Every launch that used the word before ended on a multiple of
// nblocks (the host zeroes the word when a kernel's grid size changes, and
// after an error), and until this CTA arrives fewer than nblocks arrivals of
// this launch can have happened, so rounding down gives the exact base.
__device__ __forceinline__ unsigned long long barrier_base(const GridBarrier* bar, unsigned nblocks) {
  const unsigned long long c = ld_acquire_u64(&bar->count);
  return c - c % nblocks;
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

}  // namespace bfsdev
