// Device helpers shared by the traversal kernels: grid barrier with a bounded
// wait, global timer, warp utilities.  sm_103a only.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "bfs.h"

namespace bfsdev {

constexpr unsigned kFull = 0xffffffffu;

// Barrier words in global memory, 128-byte aligned so that the arrival
// counter and the release epoch sit in separate L2 sectors.
struct __align__(128) GridBarrier {
  unsigned count;
  unsigned pad0[31];
  unsigned epoch;
  unsigned pad1[31];
};

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
// wait is bounded: after `spin_limit` polls (or once another CTA has posted an
// error) the CTA records BFS_ERR_TIMEOUT in *status and the barrier returns
// false, so that the kernel can return instead of hanging.  `epoch` is the
// CTA's copy of the release counter (read once at kernel start).
// Ordering: __syncthreads + a gpu-scope fence by thread 0 publish the CTA's
// writes before its arrival; the acquire load that sees the new epoch, then
// __syncthreads, order the CTA's later reads after every CTA's writes.
__device__ __forceinline__ bool grid_barrier(GridBarrier* bar, unsigned nblocks, unsigned& epoch,
                                             unsigned spin_limit, int* status) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned target = epoch + 1;
    __threadfence();
    const unsigned arrived = atom_add_acqrel_u32(&bar->count, 1u);
    if (arrived == nblocks - 1) {
      bar->count = 0;  // nobody arrives at the next barrier before the release below
      st_release_u32(&bar->epoch, target);
    } else {
      unsigned polls = 0;
      while (ld_acquire_u32(&bar->epoch) != target) {
        if (++polls > spin_limit || ld_relaxed_i32(status) != 0) {
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    if (!ok) atomicCAS(status, 0, (int)BFS_ERR_TIMEOUT);
    epoch = target;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

}  // namespace bfsdev
