// bfs_run_static: the single-source traversal for callers that cannot
// allocate device memory.
//
// It runs the same level-loop kernel as bfs_run, but every scratch buffer of
// the traversal (frontier queues and bitmaps, visited bitmap, chunk items,
// level counters, grid-barrier words, status) lives in one file-scope
// `static __device__` array of fixed size instead of a workspace from
// cudaMalloc.  Each GPU that loads the library holds that array until the
// process exits.  Host code cannot use the array's name as a device address
// (in host code it names a host-side stand-in), so the device address is
// obtained once per device with cudaGetSymbolAddress and passed to the kernel.
#include <mutex>

#include "device_common.cuh"
#include "internal.h"
#include "nvtx_range.h"

namespace bfsint {
namespace {

constexpr int32_t kStaticMaxVertices = 1 << 20;   // n <= 1,048,576
constexpr int64_t kStaticMaxEntries = 1ll << 26;  // nnz <= 67,108,864

constexpr size_t round256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t kQueueBytes = round256(sizeof(int32_t) * kStaticMaxVertices);
constexpr size_t kBitsBytes = round256(sizeof(uint32_t) * (kStaticMaxVertices / 32));
constexpr int64_t kChunkCap = 2 * (kStaticMaxEntries / kChunkEdges) + kMaxSources + 1024;
constexpr size_t kChunkBytes = round256(sizeof(int64_t) * kChunkCap);
constexpr size_t kCtrBytes = round256(sizeof(LevelCtr) * kCtrRing);
constexpr size_t kBarrierBytes = round256(sizeof(bfsdev::GridBarrier));
constexpr size_t kSmallBytes = 256;  // status (int[4]), misc, edge count, offset-check flag

constexpr size_t kOffQueue = 0;
constexpr size_t kOffBits = kOffQueue + 3 * kQueueBytes;
constexpr size_t kOffVis = kOffBits + 3 * kBitsBytes;
constexpr size_t kOffChunks = kOffVis + kBitsBytes;
constexpr size_t kOffCtr = kOffChunks + 2 * kChunkBytes;
constexpr size_t kOffBarrier = kOffCtr + kCtrBytes;
constexpr size_t kOffSmall = kOffBarrier + kBarrierBytes;
constexpr size_t kScratchBytes = kOffSmall + kSmallBytes;  // 15,287,296 bytes

// The scratch shared by every call in this process (zero-initialised at module load).
static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

std::mutex g_mu;
unsigned char* g_addr[64] = {nullptr};  // device address of g_static_scratch, per device ordinal

// Set-up on the first call on a device (that device current): look up the
// array's device address and clear the barrier and status words.
int scratch_address(unsigned char** out) {
  int dev = 0;
  BFS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(BFS_ERR_UNSUPPORTED, "bfs_run_static: device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "bfs_run_static: cudaGetSymbolAddress of the static scratch");
    e = cudaMemset(static_cast<unsigned char*>(p) + kOffBarrier, 0, kBarrierBytes + kSmallBytes);
    if (e != cudaSuccess) return cuda_fail(e, "bfs_run_static: clearing the static scratch");
    g_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_addr[dev];
  return BFS_OK;
}

}  // namespace
}  // namespace bfsint

using namespace bfsint;

extern "C" int bfs_run_static(const int64_t* offsets, const int32_t* adj, int32_t n, int64_t nnz, int32_t source,
                              int32_t* parent_out, int32_t* level_out, void* stream) {
  NvtxRange nvtx_range("bfs_run_static");
  if (n < 1 || n > kStaticMaxVertices)
    return fail(BFS_ERR_INVALID_ARG, "bfs_run_static: n must be in [1, 1048576] (size of the static scratch)");
  if (nnz < 0 || nnz > kStaticMaxEntries)
    return fail(BFS_ERR_INVALID_ARG, "bfs_run_static: nnz must be in [0, 67108864] (size of the static scratch)");
  if (!offsets || (nnz > 0 && !adj) || !parent_out || !level_out)
    return fail(BFS_ERR_INVALID_ARG, "bfs_run_static: NULL pointer");
  if (source < 0 || source >= n) return fail(BFS_ERR_INVALID_ARG, "bfs_run_static: source outside [0, n)");
  unsigned char* base = nullptr;
  if (int e = scratch_address(&base)) return e;
  cudaStream_t s = (cudaStream_t)stream;
  if (bfsdev::kBoundsCheck) {  // the caller's rows must lie inside [0, nnz) before the kernel trusts them
    int ok = 0;
    if (int e = check_offsets(offsets, n, nnz, reinterpret_cast<int*>(base + kOffSmall + 192), s, &ok)) return e;
    if (!ok) return fail(BFS_ERR_BOUNDS, "bfs_run_static: row offsets are not non-decreasing from 0 to nnz");
  }

  // A graph and a workspace that only point at caller memory and at the scratch.
  bfs_graph g;
  g.n = n;
  g.nnz = nnz;
  g.d_off = const_cast<int64_t*>(offsets);
  g.d_adj = const_cast<int32_t*>(adj);
  g.d_toff = g.d_off;  // undirected: the pull scans the same rows
  g.d_tadj = g.d_adj;
  g.parts = 1;
  Workspace w;
  w.stream = s;
  w.n = n;
  w.nwords = (n + 31) / 32;
  for (int i = 0; i < 3; ++i) {
    w.queue[i] = reinterpret_cast<int32_t*>(base + kOffQueue + i * kQueueBytes);
    w.bits[i] = reinterpret_cast<uint32_t*>(base + kOffBits + i * kBitsBytes);
  }
  w.vis = reinterpret_cast<uint32_t*>(base + kOffVis);
  w.chunks[0] = reinterpret_cast<int64_t*>(base + kOffChunks);
  w.chunks[1] = reinterpret_cast<int64_t*>(base + kOffChunks + kChunkBytes);
  w.chunk_cap = kChunkCap;
  w.ctr = reinterpret_cast<LevelCtr*>(base + kOffCtr);
  w.barrier = base + kOffBarrier;
  w.status = reinterpret_cast<int*>(base + kOffSmall);
  w.misc = reinterpret_cast<int32_t*>(base + kOffSmall + 64);
  w.edges_out = reinterpret_cast<long long*>(base + kOffSmall + 128);

  RunRequest r;
  r.g = &g;
  r.w = &w;
  r.h_sources = &source;
  r.nsources = 1;
  r.level = level_out;
  r.parent = parent_out;
  if (int e = launch_level_loop(r, s)) return e;
  // the status words are read on the caller's stream, so that the call waits
  // for that stream alone and not for other work on the device
  int st[4] = {0, 0, 0, 0};
  BFS_CUDA_TRY(cudaMemcpyAsync(st, w.status, sizeof(st), cudaMemcpyDeviceToHost, s));
  BFS_CUDA_TRY(cudaStreamSynchronize(s));
  if (st[0] != 0) {
    BFS_CUDA_TRY(cudaMemsetAsync(base + kOffBarrier, 0, kBarrierBytes + kSmallBytes, s));
    BFS_CUDA_TRY(cudaStreamSynchronize(s));
    return fail(st[0], "bfs_run_static: " + device_status_message(st));
  }
  return BFS_OK;
}
