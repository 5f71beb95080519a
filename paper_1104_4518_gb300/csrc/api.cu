// C ABI of libbfs_gb300: argument checking, device memory owned by the
// library (graph copies, per-stream workspaces), and the host side of every
// entry point declared in include/bfs.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "device_common.cuh"
#include "internal.h"
#include "nvtx_range.h"

namespace bfsint {

namespace {
thread_local std::string t_last_error;
}

void set_error(const std::string& msg) { t_last_error = msg; }

int fail(int code, const std::string& msg) {
  t_last_error = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  t_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  if (e == cudaErrorMemoryAllocation) return BFS_ERR_OOM;
  if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return BFS_ERR_UNSUPPORTED;
  return BFS_ERR_CUDA;
}

int dev_alloc(void** p, size_t bytes, const char* what) {
  *p = nullptr;
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 1);
  if (e != cudaSuccess) {
    cudaGetLastError();  // clear the sticky-free allocation error
    *p = nullptr;
    return fail(e == cudaErrorMemoryAllocation ? BFS_ERR_OOM : BFS_ERR_CUDA,
                std::string("device allocation of ") + std::to_string(bytes) + " bytes for " + what + " failed: " +
                    cudaGetErrorString(e));
  }
  return BFS_OK;
}

int current_device_info(DeviceInfo* out) {
  static thread_local DeviceInfo cache[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) return fail(BFS_ERR_UNSUPPORTED, "device ordinal out of range");
  if (cache[dev].device != dev) {
    DeviceInfo d;
    d.device = dev;
    BFS_CUDA_TRY(cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev));
    BFS_CUDA_TRY(cudaDeviceGetAttribute(&d.major, cudaDevAttrComputeCapabilityMajor, dev));
    BFS_CUDA_TRY(cudaDeviceGetAttribute(&d.minor, cudaDevAttrComputeCapabilityMinor, dev));
    int l2 = 0;
    BFS_CUDA_TRY(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
    d.l2_bytes = l2;
    int coop = 0;
    BFS_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    if (d.major * 10 + d.minor != 103 || !coop)
      return fail(BFS_ERR_UNSUPPORTED, "libbfs_gb300 is built for sm_103a (GB300) with cooperative launch; device is sm_" +
                                           std::to_string(d.major * 10 + d.minor));
    cache[dev] = d;
  }
  *out = cache[dev];
  return BFS_OK;
}

bfs_tuning effective_tuning(const bfs_graph* g) {
  bfs_tuning t = g->tuning;
  if (t.warp_degree <= 0) t.warp_degree = 32;
  if (t.cta_degree <= 0) t.cta_degree = 256;
  if (t.cta_degree < t.warp_degree) t.cta_degree = t.warp_degree;
  if (t.pull_thread_degree <= 0) t.pull_thread_degree = 4;
  if (t.pull_thread_degree > 4) t.pull_thread_degree = 4;
  if (t.chunk_degree <= 0) t.chunk_degree = 1024;
  if (t.chunk_degree < kChunkEdges) t.chunk_degree = kChunkEdges;
  if (!(t.alpha > 0.0f)) t.alpha = 20.0f;
  if (!(t.beta > 0.0f)) t.beta = 24.0f;
  if (t.batch_topdown_limit <= 0) t.batch_topdown_limit = std::max(1024, g->n / 64);
  if (t.batch_width != 8 && t.batch_width != 16 && t.batch_width != 32 && t.batch_width != 64) t.batch_width = 64;
  if (t.ctas_per_sm < 0 || t.ctas_per_sm > 1) t.ctas_per_sm = 0;  // 0: as many as fit
  return t;
}

void free_workspace(Workspace* w) {
  if (!w) return;
  void* ptrs[] = {w->queue[0], w->queue[1], w->queue[2], w->queue[3], w->bits[0], w->bits[1], w->bits[2],
                  w->bits[3], w->vis, w->chunks[0], w->chunks[1], w->ctr, w->barrier, w->status, w->stats, w->misc,
                  w->edges_out, w->schedule, w->sources, w->tmp_level, w->tmp_parent, w->bset[0], w->bset[1],
                  w->bset[2], w->bvis, w->bscr, w->part_out, w->tmp2_level, w->tmp2_parent};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (w->copy_stream) cudaStreamDestroy(w->copy_stream);
  for (int i = 0; i < 2; ++i) {
    if (w->staged_ev[i]) cudaEventDestroy(w->staged_ev[i]);
    if (w->copied_ev[i]) cudaEventDestroy(w->copied_ev[i]);
  }
  if (w->h_stage) cudaFreeHost(w->h_stage);
  if (w->stage_ev) cudaEventDestroy(w->stage_ev);
  delete w;
}

int get_workspace(bfs_graph* g, cudaStream_t s, Workspace** out) {
  std::lock_guard<std::mutex> lk(g->mu);
  for (Workspace* w : g->ws)
    if (w->stream == s) {
      *out = w;
      return BFS_OK;
    }
  Workspace* w = new Workspace();
  w->stream = s;
  w->n = g->n;
  w->nwords = (g->n + 31) / 32;
  w->chunk_cap = 2 * (g->nnz / kChunkEdges) + kMaxSources + 1024;
  int rc = BFS_OK;
  const size_t nq = sizeof(int32_t) * (size_t)g->n;
  const size_t nb = sizeof(uint32_t) * (size_t)w->nwords;
  for (int i = 0; i < 3 && !rc; ++i) rc = dev_alloc((void**)&w->queue[i], nq, "frontier queue");
  for (int i = 0; i < 3 && !rc; ++i) rc = dev_alloc((void**)&w->bits[i], nb, "frontier bitmap");
  if (!rc) rc = dev_alloc((void**)&w->vis, nb, "visited bitmap");
  for (int i = 0; i < 2 && !rc; ++i) rc = dev_alloc((void**)&w->chunks[i], sizeof(int64_t) * w->chunk_cap, "chunk items");
  if (!rc) rc = dev_alloc((void**)&w->ctr, sizeof(LevelCtr) * kCtrRing, "level counters");
  if (!rc) rc = dev_alloc(&w->barrier, 2 * sizeof(bfsdev::GridBarrier), "grid barriers");
  if (!rc) rc = dev_alloc((void**)&w->status, sizeof(int) * 4, "status");
  if (!rc) rc = dev_alloc((void**)&w->stats, sizeof(bfs_level_stat) * kMaxStatLevels, "level statistics");
  if (!rc) rc = dev_alloc((void**)&w->misc, sizeof(int32_t) * 16, "misc");
  if (!rc) rc = dev_alloc((void**)&w->edges_out, sizeof(long long) * 2, "edge count");
  if (!rc) rc = dev_alloc((void**)&w->schedule, sizeof(int32_t) * kMaxSchedule, "schedule");
  if (!rc) rc = dev_alloc((void**)&w->sources, sizeof(int32_t) * kMaxSources, "sources");
  if (!rc) {
    cudaError_t e = cudaMallocHost((void**)&w->h_stage, sizeof(int32_t) * (kMaxSchedule + kMaxSources));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&w->stage_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) rc = cuda_fail(e, "pinned staging");
  }
  if (!rc) {
    cudaError_t e = cudaMemset(w->barrier, 0, 2 * sizeof(bfsdev::GridBarrier));
    if (e == cudaSuccess) e = cudaMemset(w->status, 0, sizeof(int) * 4);
    if (e == cudaSuccess) e = cudaMemset(w->ctr, 0, sizeof(LevelCtr) * kCtrRing);
    if (e != cudaSuccess) rc = cuda_fail(e, "workspace initialisation");
  }
  if (rc) {
    free_workspace(w);
    return rc;
  }
  g->ws.push_back(w);
  *out = w;
  return BFS_OK;
}

// Staging pair 0 is shared by synchronous host outputs, ragged runs and
// asynchronous host outputs: work that rewrites it on stream s first waits
// until its last asynchronous copy-out has read it.
static int stage0_ready(Workspace* w, cudaStream_t s) {
  if (w->copy_stream) BFS_CUDA_TRY(cudaStreamWaitEvent(s, w->copied_ev[0], 0));
  return BFS_OK;
}

int ensure_tmp_outputs(bfs_graph* g, Workspace* w) {
  if (w->tmp_level) return BFS_OK;
  const size_t nq = sizeof(int32_t) * (size_t)g->n;
  if (int e = dev_alloc((void**)&w->tmp_level, nq, "union-space levels")) return e;
  if (int e = dev_alloc((void**)&w->tmp_parent, nq, "union-space parents")) return e;
  return BFS_OK;
}

int ensure_async_outputs(bfs_graph* g, Workspace* w) {
  if (int e = ensure_tmp_outputs(g, w)) return e;
  if (w->copy_stream) return BFS_OK;
  const size_t nq = sizeof(int32_t) * (size_t)g->n;
  if (int e = dev_alloc((void**)&w->tmp2_level, nq, "second staging levels")) return e;
  if (int e = dev_alloc((void**)&w->tmp2_parent, nq, "second staging parents")) return e;
  for (int i = 0; i < 2; ++i) {
    BFS_CUDA_TRY(cudaEventCreateWithFlags(&w->staged_ev[i], cudaEventDisableTiming));
    BFS_CUDA_TRY(cudaEventCreateWithFlags(&w->copied_ev[i], cudaEventDisableTiming));
  }
  BFS_CUDA_TRY(cudaStreamCreateWithFlags(&w->copy_stream, cudaStreamNonBlocking));
  return BFS_OK;
}

int ensure_batch_state(bfs_graph* g, Workspace* w) {
  if (w->bset[0]) return BFS_OK;
  const size_t n8 = sizeof(uint64_t) * (size_t)g->n;
  for (int i = 0; i < 3; ++i)
    if (int e = dev_alloc((void**)&w->bset[i], n8, "batch frontier bitsets")) return e;
  if (int e = dev_alloc((void**)&w->bvis, n8, "batch visited bitsets")) return e;
  if (int e = dev_alloc((void**)&w->bscr, sizeof(int32_t) * 2 * 64 * (size_t)g->n, "batch scratch results"))
    return e;
  return BFS_OK;
}

int prepare_barrier(Workspace* w, int kind, int grid, cudaStream_t s, bfsdev::GridBarrier** out) {
  bfsdev::GridBarrier* bar = static_cast<bfsdev::GridBarrier*>(w->barrier) + kind;
  if (w->bar_grid[kind] != grid) {
    BFS_CUDA_TRY(cudaMemsetAsync(bar, 0, sizeof(bfsdev::GridBarrier), s));
    w->bar_grid[kind] = grid;
  }
  *out = bar;
  return BFS_OK;
}

int stage_wait(Workspace* w) {
  BFS_CUDA_TRY(cudaEventSynchronize(w->stage_ev));
  return BFS_OK;
}

// Message of a nonzero device status word quad (code, site, 64-bit index).
std::string device_status_message(const int* st) {
  if (st[0] == BFS_ERR_TIMEOUT) return "a device-side wait reached its limit; the traversal was abandoned";
  if (st[0] == BFS_ERR_BOUNDS) {
    static const char* const sites[] = {"?", "top-down adjacency id", "pull adjacency id", "frontier queue slot",
                                        "chunk list slot", "batched top-down adjacency id",
                                        "batched pull adjacency id"};
    long long idx = 0;
    std::memcpy(&idx, st + 2, sizeof(idx));
    const int site = st[1] >= 1 && st[1] <= 6 ? st[1] : 0;
    return std::string("bounds check failed: ") + sites[site] + " " + std::to_string(idx) +
           " outside its range; the traversal was abandoned";
  }
  return "device reported an error";
}

// Reads (and clears) the device status of a workspace; resets the barrier on error.
static int read_status(Workspace* w, cudaStream_t s) {
  int st[4] = {0, 0, 0, 0};
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronisation");
  e = cudaMemcpy(st, w->status, sizeof(st), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "status read");
  if (st[0] != 0) {
    cudaMemset(w->status, 0, sizeof(st));
    cudaMemset(w->barrier, 0, 2 * sizeof(bfsdev::GridBarrier));
    w->bar_grid[0] = w->bar_grid[1] = 0;
    return fail(st[0], device_status_message(st));
  }
  return BFS_OK;
}

void free_half(const bfs_graph* g);  // half_storage.cu: the graph's half storage, if any

static int check_graph(const bfs_graph* g) {
  if (!g) return fail(BFS_ERR_INVALID_ARG, "NULL graph");
  return BFS_OK;
}

// Takes ownership of the out-rows (d_off, d_adj) and, for a directed graph, of
// the in-rows (d_toff, d_tadj; nullptr for an undirected graph).
static int make_graph_from_device_csr(int64_t* d_off, int32_t* d_adj, int32_t n, int64_t nnz, int64_t* d_toff,
                                      int32_t* d_tadj, bfs_graph** out) {
  if (bfsdev::kBoundsCheck) {  // every row inside [0, nnz), so that the kernels only need to check ids
    int* d_flag = nullptr;
    if (int e = dev_alloc((void**)&d_flag, sizeof(int), "offset check flag")) return e;
    int ok = 0, rc = check_offsets(d_off, n, nnz, d_flag, nullptr, &ok);
    if (!rc && ok && d_toff) rc = check_offsets(d_toff, n, nnz, d_flag, nullptr, &ok);
    cudaFree(d_flag);
    if (rc) return rc;
    if (!ok) return fail(BFS_ERR_BOUNDS, "bounds check failed: row offsets are not non-decreasing from 0 to nnz");
  }
  bfs_graph* g = new bfs_graph();
  g->n = n;
  g->nnz = nnz;
  g->d_off = d_off;
  g->d_adj = d_adj;
  g->directed = d_toff != nullptr;
  g->d_toff = g->directed ? d_toff : d_off;
  g->d_tadj = g->directed ? d_tadj : d_adj;
  g->parts = 1;
  g->part_base = {0, (int64_t)n};
  cudaGetDevice(&g->device);
  if (int e = dev_alloc((void**)&g->d_part_base, sizeof(int64_t) * 2, "part table")) {
    delete g;
    return e;
  }
  cudaError_t err = cudaMemcpy(g->d_part_base, g->part_base.data(), sizeof(int64_t) * 2, cudaMemcpyHostToDevice);
  if (err != cudaSuccess) {
    cudaFree(g->d_part_base);
    delete g;
    return cuda_fail(err, "part table copy");
  }
  int rc = dev_alloc((void**)&g->d_dead, sizeof(uint32_t) * (((size_t)n + 31) / 32), "edgeless-vertex bitmap");
  // no arc enters a dead vertex; the big-row chunks serve the batched pull, which scans in-rows
  if (!rc) rc = compute_dead_bits(g->d_toff, n, g->d_dead, nullptr);
  if (!rc) rc = build_big_chunks(g->d_toff, n, nnz, nullptr, &g->d_big, &g->nbig);
  if (!rc) {
    err = cudaDeviceSynchronize();
    if (err != cudaSuccess) rc = cuda_fail(err, "edgeless-vertex bitmap");
  }
  if (rc) {
    if (g->d_dead) cudaFree(g->d_dead);
    if (g->d_big) cudaFree(g->d_big);
    cudaFree(g->d_part_base);
    delete g;
    return rc;
  }
  *out = g;
  return BFS_OK;
}

}  // namespace bfsint

using namespace bfsint;

extern "C" {

const char* bfs_last_error(void) { return t_last_error.c_str(); }

const char* bfs_version(void) {
  return bfsdev::kBoundsCheck ? "bfs_gb300 1.0 (sm_103a, bounds-checking build)" : "bfs_gb300 1.0 (sm_103a)";
}

int bfs_bounds_checked(void) { return bfsdev::kBoundsCheck ? 1 : 0; }

int bfs_graph_create(const int64_t* offsets, const int32_t* adj, int32_t n, int64_t nnz, uint32_t flags,
                     bfs_graph** out) {
  NvtxRange nvtx_range("bfs_graph_create");
  if (!out) return fail(BFS_ERR_INVALID_ARG, "bfs_graph_create: NULL out");
  *out = nullptr;
  if (n < 1 || n >= 2147483647) return fail(BFS_ERR_INVALID_ARG, "bfs_graph_create: n out of range");
  if (nnz < 0 || nnz >= (1ll << 40)) return fail(BFS_ERR_INVALID_ARG, "bfs_graph_create: nnz out of range");
  if (!offsets || (nnz > 0 && !adj)) return fail(BFS_ERR_INVALID_ARG, "bfs_graph_create: NULL array");
  DeviceInfo di;
  if (int e = current_device_info(&di)) return e;
  int64_t* d_off = nullptr;
  int32_t* d_adj = nullptr;
  if (int e = dev_alloc((void**)&d_off, sizeof(int64_t) * ((size_t)n + 1), "CSR offsets")) return e;
  if (int e = dev_alloc((void**)&d_adj, sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1), "CSR adjacency")) {
    cudaFree(d_off);
    return e;
  }
  const cudaMemcpyKind kind = (flags & BFS_HOST_PTRS) ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  cudaError_t err = cudaMemcpy(d_off, offsets, sizeof(int64_t) * ((size_t)n + 1), kind);
  if (err == cudaSuccess && nnz > 0) err = cudaMemcpy(d_adj, adj, sizeof(int32_t) * (size_t)nnz, kind);
  if (err != cudaSuccess) {
    cudaFree(d_off);
    cudaFree(d_adj);
    return cuda_fail(err, "bfs_graph_create: copy");
  }
  const bool directed = (flags & BFS_DIRECTED) != 0;
  if (flags & BFS_VALIDATE) {
    int ok = 0;
    if (int e = validate_csr(d_off, d_adj, n, nnz, !directed, nullptr, &ok)) {
      cudaFree(d_off);
      cudaFree(d_adj);
      return e;
    }
    if (!ok) {
      cudaFree(d_off);
      cudaFree(d_adj);
      return fail(BFS_ERR_INVALID_GRAPH, "bfs_graph_create: CSR failed validation (offsets, ids, order, loops or symmetry)");
    }
  }
  int64_t* d_toff = nullptr;
  int32_t* d_tadj = nullptr;
  if (directed) {
    if (int e = build_transpose(d_off, d_adj, n, nnz, nullptr, &d_toff, &d_tadj)) {
      cudaFree(d_off);
      cudaFree(d_adj);
      return e;
    }
  }
  const int rc = make_graph_from_device_csr(d_off, d_adj, n, nnz, d_toff, d_tadj, out);
  if (rc) {
    cudaFree(d_off);
    cudaFree(d_adj);
    if (d_toff) cudaFree(d_toff);
    if (d_tadj) cudaFree(d_tadj);
  }
  return rc;
}

int bfs_graph_create_from_edges(const int32_t* src, const int32_t* dst, int64_t m, int32_t n, uint32_t flags,
                                void* stream, bfs_graph** out) {
  NvtxRange nvtx_range("bfs_graph_create_from_edges");
  if (!out) return fail(BFS_ERR_INVALID_ARG, "bfs_graph_create_from_edges: NULL out");
  *out = nullptr;
  if (n < 1 || n >= 2147483647) return fail(BFS_ERR_INVALID_ARG, "bfs_graph_create_from_edges: n out of range");
  if (m < 0 || m > (1ll << 38)) return fail(BFS_ERR_INVALID_ARG, "bfs_graph_create_from_edges: m out of range");
  if (m > 0 && (!src || !dst)) return fail(BFS_ERR_INVALID_ARG, "bfs_graph_create_from_edges: NULL array");
  DeviceInfo di;
  if (int e = current_device_info(&di)) return e;
  cudaStream_t s = (cudaStream_t)stream;
  const int32_t* d_src = src;
  const int32_t* d_dst = dst;
  int32_t* tmp = nullptr;
  if ((flags & BFS_HOST_PTRS) && m > 0) {
    if (int e = dev_alloc((void**)&tmp, sizeof(int32_t) * 2 * (size_t)m, "edge list copy")) return e;
    cudaError_t err = cudaMemcpyAsync(tmp, src, sizeof(int32_t) * m, cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess) err = cudaMemcpyAsync(tmp + m, dst, sizeof(int32_t) * m, cudaMemcpyHostToDevice, s);
    if (err != cudaSuccess) {
      cudaFree(tmp);
      return cuda_fail(err, "edge list copy");
    }
    d_src = tmp;
    d_dst = tmp + m;
  }
  int64_t* d_off = nullptr;
  int32_t* d_adj = nullptr;
  int64_t nnz = 0;
  const bool directed = (flags & BFS_DIRECTED) != 0;
  int rc = build_csr_from_edges(d_src, d_dst, m, n, directed ? 1 : 0, s, &d_off, &d_adj, &nnz);
  int64_t* d_toff = nullptr;
  int32_t* d_tadj = nullptr;
  int64_t tnnz = 0;
  if (!rc && directed) {
    rc = build_csr_from_edges(d_src, d_dst, m, n, 2, s, &d_toff, &d_tadj, &tnnz);
    if (rc) {
      cudaFree(d_off);
      cudaFree(d_adj);
    }
  }
  if (tmp) cudaFree(tmp);
  if (rc) return rc;
  rc = make_graph_from_device_csr(d_off, d_adj, n, nnz, d_toff, d_tadj, out);
  if (rc) {
    cudaFree(d_off);
    cudaFree(d_adj);
    if (d_toff) cudaFree(d_toff);
    if (d_tadj) cudaFree(d_tadj);
  }
  return rc;
}

int bfs_graph_union(bfs_graph* const* graphs, int32_t count, void* stream, bfs_graph** out) {
  NvtxRange nvtx_range("bfs_graph_union");
  if (!out || !graphs || count < 1) return fail(BFS_ERR_INVALID_ARG, "bfs_graph_union: bad argument");
  *out = nullptr;
  std::vector<int64_t> base(count + 1, 0);
  int64_t nnz = 0;
  for (int i = 0; i < count; ++i) {
    if (!graphs[i]) return fail(BFS_ERR_INVALID_ARG, "bfs_graph_union: NULL part");
    if (graphs[i]->directed) return fail(BFS_ERR_UNSUPPORTED, "bfs_graph_union: directed parts are not supported");
    base[i + 1] = base[i] + graphs[i]->n;
    nnz += graphs[i]->nnz;
  }
  if (base[count] >= 2147483647) return fail(BFS_ERR_INVALID_ARG, "bfs_graph_union: union too large for int32 ids");
  const int32_t n = (int32_t)base[count];
  cudaStream_t s = (cudaStream_t)stream;
  int64_t* d_off = nullptr;
  int32_t* d_adj = nullptr;
  if (int e = dev_alloc((void**)&d_off, sizeof(int64_t) * ((size_t)n + 1), "union offsets")) return e;
  if (int e = dev_alloc((void**)&d_adj, sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1), "union adjacency")) {
    cudaFree(d_off);
    return e;
  }
  // part i: offsets and ids copied, then shifted on the device
  int64_t nnz_at = 0;
  int rc = BFS_OK;
  for (int i = 0; i < count && !rc; ++i) {
    const bfs_graph* g = graphs[i];
    cudaError_t err = cudaMemcpyAsync(d_off + base[i], g->d_off, sizeof(int64_t) * (size_t)g->n,
                                      cudaMemcpyDeviceToDevice, s);
    if (err == cudaSuccess && g->nnz > 0)
      err = cudaMemcpyAsync(d_adj + nnz_at, g->d_adj, sizeof(int32_t) * (size_t)g->nnz, cudaMemcpyDeviceToDevice, s);
    if (err != cudaSuccess) rc = cuda_fail(err, "union copy");
    if (!rc) rc = union_shift(d_off + base[i], d_adj + nnz_at, g->n, g->nnz, nnz_at, (int32_t)base[i], s);
    nnz_at += g->nnz;
  }
  if (!rc) {
    cudaError_t err = cudaMemcpyAsync(d_off + n, &nnz, sizeof(int64_t), cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) rc = cuda_fail(err, "union finish");
  }
  if (rc) {
    cudaFree(d_off);
    cudaFree(d_adj);
    return rc;
  }
  bfs_graph* u = nullptr;
  if (int e = make_graph_from_device_csr(d_off, d_adj, n, nnz, nullptr, nullptr, &u)) {
    cudaFree(d_off);
    cudaFree(d_adj);
    return e;
  }
  cudaFree(u->d_part_base);
  u->d_part_base = nullptr;
  u->parts = count;
  u->part_base = base;
  if (int e = dev_alloc((void**)&u->d_part_base, sizeof(int64_t) * (count + 1), "part table")) {
    bfs_graph_destroy(u);
    return e;
  }
  cudaError_t err = cudaMemcpy(u->d_part_base, base.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice);
  if (err != cudaSuccess) {
    bfs_graph_destroy(u);
    return cuda_fail(err, "part table copy");
  }
  *out = u;
  return BFS_OK;
}

int bfs_graph_info(const bfs_graph* g, int32_t* n, int64_t* nnz, int32_t* parts) {
  if (int e = check_graph(g)) return e;
  if (n) *n = g->n;
  if (nnz) *nnz = g->nnz;
  if (parts) *parts = g->parts;
  return BFS_OK;
}

int bfs_graph_csr(const bfs_graph* g, const int64_t** offsets, const int32_t** adj) {
  if (int e = check_graph(g)) return e;
  if (offsets) *offsets = g->d_off;
  if (adj) *adj = g->d_adj;
  return BFS_OK;
}

int bfs_graph_copy_csr(const bfs_graph* g, int64_t* offsets_out, int32_t* adj_out, uint32_t flags) {
  if (int e = check_graph(g)) return e;
  if (!offsets_out || (g->nnz > 0 && !adj_out)) return fail(BFS_ERR_INVALID_ARG, "bfs_graph_copy_csr: NULL output");
  const cudaMemcpyKind kind = (flags & BFS_HOST_PTRS) ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  BFS_CUDA_TRY(cudaMemcpy(offsets_out, g->d_off, sizeof(int64_t) * ((size_t)g->n + 1), kind));
  if (g->nnz > 0) BFS_CUDA_TRY(cudaMemcpy(adj_out, g->d_adj, sizeof(int32_t) * (size_t)g->nnz, kind));
  return BFS_OK;
}

void bfs_graph_destroy(bfs_graph* g) {
  if (!g) return;
  cudaDeviceSynchronize();
  for (Workspace* w : g->ws) free_workspace(w);
  g->ws.clear();
  if (g->d_off) cudaFree(g->d_off);
  if (g->d_adj) cudaFree(g->d_adj);
  if (g->directed) {
    cudaFree(g->d_toff);
    cudaFree(g->d_tadj);
  }
  if (g->d_part_base) cudaFree(g->d_part_base);
  if (g->d_dead) cudaFree(g->d_dead);
  if (g->d_big) cudaFree(g->d_big);
  free_tiles(g->tiles);
  free_half(g);
  delete g;
}

int bfs_graph_tiles(bfs_graph* g, int32_t rb_bits, int32_t cb_bits, bfs_tile_info* info, void* stream) {
  NvtxRange nvtx_range("bfs_graph_tiles");
  if (int e = check_graph(g)) return e;
  if (!info) return fail(BFS_ERR_INVALID_ARG, "bfs_graph_tiles: NULL info");
  if ((rb_bits != 0 && (rb_bits < 5 || rb_bits > 16)) || (cb_bits != 0 && (cb_bits < 5 || cb_bits > 16)))
    return fail(BFS_ERR_INVALID_ARG, "bfs_graph_tiles: rb_bits and cb_bits must be 0 or in [5, 16]");
  cudaStream_t s = (cudaStream_t)stream;
  DeviceInfo di;
  if (int e = current_device_info(&di)) return e;
  std::lock_guard<std::mutex> lk(g->mu);
  const int rbb = rb_bits ? rb_bits : default_tile_rb_bits(g->n, di.sm_count);
  const int cbb = cb_bits ? cb_bits : 16;
  if (g->tiles == nullptr || g->tiles->rb_bits != rbb || g->tiles->cb_bits != cbb) {
    BFS_CUDA_TRY(cudaDeviceSynchronize());  // no traversal may still read the old tiles
    TileSet* ts = nullptr;
    if (int e = build_tiles(g, di.sm_count, rbb, cbb, s, &ts)) return e;
    free_tiles(g->tiles);
    g->tiles = ts;
  }
  const TileSet* t = g->tiles;
  info->rb_bits = t->rb_bits;
  info->cb_bits = t->cb_bits;
  info->nrb = t->nrb;
  info->ncb = t->ncb;
  info->ntiles = t->ntiles;
  info->nzc = t->nzc;
  info->nnz = g->nnz;
  info->tdir_jc = t->tdir_jc;
  info->tdir_ir = t->tdir_ir;
  info->jc = t->jc;
  info->cp = t->cp;
  info->ir = t->ir;
  return BFS_OK;
}

static int fill_run_options(const bfs_opts* opts, RunRequest& r) {
  if (!opts) return BFS_OK;
  r.selector = opts->selector;
  r.forced = opts->forced_variant;
  if (r.selector < BFS_SELECT_HEURISTIC || r.selector > BFS_SELECT_SCHEDULE)
    return fail(BFS_ERR_INVALID_ARG, "unknown selector");
  if (r.selector == BFS_SELECT_FORCED && (r.forced < 0 || r.forced >= BFS_NUM_VARIANTS))
    return fail(BFS_ERR_INVALID_ARG, "forced variant out of range");
  if (r.selector == BFS_SELECT_SCHEDULE) {
    if (opts->schedule_len < 0 || (opts->schedule_len > 0 && !opts->schedule))
      return fail(BFS_ERR_INVALID_ARG, "bad schedule");
    for (int i = 0; i < opts->schedule_len; ++i)
      if (opts->schedule[i] < 0 || opts->schedule[i] >= BFS_NUM_VARIANTS)
        return fail(BFS_ERR_INVALID_ARG, "schedule entry out of range");
    r.h_schedule = opts->schedule;
    r.schedule_len = opts->schedule_len;
  }
  r.want_stats = opts->stats != nullptr;
  r.spin_limit = opts->spin_limit;
  return BFS_OK;
}

// Copies the per-level statistics and counts of a finished run to the host.
static int finish_run(Workspace* w, const bfs_opts* opts, cudaStream_t s, int misc_index) {
  if (int e = read_status(w, s)) return e;
  int32_t nl = 0;
  long long edges = 0;
  BFS_CUDA_TRY(cudaMemcpy(&nl, w->misc + misc_index, sizeof(int32_t), cudaMemcpyDeviceToHost));
  BFS_CUDA_TRY(cudaMemcpy(&edges, w->edges_out, sizeof(long long), cudaMemcpyDeviceToHost));
  if (opts->nlevels_out) *opts->nlevels_out = nl;
  if (opts->edges_out) *opts->edges_out = edges;
  if (opts->stats && opts->max_stat_levels > 0) {
    const int cnt = std::min(std::min(nl, opts->max_stat_levels), kMaxStatLevels);
    if (cnt > 0)
      BFS_CUDA_TRY(cudaMemcpy(opts->stats, w->stats, sizeof(bfs_level_stat) * cnt, cudaMemcpyDeviceToHost));
  }
  return BFS_OK;
}

int bfs_run(bfs_graph* g, int32_t source, int32_t* parent_out, int32_t* level_out, const bfs_opts* opts,
            void* stream) {
  NvtxRange nvtx_range("bfs_run");
  if (int e = check_graph(g)) return e;
  if (source < 0 || source >= g->n) return fail(BFS_ERR_INVALID_ARG, "bfs_run: source outside [0, n)");
  if (!parent_out || !level_out) return fail(BFS_ERR_INVALID_ARG, "bfs_run: NULL output");
  cudaStream_t s = (cudaStream_t)stream;
  Workspace* w = nullptr;
  if (int e = get_workspace(g, s, &w)) return e;
  RunRequest r;
  r.g = g;
  r.w = w;
  r.h_sources = &source;
  r.nsources = 1;
  if (int e = fill_run_options(opts, r)) return e;
  const bool host = opts && (opts->flags & BFS_HOST_PTRS);
  const bool async = host && (opts->flags & BFS_HOST_ASYNC);
  int stage = 0;
  if (async) {
    // alternate staging pairs; a pair is rewritten only after its last copy-out
    if (int e = ensure_async_outputs(g, w)) return e;
    stage = w->stage_next;
    w->stage_next ^= 1;
    BFS_CUDA_TRY(cudaStreamWaitEvent(s, w->copied_ev[stage], 0));
    r.level = stage ? w->tmp2_level : w->tmp_level;
    r.parent = stage ? w->tmp2_parent : w->tmp_parent;
  } else if (host) {
    if (int e = ensure_tmp_outputs(g, w)) return e;
    if (int e = stage0_ready(w, s)) return e;
    r.level = w->tmp_level;
    r.parent = w->tmp_parent;
  } else {
    r.level = level_out;
    r.parent = parent_out;
  }
  if (int e = launch_level_loop(r, s)) return e;
  const size_t nb = sizeof(int32_t) * (size_t)g->n;
  if (async) {
    BFS_CUDA_TRY(cudaEventRecord(w->staged_ev[stage], s));
    BFS_CUDA_TRY(cudaStreamWaitEvent(w->copy_stream, w->staged_ev[stage], 0));
    BFS_CUDA_TRY(cudaMemcpyAsync(level_out, r.level, nb, cudaMemcpyDeviceToHost, w->copy_stream));
    BFS_CUDA_TRY(cudaMemcpyAsync(parent_out, r.parent, nb, cudaMemcpyDeviceToHost, w->copy_stream));
    BFS_CUDA_TRY(cudaEventRecord(w->copied_ev[stage], w->copy_stream));
    if (opts->stats || opts->nlevels_out || opts->edges_out) return finish_run(w, opts, s, 0);
    return BFS_OK;
  }
  if (host) {
    BFS_CUDA_TRY(cudaMemcpyAsync(level_out, w->tmp_level, nb, cudaMemcpyDeviceToHost, s));
    BFS_CUDA_TRY(cudaMemcpyAsync(parent_out, w->tmp_parent, nb, cudaMemcpyDeviceToHost, s));
  }
  if (opts && (host || opts->stats || opts->nlevels_out || opts->edges_out)) return finish_run(w, opts, s, 0);
  return BFS_OK;
}

int bfs_run_batch(bfs_graph* g, const int32_t* sources, int32_t k, int32_t* parent_out, int32_t* level_out,
                  const bfs_opts* opts, void* stream) {
  NvtxRange nvtx_range("bfs_run_batch");
  if (int e = check_graph(g)) return e;
  if (!sources || k < 1) return fail(BFS_ERR_INVALID_ARG, "bfs_run_batch: need k >= 1 sources");
  if (!parent_out || !level_out) return fail(BFS_ERR_INVALID_ARG, "bfs_run_batch: NULL output");
  for (int i = 0; i < k; ++i)
    if (sources[i] < 0 || sources[i] >= g->n) return fail(BFS_ERR_INVALID_ARG, "bfs_run_batch: source outside [0, n)");
  cudaStream_t s = (cudaStream_t)stream;
  Workspace* w = nullptr;
  if (int e = get_workspace(g, s, &w)) return e;
  const bool host = opts && (opts->flags & BFS_HOST_PTRS);
  const size_t n = (size_t)g->n;
  int32_t* dl = nullptr;
  int32_t* dp = nullptr;
  if (host) {
    if (int e = dev_alloc((void**)&dl, sizeof(int32_t) * n * 64 * 2, "batch host staging")) return e;
    dp = dl + n * 64;
  }
  int rc = BFS_OK;
  const int width = effective_tuning(g).batch_width;
  for (int c = 0; c < k && !rc; c += width) {
    BatchRequest br;
    br.g = g;
    br.w = w;
    br.h_sources = sources + c;
    br.k = std::min(width, k - c);
    br.width = width;
    br.level = host ? dl : level_out + (size_t)c * n;
    br.parent = host ? dp : parent_out + (size_t)c * n;
    br.spin_limit = opts ? opts->spin_limit : 0;
    br.want_stats = opts && opts->stats && c + width >= k;  // statistics of the last chunk
    rc = launch_batch(br, s);
    if (!rc && host) {
      cudaError_t err = cudaMemcpyAsync(level_out + (size_t)c * n, dl, sizeof(int32_t) * n * br.k,
                                        cudaMemcpyDeviceToHost, s);
      if (err == cudaSuccess)
        err = cudaMemcpyAsync(parent_out + (size_t)c * n, dp, sizeof(int32_t) * n * br.k, cudaMemcpyDeviceToHost, s);
      if (err != cudaSuccess) rc = cuda_fail(err, "batch output copy");
      if (!rc) rc = read_status(w, s);  // staging is reused by the next chunk
    }
  }
  if (dl) {
    cudaStreamSynchronize(s);
    cudaFree(dl);
  }
  if (rc) return rc;
  if (opts && (host || opts->nlevels_out || opts->stats)) {
    if (int e = read_status(w, s)) return e;
    int32_t nl = 0;
    BFS_CUDA_TRY(cudaMemcpy(&nl, w->misc + 1, sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (opts->nlevels_out) *opts->nlevels_out = nl;
    if (opts->stats && opts->max_stat_levels > 0) {
      const int cnt = std::min(std::min(nl, opts->max_stat_levels), kMaxStatLevels);
      if (cnt > 0)
        BFS_CUDA_TRY(cudaMemcpy(opts->stats, w->stats, sizeof(bfs_level_stat) * cnt, cudaMemcpyDeviceToHost));
    }
  }
  return BFS_OK;
}

int bfs_run_ragged(bfs_graph* u, const int32_t* sources, int32_t* const* parent_out, int32_t* const* level_out,
                   const bfs_opts* opts, void* stream) {
  NvtxRange nvtx_range("bfs_run_ragged");
  if (int e = check_graph(u)) return e;
  if (!sources || !parent_out || !level_out) return fail(BFS_ERR_INVALID_ARG, "bfs_run_ragged: NULL argument");
  const int parts = u->parts;
  if (parts > kMaxSources) return fail(BFS_ERR_INVALID_ARG, "bfs_run_ragged: too many parts");
  std::vector<int32_t> usrc(parts);
  std::vector<int32_t*> table(2 * parts);
  for (int i = 0; i < parts; ++i) {
    const int64_t size = u->part_base[i + 1] - u->part_base[i];
    if (sources[i] < 0 || sources[i] >= size)
      return fail(BFS_ERR_INVALID_ARG, "bfs_run_ragged: source outside its part");
    if (!parent_out[i] || !level_out[i]) return fail(BFS_ERR_INVALID_ARG, "bfs_run_ragged: NULL part output");
    usrc[i] = (int32_t)(u->part_base[i] + sources[i]);
    table[i] = level_out[i];
    table[parts + i] = parent_out[i];
  }
  cudaStream_t s = (cudaStream_t)stream;
  Workspace* w = nullptr;
  if (int e = get_workspace(u, s, &w)) return e;
  if (int e = ensure_tmp_outputs(u, w)) return e;
  if (!w->part_out) {
    if (int e = dev_alloc((void**)&w->part_out, sizeof(int32_t*) * 2 * parts, "part output table")) return e;
  }
  // the pointer table changes rarely; it is copied synchronously
  BFS_CUDA_TRY(cudaStreamSynchronize(s));
  BFS_CUDA_TRY(cudaMemcpy(w->part_out, table.data(), sizeof(int32_t*) * 2 * parts, cudaMemcpyHostToDevice));
  RunRequest r;
  r.g = u;
  r.w = w;
  r.h_sources = usrc.data();
  r.nsources = parts;
  if (int e = fill_run_options(opts, r)) return e;
  if (int e = stage0_ready(w, s)) return e;
  r.level = w->tmp_level;
  r.parent = w->tmp_parent;
  r.part_out = w->part_out;
  if (int e = launch_level_loop(r, s)) return e;
  if (opts && (opts->stats || opts->nlevels_out || opts->edges_out)) return finish_run(w, opts, s, 0);
  return BFS_OK;
}

int bfs_sync(bfs_graph* g, void* stream) {
  NvtxRange nvtx_range("bfs_sync");
  if (int e = check_graph(g)) return e;
  cudaStream_t s = (cudaStream_t)stream;
  Workspace* w = nullptr;
  {
    std::lock_guard<std::mutex> lk(g->mu);
    for (Workspace* x : g->ws)
      if (x->stream == s) w = x;
  }
  if (!w) {
    BFS_CUDA_TRY(cudaStreamSynchronize(s));
    return BFS_OK;
  }
  if (w->copy_stream) BFS_CUDA_TRY(cudaStreamSynchronize(w->copy_stream));  // asynchronous host outputs
  return read_status(w, s);
}

int bfs_set_tuning(bfs_graph* g, const bfs_tuning* t) {
  if (int e = check_graph(g)) return e;
  if (!t) return fail(BFS_ERR_INVALID_ARG, "bfs_set_tuning: NULL");
  g->tuning = *t;
  return BFS_OK;
}

int bfs_get_tuning(const bfs_graph* g, bfs_tuning* t) {
  if (int e = check_graph(g)) return e;
  if (!t) return fail(BFS_ERR_INVALID_ARG, "bfs_get_tuning: NULL");
  *t = effective_tuning(g);
  return BFS_OK;
}

int bfs_selector_collect(bfs_graph* g, const int32_t* roots, int32_t nroots, int32_t reps, float* X, float* T,
                         int32_t max_rows, int32_t* rows_out, void* stream) {
  NvtxRange nvtx_range("bfs_selector_collect");
  if (int e = check_graph(g)) return e;
  if (!roots || nroots < 1 || reps < 1 || !X || !T || max_rows < 0 || !rows_out)
    return fail(BFS_ERR_INVALID_ARG, "bfs_selector_collect: bad argument");
  for (int i = 0; i < nroots; ++i)
    if (roots[i] < 0 || roots[i] >= g->n) return fail(BFS_ERR_INVALID_ARG, "bfs_selector_collect: root outside [0, n)");
  const size_t n = (size_t)g->n;
  int32_t* out = nullptr;
  if (int e = dev_alloc((void**)&out, sizeof(int32_t) * n * 2, "collect outputs")) return e;
  std::vector<bfs_level_stat> st(kMaxStatLevels);
  int rows = 0;
  int rc = BFS_OK;
  for (int i = 0; i < nroots && !rc; ++i) {
    // times[v][rep][level]
    std::vector<std::vector<std::vector<double>>> times(BFS_MLP_OUT);  // the network's variants
    std::vector<bfs_level_stat> first;
    int nl = -1;
    for (int v = 0; v < BFS_MLP_OUT && !rc; ++v) {
      for (int rep = 0; rep < reps + 1 && !rc; ++rep) {  // the first run warms up
        bfs_opts o{};
        o.selector = BFS_SELECT_FORCED;
        o.forced_variant = v;
        o.stats = st.data();
        o.max_stat_levels = kMaxStatLevels;
        int32_t levels = 0;
        o.nlevels_out = &levels;
        rc = bfs_run(g, roots[i], out, out + n, &o, stream);
        if (rc) break;
        if (nl < 0) {
          nl = std::min(levels, kMaxStatLevels);
          first.assign(st.begin(), st.begin() + nl);
        }
        if (rep == 0) continue;
        std::vector<double> t(nl);
        for (int k = 0; k < nl; ++k) t[k] = (double)st[k].time_ns;
        times[v].push_back(t);
      }
    }
    if (rc) break;
    for (int k = 0; k < nl && rows < max_rows; ++k, ++rows) {
      const bfs_level_stat& s = first[k];
      const int64_t bins[3] = {s.bin_count[0], s.bin_count[1], s.bin_count[2]};
      bfs_level_features(g->n, g->nnz, k, s.frontier_count, s.frontier_edges, s.unvisited_count, s.unvisited_edges,
                         bins, X + (size_t)rows * BFS_MLP_IN);
      for (int v = 0; v < BFS_MLP_OUT; ++v) {
        std::vector<double> samples;
        for (auto& run : times[v]) samples.push_back(run[k]);
        std::sort(samples.begin(), samples.end());
        const double med = samples[samples.size() / 2];
        T[(size_t)rows * BFS_MLP_OUT + v] = (float)std::log2(std::max(med, 1.0) / 1000.0);
      }
    }
  }
  cudaStreamSynchronize((cudaStream_t)stream);
  cudaFree(out);
  if (rc) return rc;
  *rows_out = rows;
  return BFS_OK;
}

int bfs_autotune(bfs_graph* g, const int32_t* roots, int32_t nroots, bfs_tuning* best, void* stream) {
  NvtxRange nvtx_range("bfs_autotune");
  if (int e = check_graph(g)) return e;
  if (!roots || nroots < 1) return fail(BFS_ERR_INVALID_ARG, "bfs_autotune: need roots");
  for (int i = 0; i < nroots; ++i)
    if (roots[i] < 0 || roots[i] >= g->n) return fail(BFS_ERR_INVALID_ARG, "bfs_autotune: root outside [0, n)");
  cudaStream_t s = (cudaStream_t)stream;
  int32_t* out = nullptr;
  const size_t n = (size_t)g->n;
  const int kb = std::min(nroots, 64);
  if (int e = dev_alloc((void**)&out, sizeof(int32_t) * n * 2 * kb, "autotune outputs")) return e;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const bfs_tuning saved = g->tuning;
  int rc = BFS_OK;
  // time of the plain traversal over all roots (ms) under tuning t
  auto time_plain = [&](const bfs_tuning& t, float* ms) -> int {
    g->tuning = t;
    for (int rep = 0; rep < 2; ++rep) {  // first pass warms up
      cudaEventRecord(e0, s);
      for (int i = 0; i < nroots; ++i)
        if (int e = bfs_run(g, roots[i], out, out + n, nullptr, stream)) return e;
      cudaEventRecord(e1, s);
      if (int e = bfs_sync(g, stream)) return e;
    }
    cudaEventElapsedTime(ms, e0, e1);
    return BFS_OK;
  };
  auto time_batch = [&](const bfs_tuning& t, float* ms) -> int {
    g->tuning = t;
    for (int rep = 0; rep < 2; ++rep) {
      cudaEventRecord(e0, s);
      if (int e = bfs_run_batch(g, roots, kb, out, out + n * kb, nullptr, stream)) return e;
      cudaEventRecord(e1, s);
      if (int e = bfs_sync(g, stream)) return e;
    }
    cudaEventElapsedTime(ms, e0, e1);
    return BFS_OK;
  };
  bfs_tuning cur = effective_tuning(g);
  float cur_ms = 0.0f;
  rc = time_plain(cur, &cur_ms);
  // coordinate descent over one knob at a time, two sweeps
  for (int sweep = 0; sweep < 2 && !rc; ++sweep) {
    const int wd[] = {8, 16, 32, 64};
    const int cd[] = {128, 256, 1024};
    const int pd[] = {1, 2, 3, 4};
    const int ch[] = {1024, 2048, 4096};
    const float al[] = {10.0f, 14.0f, 20.0f, 30.0f, 45.0f};
    const float be[] = {8.0f, 16.0f, 24.0f, 48.0f, 96.0f};
    const int sf[] = {-1, 0, 2 * 4864, 4 * 4864};
    const int ne[] = {-1, 4096, 16384, 65536};
    const int cs[] = {0, 1};
    for (int knob = 0; knob < 9 && !rc; ++knob) {
      const int cnt = knob == 0 ? 4 : knob == 1 ? 3 : knob == 2 ? 4 : knob == 3 ? 3 : knob == 8 ? 2 : knob >= 6 ? 4 : 5;
      for (int c = 0; c < cnt && !rc; ++c) {
        bfs_tuning t = cur;
        switch (knob) {
          case 0: t.warp_degree = wd[c]; break;
          case 1: t.cta_degree = cd[c]; break;
          case 2: t.pull_thread_degree = pd[c]; break;
          case 3: t.chunk_degree = ch[c]; break;
          case 4: t.alpha = al[c]; break;
          case 5: t.beta = be[c]; break;
          case 6: t.small_frontier = sf[c]; break;
          case 7: t.narrow_edges = ne[c]; break;
          default: t.ctas_per_sm = cs[c]; break;
        }
        float ms = 0.0f;
        rc = time_plain(t, &ms);
        if (!rc && ms < 0.97f * cur_ms) {  // a change must beat the timing noise of a few roots
          cur_ms = ms;
          cur = t;
        }
      }
    }
  }
  if (!rc) {  // batched: the top-down / pull switch of the bitset traversal
    float bms = 0.0f;
    rc = time_batch(cur, &bms);
    const double fr[] = {1.0 / 1024, 1.0 / 256, 1.0 / 64, 1.0 / 16, 1.0 / 4};
    for (int c = 0; c < 5 && !rc; ++c) {
      bfs_tuning t = cur;
      t.batch_topdown_limit = std::max(1, (int)(g->n * fr[c]));
      float ms = 0.0f;
      rc = time_batch(t, &ms);
      if (!rc && ms < 0.97f * bms) {
        bms = ms;
        cur = t;
      }
    }
    for (int wbits = 8; wbits <= 64 && kb == 64 && !rc; wbits *= 2) {  // roots per traversal (64 roots timed)
      bfs_tuning t = cur;
      t.batch_width = wbits;
      float ms = 0.0f;
      rc = time_batch(t, &ms);
      if (!rc && ms < 0.97f * bms) {
        bms = ms;
        cur = t;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  cudaFree(out);
  if (rc) {
    g->tuning = saved;
    return rc;
  }
  g->tuning = cur;
  if (best) *best = cur;
  return BFS_OK;
}

}  // extern "C"
