// Host-side internals of libbfs_gb300 shared by its translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "bfs.h"

namespace bfsdev {
struct GridBarrier;
}

namespace bfsint {

// ---------------- error reporting ----------------
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define BFS_CUDA_TRY(expr)                                  \
  do {                                                      \
    cudaError_t _e = (expr);                                \
    if (_e != cudaSuccess) return bfsint::cuda_fail(_e, #expr); \
  } while (0)

// Device allocation that reports OOM as BFS_ERR_OOM.
int dev_alloc(void** p, size_t bytes, const char* what);

// ---------------- device properties ----------------
struct DeviceInfo {
  int device = -1;
  int sm_count = 0;
  int major = 0, minor = 0;
  long long l2_bytes = 0;
};
int current_device_info(DeviceInfo* out);

// ---------------- level counters (device) ----------------
// One slot per level in a ring of kCtrRing: filled while the frontier of that
// level is built, read after the grid barrier that ends the phase.
constexpr int kCtrRing = 8;
struct __align__(64) LevelCtr {
  unsigned int count;             // frontier vertices (also the queue tail)
  unsigned int chunks;            // chunk items of high-degree frontier vertices
  unsigned long long edges;       // degree sum of the frontier
  unsigned long long bins[3];     // degree <= 32, <= 1024, larger
  unsigned long long pad;          // the level's cursor of dynamically handed-out pull chunks / chunk items
};

// Edges per chunk item of a high-degree top-down vertex (one CTA pass).
constexpr int kChunkEdges = 1024;

// Device stats record written by the level loop (mirrors bfs_level_stat).
static_assert(sizeof(bfs_level_stat) == 72, "bfs_level_stat layout");

// ---------------- workspace of single / multi-source runs ----------------
struct Workspace {
  cudaStream_t stream = nullptr;
  int32_t n = 0;
  int32_t nwords = 0;
  int32_t* queue[4] = {nullptr, nullptr, nullptr, nullptr};
  uint32_t* bits[4] = {nullptr, nullptr, nullptr, nullptr};
  uint32_t* vis = nullptr;
  int64_t* chunks[2] = {nullptr, nullptr};
  int64_t chunk_cap = 0;
  LevelCtr* ctr = nullptr;
  void* barrier = nullptr;  // bfsdev::GridBarrier[2]: level loop, batched kernel
  int bar_grid[2] = {0, 0};  // grid size of each kernel's last launch (host side)
  int* status = nullptr;
  bfs_level_stat* stats = nullptr;  // device, kMaxStatLevels
  int32_t* misc = nullptr;          // [0] level count, [1..] spare
  long long* edges_out = nullptr;   // device TEPS edge count
  int32_t* schedule = nullptr;      // device, kMaxSchedule
  int32_t* sources = nullptr;       // device, up to kMaxSources
  int32_t* tmp_level = nullptr;     // union-space outputs (ragged / host outputs), lazily
  int32_t* tmp_parent = nullptr;
  // asynchronous host outputs: a second staging pair, the copy stream, and per
  // staging pair the events "traversal written" and "copied out"
  int32_t* tmp2_level = nullptr;
  int32_t* tmp2_parent = nullptr;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t staged_ev[2] = {nullptr, nullptr};
  cudaEvent_t copied_ev[2] = {nullptr, nullptr};
  int stage_next = 0;
  // batched (64-root bitset) state, lazily
  uint64_t* bset[3] = {nullptr, nullptr, nullptr};
  uint64_t* bvis = nullptr;
  int32_t* bscr = nullptr;  // batched: vertex-major scratch results, levels then parents, int32[2][n][64]
  // pinned host staging for schedules and multi-source seeds; `stage_ev` is
  // recorded after each copy out of it and waited on before it is rewritten
  int32_t* h_stage = nullptr;
  cudaEvent_t stage_ev = nullptr;
  // ragged output pointer tables
  int32_t** part_out = nullptr;
  // scratch for bfs_graph_union / misc
};

constexpr int kMaxStatLevels = 8192;
constexpr int kMaxSchedule = 8192;
constexpr int kMaxSources = 4096;

}  // namespace bfsint

namespace bfsint {
// Hypersparse 2D tiles of the in-adjacency (rows = the vertices a pull level
// reaches, columns = their candidate parents), in the doubly compressed
// sparse column form of Sec. 4.1: rows are split into blocks of 2^rb_bits
// vertices and columns into blocks of 2^cb_bits; tile t = rb * ncb + cb holds
// the entries (v, u) with v in row block rb and u in column block cb.  Within
// a tile, jc lists the tile-local ids of the non-empty columns (ascending), cp
// the start of each column's rows relative to the tile's first entry, and ir
// the tile-local row ids (ascending within a column).  tdir_jc[t] / tdir_ir[t]
// give tile t's first column / first entry (T + 1 entries each).
struct TileSet {
  int rb_bits = 0, cb_bits = 0;
  int32_t nrb = 0, ncb = 0;
  int64_t ntiles = 0, nzc = 0;
  uint16_t* jc = nullptr;
  uint32_t* cp = nullptr;
  uint16_t* ir = nullptr;
  int64_t* tdir_jc = nullptr;
  int64_t* tdir_ir = nullptr;
};
}  // namespace bfsint

struct bfs_graph {
  int32_t n = 0;
  int64_t nnz = 0;
  int64_t* d_off = nullptr;   // rows of out-neighbours (all neighbours when undirected)
  int32_t* d_adj = nullptr;
  bool directed = false;
  int64_t* d_toff = nullptr;  // rows of in-neighbours: the transpose when directed, else d_off
  int32_t* d_tadj = nullptr;
  uint32_t* d_dead = nullptr;  // bitmap of vertices no arc enters (tail bits set)
  int64_t* d_big = nullptr;    // (v << 32 | c) for every kChunkEdges-entry chunk c of rows longer than kChunkEdges
  int64_t nbig = 0;
  int32_t parts = 1;
  std::vector<int64_t> part_base;  // parts + 1 entries (union graphs)
  int64_t* d_part_base = nullptr;
  bfs_tuning tuning{};
  bfsint::TileSet* tiles = nullptr;  // built on the first run that may use the tiled variant
  int device = 0;
  std::mutex mu;
  std::vector<bfsint::Workspace*> ws;
};

namespace bfsint {

// Waits until the pinned staging buffer of w may be rewritten.
int stage_wait(Workspace* w);
// Workspace of (g, stream), created on first use.
int get_workspace(bfs_graph* g, cudaStream_t s, Workspace** out);
void free_workspace(Workspace* w);
int ensure_batch_state(bfs_graph* g, Workspace* w);
int ensure_tmp_outputs(bfs_graph* g, Workspace* w);
int ensure_async_outputs(bfs_graph* g, Workspace* w);

// Effective tuning with defaults filled in.
bfs_tuning effective_tuning(const bfs_graph* g);

// ---------------- kernels (launchers) ----------------
// CSR construction from an edge list (device pointers).  Allocates d_off/d_adj.
// mode 0: undirected (both arcs of every edge), 1: arcs src -> dst, 2: arcs dst -> src.
int build_csr_from_edges(const int32_t* d_src, const int32_t* d_dst, int64_t m, int32_t n, int mode,
                         cudaStream_t s, int64_t** d_off, int32_t** d_adj, int64_t* nnz);
// Stable least-significant-digit radix sort of N 64-bit keys on bits
// [lo_bit, hi_bit), 8 bits per pass; alt is scratch of N keys; *sorted is
// whichever of the two buffers holds the result.  Synchronises s.
int radix_sort_u64(uint64_t* keys, uint64_t* alt, long long N, int lo_bit, int hi_bit, cudaStream_t s,
                   uint64_t** sorted);
// Exclusive prefix sum of N uint32 values into int64 out; *total receives the sum.
int exclusive_scan_u32(const uint32_t* in, long long N, int64_t* out, cudaStream_t s, long long* total);
// The 2D tiles of g's in-adjacency (see TileSet) with 2^rb_bits rows and
// 2^cb_bits columns per tile (0: the defaults); synchronises s.
int default_tile_rb_bits(int32_t n, int sm_count);
int build_tiles(const bfs_graph* g, int sm_count, int rb_bits, int cb_bits, cudaStream_t s, TileSet** out);
// g's tiles, built with the default layout if g has none (under g's lock).
int ensure_tiles(bfs_graph* g, cudaStream_t s, TileSet** out);
void free_tiles(TileSet* t);
// Message of a nonzero device status (status[0] code, [1] site, [2..3] index).
std::string device_status_message(const int* status4);
// Row offsets non-decreasing from 0 to nnz?  d_flag: one device int of scratch.
// Synchronises s.
int check_offsets(const int64_t* d_off, int32_t n, int64_t nnz, int* d_flag, cudaStream_t s, int* ok);
// The transpose of a directed CSR (row v lists the tails u of the arcs u -> v).
int build_transpose(const int64_t* d_off, const int32_t* d_adj, int32_t n, int64_t nnz, cudaStream_t s,
                    int64_t** d_toff, int32_t** d_tadj);
// Bitmap of the vertices without edges (bits beyond n set), one word per 32 vertices.
int compute_dead_bits(const int64_t* d_off, int32_t n, uint32_t* d_dead, cudaStream_t s);
// Chunk items of every row longer than kChunkEdges (order unspecified); *count receives their number.
int build_big_chunks(const int64_t* d_off, int32_t n, int64_t nnz, cudaStream_t s, int64_t** items, int64_t* count);
// Adds off_shift to n_part offsets and id_shift to nnz_part ids (union building).
int union_shift(int64_t* off, int32_t* adj, int64_t n_part, int64_t nnz_part, int64_t off_shift, int32_t id_shift,
                cudaStream_t s);
// CSR validation on the device; *ok = 1 when valid.
int validate_csr(const int64_t* d_off, const int32_t* d_adj, int32_t n, int64_t nnz, bool symmetric, cudaStream_t s,
                 int* ok);

struct RunRequest {
  bfs_graph* g = nullptr;
  Workspace* w = nullptr;
  const int32_t* h_sources = nullptr;  // host, union ids
  int32_t nsources = 0;
  int32_t* level = nullptr;   // device outputs (union space)
  int32_t* parent = nullptr;
  int32_t selector = BFS_SELECT_HEURISTIC;
  int32_t forced = 0;
  const int32_t* h_schedule = nullptr;
  int32_t schedule_len = 0;
  bool want_stats = false;
  unsigned spin_limit = 0;
  // ragged: scatter union outputs into per-part outputs (device table of 2*parts pointers)
  int32_t** part_out = nullptr;
  // the graph's 2D tiles when a level may take the tiled variant (else the variant runs untiled)
  const TileSet* tiles = nullptr;
};
// The grid barrier of kernel `kind` (0: level loop, 1: batched) in w, zeroed
// on the stream first when that kernel's grid size differs from its last launch.
int prepare_barrier(Workspace* w, int kind, int grid, cudaStream_t s, bfsdev::GridBarrier** out);
int launch_level_loop(const RunRequest& r, cudaStream_t s);

struct BatchRequest {
  bfs_graph* g = nullptr;
  Workspace* w = nullptr;
  const int32_t* h_sources = nullptr;  // up to 64
  int32_t k = 0;              // roots, at most width
  int32_t width = 64;         // bits per frontier word: 8, 16, 32 or 64
  int32_t* level = nullptr;   // device [k][n]
  int32_t* parent = nullptr;
  unsigned spin_limit = 0;
  bool want_stats = false;
};
int launch_batch(const BatchRequest& r, cudaStream_t s);

// Selector network parameters on the current device (nullptr if none).
// The selector features' constants of a graph, float32: log2 n / 32,
// log2 nnz / 32, 1 / n, 1 / nnz (n and nnz taken as at least 1).
void graph_feature_constants(int32_t n, int64_t nnz, float* log_n, float* log_nnz, float* inv_n, float* inv_nnz);
const float* learned_params_device();

}  // namespace bfsint
