// Hypersparse 2D tiles of the in-adjacency, built on the device from the CSR.
//
// Sec. 3.2 splits the adjacency matrix into a 2D grid of blocks, and Sec. 4.1
// stores each block in doubly compressed sparse column form (DCSC: the row ids
// IR of the non-zeros, indexed by the parallel arrays JC of non-empty column
// ids and CP of column pointers), because blocks of a 2D split are hypersparse
// and a CSR per block would cost O(n sqrt(p) + m) memory.  On one GPU the
// blocks are tiles that the tiled pull variant walks with a tile-local slice
// of the frontier and of the row state in shared memory.
//
// Here a row is a vertex v that a pull level may reach and a column is a
// candidate parent u (the entries of v's in-row), so tile (rb, cb) holds the
// entries with v >> rb_bits == rb and u >> cb_bits == cb.  Local ids fit in
// 16 bits, so jc and ir are uint16 and cp is relative to the tile's first
// entry.  Construction: one 64-bit key per entry (tile, local column, local
// row), emitted in CSR order; a stable radix sort on the tile and column bits
// (the rows of one column are already ascending in CSR order); column starts
// flagged and scanned; the tile directory filled at tile boundaries.
#include <algorithm>
#include <mutex>
#include <string>

#include "device_common.cuh"
#include "internal.h"

namespace bfsint {
namespace {

constexpr int kTileThreads = 256;

// Key of entry j = (v, u) of v's in-row: tile id << 32 | local column << 16 | local row.
// An id u outside [0, n) (a malformed graph) gets no key: the first one is
// recorded in bad[0] (flag) and bad[1] (the id), and the build stops before
// any tile id is used as an index.
__global__ void tile_keys_kernel(const int64_t* __restrict__ off, const int32_t* __restrict__ adj, int32_t n,
                                 int rb_bits, int cb_bits, int32_t ncb, uint64_t* __restrict__ keys,
                                 long long* __restrict__ bad) {
  const int lane = threadIdx.x & 31;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const uint32_t cmask = (1u << cb_bits) - 1u;
  for (long long v = gw; v < n; v += nw) {
    const long long b = off[v], e = off[v + 1];
    const uint64_t rb = (uint64_t)(v >> rb_bits);
    const uint64_t vl = (uint64_t)(v & ((1ll << rb_bits) - 1));
    for (long long j = b + lane; j < e; j += 32) {
      const int32_t a = adj[j];
      if (a < 0 || a >= n) {
        if (atomicCAS(reinterpret_cast<unsigned long long*>(bad), 0ull, 1ull) == 0ull) bad[1] = a;
        keys[j] = ~0ull;
        continue;
      }
      const uint32_t u = (uint32_t)a;
      const uint64_t t = rb * (uint64_t)ncb + (u >> cb_bits);
      keys[j] = (t << 32) | ((uint64_t)(u & cmask) << 16) | vl;
    }
  }
}

// 1 where sorted key i starts a column of a tile (its tile or its column differs from key i - 1).
__global__ void col_flags_kernel(const uint64_t* __restrict__ keys, long long N, uint32_t* __restrict__ flags) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride)
    flags[i] = (i == 0 || (keys[i] >> 16) != (keys[i - 1] >> 16)) ? 1u : 0u;
}

// Tile directory: at every tile boundary the key's thread fills the entries of
// the tiles from the previous key's tile (exclusive) to its own (inclusive),
// so empty tiles get empty ranges; the last key also fills the tiles after it.
__global__ void tile_bounds_kernel(const uint64_t* __restrict__ keys, long long N, const int64_t* __restrict__ colpos,
                                   long long nzc, long long T, int64_t* __restrict__ tdir_jc,
                                   int64_t* __restrict__ tdir_ir) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
    const long long t = (long long)(keys[i] >> 32);
    const long long tp = i == 0 ? -1 : (long long)(keys[i - 1] >> 32);
    for (long long q = tp + 1; q <= t; ++q) {
      tdir_ir[q] = i;
      tdir_jc[q] = colpos[i];
    }
    if (i == N - 1)
      for (long long q = t + 1; q <= T; ++q) {
        tdir_ir[q] = N;
        tdir_jc[q] = nzc;
      }
  }
}

__global__ void tile_emit_kernel(const uint64_t* __restrict__ keys, long long N, const uint32_t* __restrict__ flags,
                                 const int64_t* __restrict__ colpos, const int64_t* __restrict__ tdir_ir,
                                 uint16_t* __restrict__ ir, uint16_t* __restrict__ jc, uint32_t* __restrict__ cp) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
    const uint64_t k = keys[i];
    ir[i] = (uint16_t)(k & 0xffffu);
    if (flags[i]) {
      const long long c = colpos[i];
      jc[c] = (uint16_t)((k >> 16) & 0xffffu);
      cp[c] = (uint32_t)(i - tdir_ir[k >> 32]);
    }
  }
}

__global__ void fill_i64_kernel(int64_t* a, long long count, long long value) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) a[i] = value;
}

int ceil_log2(long long x) {
  int b = 0;
  while (b < 62 && (1ll << b) < x) ++b;
  return b;
}

}  // namespace

void free_tiles(TileSet* t) {
  if (!t) return;
  cudaFree(t->jc);
  cudaFree(t->cp);
  cudaFree(t->ir);
  cudaFree(t->tdir_jc);
  cudaFree(t->tdir_ir);
  delete t;
}

int default_tile_rb_bits(int32_t n, int sm_count) {
  // about two row blocks per CTA of a two-CTA-per-SM grid, between 2^8 and 2^16 rows
  return std::min(16, std::max(8, ceil_log2((long long)n / (4ll * std::max(sm_count, 1)))));
}

int build_tiles(const bfs_graph* g, int sm_count, int rb_bits, int cb_bits, cudaStream_t s, TileSet** out) {
  const int32_t n = g->n;
  const long long N = g->nnz;
  TileSet* ts = new TileSet();
  ts->rb_bits = rb_bits > 0 ? rb_bits : default_tile_rb_bits(n, sm_count);
  ts->cb_bits = cb_bits > 0 ? cb_bits : 16;
  ts->nrb = (int32_t)(((long long)n + (1ll << ts->rb_bits) - 1) >> ts->rb_bits);
  ts->ncb = (int32_t)(((long long)n + (1ll << ts->cb_bits) - 1) >> ts->cb_bits);
  ts->ntiles = (long long)ts->nrb * ts->ncb;
  const long long T = ts->ntiles;
  uint64_t* keys = nullptr;
  uint64_t* alt = nullptr;
  uint32_t* flags = nullptr;
  int64_t* colpos = nullptr;
  auto fail_clean = [&](int rc) {
    cudaFree(keys);
    cudaFree(alt);
    cudaFree(flags);
    cudaFree(colpos);
    free_tiles(ts);
    return rc;
  };
  int rc = BFS_OK;
  if ((rc = dev_alloc((void**)&ts->tdir_jc, sizeof(int64_t) * (T + 1), "tile directory"))) return fail_clean(rc);
  if ((rc = dev_alloc((void**)&ts->tdir_ir, sizeof(int64_t) * (T + 1), "tile directory"))) return fail_clean(rc);
  if ((rc = dev_alloc((void**)&ts->ir, sizeof(uint16_t) * (N > 0 ? N : 1), "tile rows"))) return fail_clean(rc);
  const int grid = std::max(sm_count, 1) * 8;
  if (N == 0) {
    if ((rc = dev_alloc((void**)&ts->jc, sizeof(uint16_t), "tile columns"))) return fail_clean(rc);
    if ((rc = dev_alloc((void**)&ts->cp, sizeof(uint32_t), "tile column pointers"))) return fail_clean(rc);
    fill_i64_kernel<<<grid, kTileThreads, 0, s>>>(ts->tdir_jc, T + 1, 0);
    fill_i64_kernel<<<grid, kTileThreads, 0, s>>>(ts->tdir_ir, T + 1, 0);
  } else {
    if ((rc = dev_alloc((void**)&keys, sizeof(uint64_t) * N, "tile keys"))) return fail_clean(rc);
    if ((rc = dev_alloc((void**)&alt, sizeof(uint64_t) * N, "tile keys (alternate)"))) return fail_clean(rc);
    long long* d_bad = nullptr;
    if ((rc = dev_alloc((void**)&d_bad, 2 * sizeof(long long), "tile check flag"))) return fail_clean(rc);
    long long h_bad[2] = {0, 0};
    cudaError_t e0 = cudaMemsetAsync(d_bad, 0, 2 * sizeof(long long), s);
    if (e0 == cudaSuccess) {
      tile_keys_kernel<<<grid, kTileThreads, 0, s>>>(g->d_toff, g->d_tadj, n, ts->rb_bits, ts->cb_bits, ts->ncb, keys,
                                                     d_bad);
      e0 = cudaGetLastError();
    }
    if (e0 == cudaSuccess) e0 = cudaMemcpyAsync(h_bad, d_bad, sizeof(h_bad), cudaMemcpyDeviceToHost, s);
    if (e0 == cudaSuccess) e0 = cudaStreamSynchronize(s);
    cudaFree(d_bad);
    if (e0 != cudaSuccess) return fail_clean(cuda_fail(e0, "tile keys"));
    if (h_bad[0])
      return fail_clean(fail(bfsdev::kBoundsCheck ? BFS_ERR_BOUNDS : BFS_ERR_INVALID_GRAPH,
                             "bounds check failed: tile adjacency id " + std::to_string(h_bad[1]) +
                                 " outside [0, n) while building the 2D tiles"));
    uint64_t* sorted = nullptr;
    if ((rc = radix_sort_u64(keys, alt, N, 16, 32 + std::max(1, ceil_log2(T)), s, &sorted))) return fail_clean(rc);
    if (sorted == keys) {
      cudaFree(alt);
    } else {
      cudaFree(keys);
      keys = alt;
    }
    alt = nullptr;
    if ((rc = dev_alloc((void**)&flags, sizeof(uint32_t) * N, "tile column flags"))) return fail_clean(rc);
    if ((rc = dev_alloc((void**)&colpos, sizeof(int64_t) * N, "tile column positions"))) return fail_clean(rc);
    col_flags_kernel<<<grid, kTileThreads, 0, s>>>(keys, N, flags);
    long long nzc = 0;
    if ((rc = exclusive_scan_u32(flags, N, colpos, s, &nzc))) return fail_clean(rc);
    ts->nzc = nzc;
    if ((rc = dev_alloc((void**)&ts->jc, sizeof(uint16_t) * nzc, "tile columns"))) return fail_clean(rc);
    if ((rc = dev_alloc((void**)&ts->cp, sizeof(uint32_t) * nzc, "tile column pointers"))) return fail_clean(rc);
    tile_bounds_kernel<<<grid, kTileThreads, 0, s>>>(keys, N, colpos, nzc, T, ts->tdir_jc, ts->tdir_ir);
    tile_emit_kernel<<<grid, kTileThreads, 0, s>>>(keys, N, flags, colpos, ts->tdir_ir, ts->ir, ts->jc, ts->cp);
  }
  cudaError_t err = cudaGetLastError();
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  cudaFree(keys);
  cudaFree(flags);
  cudaFree(colpos);
  keys = nullptr;
  flags = nullptr;
  colpos = nullptr;
  if (err != cudaSuccess) return fail_clean(cuda_fail(err, "tile construction"));
  *out = ts;
  return BFS_OK;
}

int ensure_tiles(bfs_graph* g, cudaStream_t s, TileSet** out) {
  std::lock_guard<std::mutex> lk(g->mu);
  if (g->tiles == nullptr) {
    DeviceInfo di;
    if (int e = current_device_info(&di)) return e;
    TileSet* ts = nullptr;
    if (int e = build_tiles(g, di.sm_count, 0, 0, s, &ts)) return e;
    g->tiles = ts;
  }
  *out = g->tiles;
  return BFS_OK;
}

}  // namespace bfsint
