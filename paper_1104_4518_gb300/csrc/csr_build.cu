// Edge list -> symmetric, deduplicated, row-sorted CSR on the device, and the
// CSR validation used by bfs_graph_create(BFS_VALIDATE).
//
// The paper stores each undirected edge in both rows with every row sorted
// (Sec. 4.1) and its benchmark symmetrises the generated edges (Sec. 6).  Here:
//   1. every non-loop edge (u, v) emits the keys (u << b) | v and (v << b) | u,
//      b = bits of n - 1 (warp-aggregated append);
//   2. the keys are sorted by a least-significant-digit radix sort over their
//      2b significant bits, 8 bits per pass; each pass is a tile histogram, an
//      exclusive scan of the digit-major histogram and a stable scatter whose
//      in-tile ranks come from __match_any_sync on the digit;
//   3. a key equal to its predecessor is a repeat; an exclusive scan of the
//      "first of its value" flags gives every kept key its slot, the low b
//      bits are the column, and the row changes between consecutive kept keys
//      give the int64 row offsets.
#include <cstdio>

#include "device_common.cuh"
#include "internal.h"

namespace bfsint {
namespace {

using bfsdev::kFull;

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kKeysPerThread = 16;
constexpr int kTile = kSortThreads * kKeysPerThread;  // 4096 keys
constexpr int kRadix = 256;

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// ---------------- key emission ----------------
// Keys of the arcs of edge e = (u, v): mode 0 (undirected) emits u -> v and
// v -> u, mode 1 u -> v only, mode 2 v -> u only (the transpose).
__global__ void make_keys_kernel(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t m,
                                 int32_t n, int vbits, int mode, uint64_t* __restrict__ keys,
                                 unsigned long long* __restrict__ count, int* __restrict__ bad) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long mr = (m + 31) / 32 * 32;
  const int lane = threadIdx.x & 31;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < mr; e += stride) {
    int u = 0, v = 0;
    bool ok = false;
    if (e < m) {
      u = src[e];
      v = dst[e];
      if (u < 0 || u >= n || v < 0 || v >= n) atomicExch(bad, 1);
      else ok = (u != v);
    }
    const unsigned bm = __ballot_sync(kFull, ok);
    if (!bm) continue;
    const unsigned long long per = mode == 0 ? 2ull : 1ull;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(count, per * __popc(bm));
    base = __shfl_sync(kFull, base, 0);
    if (ok) {
      const unsigned long long at = base + per * __popc(bm & bfsdev::lanemask_lt());
      if (mode != 2) keys[at] = ((uint64_t)u << vbits) | (uint64_t)v;
      if (mode != 1) keys[at + (mode == 0 ? 1 : 0)] = ((uint64_t)v << vbits) | (uint64_t)u;
    }
  }
}

// ---------------- exclusive scan (int64 output) ----------------
// Input element i is in[i] (uint32 or int64 source) or, for the dedup flags,
// "keys[i] differs from keys[i-1]".
struct ScanInput {
  const uint32_t* u32 = nullptr;
  const int64_t* i64 = nullptr;
  const uint64_t* keys = nullptr;  // dedup flags
  __device__ __forceinline__ long long at(long long i) const {
    if (u32) return u32[i];
    if (i64) return i64[i];
    return (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
  }
};

__device__ __forceinline__ long long block_scan_ll(long long x, long long* s_warp, long long& total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_warp[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x / 32;
    long long v = lane < nw ? s_warp[lane] : 0;
    long long inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(kFull, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane < nw) s_warp[lane] = inc - v;
    if (lane == nw - 1) s_warp[32] = inc;
  }
  __syncthreads();
  const long long excl = s_warp[wid] + incl - x;
  total = s_warp[32];
  __syncthreads();
  return excl;
}

// Tile sums.
__global__ void scan_reduce_kernel(ScanInput in, long long N, int64_t* __restrict__ sums) {
  __shared__ long long s_warp[33];
  const long long base = (long long)blockIdx.x * kScanTile;
  long long x = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const long long idx = base + (long long)threadIdx.x * kScanItems + i;
    if (idx < N) x += in.at(idx);
  }
  long long total;
  block_scan_ll(x, s_warp, total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// Exclusive scan of each tile plus its tile offset.
__global__ void scan_down_kernel(ScanInput in, long long N, const int64_t* __restrict__ tile_off,
                                 int64_t* __restrict__ out) {
  __shared__ long long s_warp[33];
  const long long base = (long long)blockIdx.x * kScanTile;
  long long vals[kScanItems];
  long long x = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const long long idx = base + (long long)threadIdx.x * kScanItems + i;
    vals[i] = idx < N ? in.at(idx) : 0;
    x += vals[i];
  }
  long long total;
  long long run = block_scan_ll(x, s_warp, total) + (tile_off ? tile_off[blockIdx.x] : 0);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const long long idx = base + (long long)threadIdx.x * kScanItems + i;
    if (idx < N) out[idx] = run;
    run += vals[i];
  }
}

// Exclusive scan of N elements into out (int64); returns the total in *total (host).
int exclusive_scan(const ScanInput& in, long long N, int64_t* out, cudaStream_t s, long long* total) {
  if (N <= 0) {
    *total = 0;
    return BFS_OK;
  }
  const long long tiles = (N + kScanTile - 1) / kScanTile;
  int64_t* sums = nullptr;
  int64_t* sums_off = nullptr;
  if (tiles > 1) {
    if (int e = dev_alloc((void**)&sums, sizeof(int64_t) * tiles, "scan tile sums")) return e;
    if (int e = dev_alloc((void**)&sums_off, sizeof(int64_t) * tiles, "scan tile offsets")) {
      cudaFree(sums);
      return e;
    }
    scan_reduce_kernel<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, N, sums);
    ScanInput si;
    si.i64 = sums;
    long long t2 = 0;
    if (int e = exclusive_scan(si, tiles, sums_off, s, &t2)) {
      cudaFree(sums);
      cudaFree(sums_off);
      return e;
    }
  }
  scan_down_kernel<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, N, sums_off, out);
  cudaError_t err = cudaGetLastError();
  // total = out[N-1] + in[N-1]
  long long last_out = 0, last_in = 0;
  if (err == cudaSuccess) err = cudaMemcpyAsync(&last_out, out + (N - 1), sizeof(long long), cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess) {
    if (in.u32) {
      uint32_t v = 0;
      err = cudaMemcpyAsync(&v, in.u32 + (N - 1), sizeof(v), cudaMemcpyDeviceToHost, s);
      if (err == cudaSuccess) err = cudaStreamSynchronize(s);
      last_in = v;
    } else if (in.i64) {
      err = cudaMemcpyAsync(&last_in, in.i64 + (N - 1), sizeof(long long), cudaMemcpyDeviceToHost, s);
      if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    } else {
      uint64_t kk[2] = {0, 0};
      if (N >= 2) err = cudaMemcpyAsync(kk, in.keys + (N - 2), 2 * sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
      if (err == cudaSuccess) err = cudaStreamSynchronize(s);
      last_in = (N == 1 || kk[0] != kk[1]) ? 1 : 0;
    }
  }
  if (sums) cudaFree(sums);
  if (sums_off) cudaFree(sums_off);
  if (err != cudaSuccess) return cuda_fail(err, "exclusive scan");
  *total = last_out + last_in;
  return BFS_OK;
}

// ---------------- radix sort passes ----------------
__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(const uint64_t* __restrict__ keys, long long N,
                                                                  int shift, uint32_t* __restrict__ hist,
                                                                  long long ntiles) {
  __shared__ uint32_t s_h[kRadix];
  for (int i = threadIdx.x; i < kRadix; i += kSortThreads) s_h[i] = 0;
  __syncthreads();
  const long long base = (long long)blockIdx.x * kTile;
  for (int i = threadIdx.x; i < kTile; i += kSortThreads) {
    const long long idx = base + i;
    if (idx < N) atomicAdd(&s_h[(keys[idx] >> shift) & (kRadix - 1)], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kRadix; d += kSortThreads) hist[(long long)d * ntiles + blockIdx.x] = s_h[d];
}

__global__ void __launch_bounds__(kSortThreads) radix_scatter_kernel(const uint64_t* __restrict__ keys_in,
                                                                     uint64_t* __restrict__ keys_out, long long N,
                                                                     int shift, const int64_t* __restrict__ offs,
                                                                     long long ntiles) {
  __shared__ uint32_t s_cnt[kSortWarps][kRadix];
  __shared__ long long s_goff[kRadix];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kSortWarps * kRadix; i += kSortThreads) (&s_cnt[0][0])[i] = 0;
  for (int d = threadIdx.x; d < kRadix; d += kSortThreads) s_goff[d] = offs[(long long)d * ntiles + blockIdx.x];
  __syncthreads();
  const long long seg = (long long)blockIdx.x * kTile + (long long)wid * (32 * kKeysPerThread);
  uint64_t key[kKeysPerThread];
  uint32_t rank[kKeysPerThread];
  int dig[kKeysPerThread];
#pragma unroll
  for (int i = 0; i < kKeysPerThread; ++i) {
    const long long idx = seg + i * 32 + lane;
    const bool valid = idx < N;
    key[i] = valid ? keys_in[idx] : 0;
    const int d = valid ? (int)((key[i] >> shift) & (kRadix - 1)) : kRadix;
    dig[i] = d;
    const unsigned peers = __match_any_sync(kFull, d);
    uint32_t r = 0;
    if (valid) r = s_cnt[wid][d] + __popc(peers & bfsdev::lanemask_lt());
    __syncwarp();
    if (valid && (peers & bfsdev::lanemask_lt()) == 0) s_cnt[wid][d] += __popc(peers);
    __syncwarp();
    rank[i] = r;
  }
  __syncthreads();
  // per digit: exclusive prefix over the warps of the tile
  for (int d = threadIdx.x; d < kRadix; d += kSortThreads) {
    uint32_t run = 0;
    for (int w = 0; w < kSortWarps; ++w) {
      const uint32_t c = s_cnt[w][d];
      s_cnt[w][d] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kKeysPerThread; ++i) {
    const int d = dig[i];
    if (d < kRadix) keys_out[s_goff[d] + s_cnt[wid][d] + rank[i]] = key[i];
  }
}

// ---------------- dedup + CSR emission ----------------
__global__ void emit_csr_kernel(const uint64_t* __restrict__ keys, const int64_t* __restrict__ pos, long long N,
                                int vbits, int32_t n, long long nnz, int64_t* __restrict__ off,
                                int32_t* __restrict__ adj) {
  const uint64_t vmask = (1ull << vbits) - 1ull;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
    const uint64_t k = keys[i];
    // the rows after the last key's row end at nnz (the last key may repeat an
    // earlier one, so this cannot wait for a first occurrence)
    if (i == N - 1)
      for (long long r = (long long)(k >> vbits) + 1; r <= n; ++r) off[r] = nnz;
    const bool first = (i == 0) || k != keys[i - 1];
    if (!first) continue;
    const long long p = pos[i];
    adj[p] = (int32_t)(k & vmask);
    const long long u = (long long)(k >> vbits);
    const long long pu = (i == 0) ? -1 : (long long)(keys[i - 1] >> vbits);
    for (long long r = pu + 1; r <= u; ++r) off[r] = p;
  }
}

__global__ void fill_offsets_kernel(int64_t* off, int32_t n, long long value) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r <= n; r += stride) off[r] = value;
}

// ---------------- validation ----------------
__global__ void validate_kernel(const int64_t* __restrict__ off, const int32_t* __restrict__ adj, int32_t n,
                                long long nnz, int symmetric, int* __restrict__ bad) {
  const int lane = threadIdx.x & 31;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const long long nwarps = (long long)gridDim.x * blockDim.x / 32;
  if (gw == 0 && lane == 0 && (off[0] != 0 || off[n] != nnz)) atomicExch(bad, 1);
  for (long long u = gw; u < n; u += nwarps) {
    const long long b = off[u], e = off[u + 1];
    if (b > e || b < 0 || e > nnz) {
      if (lane == 0) atomicExch(bad, 2);
      continue;
    }
    for (long long j = b + lane; j < e; j += 32) {
      const int v = adj[j];
      if (v < 0 || v >= n || v == u || (j + 1 < e && adj[j + 1] <= v)) {
        atomicExch(bad, 3);
        continue;
      }
      if (!symmetric) continue;
      // symmetry: u must appear in v's row (binary search; v's row is checked by its own warp)
      long long lo = off[v], hi = off[v + 1];
      if (lo < 0 || hi > nnz || lo > hi) {
        atomicExch(bad, 4);
        continue;
      }
      bool found = false;
      while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        const int x = adj[mid];
        if (x == u) {
          found = true;
          break;
        }
        if (x < u) lo = mid + 1;
        else hi = mid;
      }
      if (!found) atomicExch(bad, 5);
    }
  }
}

// Row offsets non-decreasing from 0 to nnz (every row inside [0, nnz)).
__global__ void offsets_kernel(const int64_t* __restrict__ off, int32_t n, long long nnz, int* __restrict__ bad) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i0 == 0 && (off[0] != 0 || off[n] != nnz)) atomicExch(bad, 1);
  for (long long v = i0; v < n; v += stride)
    if (off[v] > off[v + 1]) atomicExch(bad, 1);
}

__global__ void shift_kernel(int64_t* off, int32_t* adj, long long n_part, long long nnz_part, long long off_shift,
                             int32_t id_shift) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_part; i += stride) off[i] += off_shift;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < nnz_part; j += stride) adj[j] += id_shift;
}

__global__ void dead_bits_kernel(const int64_t* __restrict__ off, int32_t n, long long nwords, uint32_t* out) {
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const long long stride = (long long)gridDim.x * blockDim.x / 32;
  const int lane = threadIdx.x & 31;
  for (long long w = gw; w < nwords; w += stride) {
    const long long v = w * 32 + lane;
    const bool dead = v >= n || off[v + 1] == off[v];
    const unsigned m = __ballot_sync(kFull, dead);
    if (lane == 0) out[w] = m;
  }
}

// src[j] = u for every entry j of row u (one warp per row; entries outside
// [0, nnz) of a malformed CSR are skipped).
__global__ void expand_rows_kernel(const int64_t* __restrict__ off, int32_t n, long long nnz,
                                   int32_t* __restrict__ src) {
  const int lane = threadIdx.x & 31;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const long long nwarps = (long long)gridDim.x * blockDim.x / 32;
  for (long long u = gw; u < n; u += nwarps) {
    const long long b = max((long long)off[u], 0ll), e = min((long long)off[u + 1], nnz);
    for (long long j = b + lane; j < e; j += 32) src[j] = (int32_t)u;
  }
}

__global__ void big_chunks_kernel(const int64_t* __restrict__ off, int32_t n, int64_t* items,
                                  unsigned long long* count) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    const long long deg = off[v + 1] - off[v];
    if (deg <= kChunkEdges) continue;
    const unsigned long long nch = (unsigned long long)((deg + kChunkEdges - 1) / kChunkEdges);
    const unsigned long long pos = atomicAdd(count, nch);
    for (unsigned long long c = 0; c < nch; ++c) items[pos + c] = (v << 32) | (long long)c;
  }
}

int bits_for(int32_t n) {
  int b = 1;
  while (b < 31 && ((int64_t)1 << b) < (int64_t)n) ++b;
  return b;
}

}  // namespace

int radix_sort_u64(uint64_t* keys, uint64_t* alt, long long N, int lo_bit, int hi_bit, cudaStream_t s,
                   uint64_t** sorted) {
  *sorted = keys;
  if (N <= 0 || lo_bit >= hi_bit) return BFS_OK;
  const long long ntiles = (N + kTile - 1) / kTile;
  const long long hsize = ntiles * kRadix;
  uint32_t* hist = nullptr;
  int64_t* hoff = nullptr;
  if (int e = dev_alloc((void**)&hist, sizeof(uint32_t) * hsize, "radix histogram")) return e;
  if (int e = dev_alloc((void**)&hoff, sizeof(int64_t) * hsize, "radix offsets")) {
    cudaFree(hist);
    return e;
  }
  uint64_t* a = keys;
  uint64_t* b = alt;
  int rc = BFS_OK;
  for (int shift = lo_bit; shift < hi_bit && !rc; shift += 8) {
    radix_hist_kernel<<<(unsigned)ntiles, kSortThreads, 0, s>>>(a, N, shift, hist, ntiles);
    ScanInput si;
    si.u32 = hist;
    long long tot = 0;
    rc = exclusive_scan(si, hsize, hoff, s, &tot);
    if (rc) break;
    radix_scatter_kernel<<<(unsigned)ntiles, kSortThreads, 0, s>>>(a, b, N, shift, hoff, ntiles);
    uint64_t* t = a;
    a = b;
    b = t;
  }
  cudaError_t err = cudaGetLastError();
  if (!rc && err == cudaSuccess) err = cudaStreamSynchronize(s);
  cudaFree(hist);
  cudaFree(hoff);
  if (rc) return rc;
  if (err != cudaSuccess) return cuda_fail(err, "radix sort");
  *sorted = a;
  return BFS_OK;
}

int exclusive_scan_u32(const uint32_t* in, long long N, int64_t* out, cudaStream_t s, long long* total) {
  ScanInput si;
  si.u32 = in;
  return exclusive_scan(si, N, out, s, total);
}

int build_csr_from_edges(const int32_t* d_src, const int32_t* d_dst, int64_t m, int32_t n, int mode,
                         cudaStream_t s, int64_t** d_off_out, int32_t** d_adj_out, int64_t* nnz_out) {
  DeviceInfo di;
  if (int e = current_device_info(&di)) return e;
  const int vbits = bits_for(n);
  const int total_bits = 2 * vbits;
  uint64_t* keys = nullptr;
  uint64_t* keys_alt = nullptr;
  unsigned long long* d_count = nullptr;
  int* d_bad = nullptr;
  uint32_t* hist = nullptr;
  int64_t* hoff = nullptr;
  int64_t* pos = nullptr;
  int64_t* off = nullptr;
  int32_t* adj = nullptr;
  int rc = BFS_OK;
  long long N = 0, nnz = 0;
  const long long cap = (mode == 0 ? 2 : 1) * (long long)m;
  auto cleanup = [&]() {
    if (keys) cudaFree(keys);
    if (keys_alt) cudaFree(keys_alt);
    if (d_count) cudaFree(d_count);
    if (d_bad) cudaFree(d_bad);
    if (hist) cudaFree(hist);
    if (hoff) cudaFree(hoff);
    if (pos) cudaFree(pos);
  };
  if ((rc = dev_alloc((void**)&d_count, sizeof(unsigned long long) + 16, "edge count"))) return cleanup(), rc;
  if ((rc = dev_alloc((void**)&d_bad, sizeof(int) * 4, "flag"))) return cleanup(), rc;
  if ((rc = dev_alloc((void**)&off, sizeof(int64_t) * ((size_t)n + 1), "CSR offsets"))) return cleanup(), rc;
  cudaError_t err = cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), s);
  if (err == cudaSuccess) err = cudaMemsetAsync(d_bad, 0, sizeof(int), s);
  if (err != cudaSuccess) {
    cleanup();
    cudaFree(off);
    return cuda_fail(err, "memset");
  }
  if (cap > 0) {
    if ((rc = dev_alloc((void**)&keys, sizeof(uint64_t) * cap, "sort keys"))) return cleanup(), cudaFree(off), rc;
    const int grid = di.sm_count * 8;
    make_keys_kernel<<<grid, 256, 0, s>>>(d_src, d_dst, m, n, vbits, mode, keys, d_count, d_bad);
    int bad = 0;
    unsigned long long cnt = 0;
    err = cudaGetLastError();
    if (err == cudaSuccess) err = cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaMemcpyAsync(&cnt, d_count, sizeof(cnt), cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) {
      cleanup();
      cudaFree(off);
      return cuda_fail(err, "key emission");
    }
    if (bad) {
      cleanup();
      cudaFree(off);
      return fail(BFS_ERR_INVALID_ARG, "edge endpoint outside [0, n)");
    }
    N = (long long)cnt;
  }
  if (N > 0) {
    if ((rc = dev_alloc((void**)&keys_alt, sizeof(uint64_t) * N, "sort keys (alternate)")))
      return cleanup(), cudaFree(off), rc;
    const long long ntiles = (N + kTile - 1) / kTile;
    const long long hsize = ntiles * kRadix;
    if ((rc = dev_alloc((void**)&hist, sizeof(uint32_t) * hsize, "radix histogram")))
      return cleanup(), cudaFree(off), rc;
    if ((rc = dev_alloc((void**)&hoff, sizeof(int64_t) * hsize, "radix offsets")))
      return cleanup(), cudaFree(off), rc;
    uint64_t* a = keys;
    uint64_t* b = keys_alt;
    for (int shift = 0; shift < total_bits; shift += 8) {
      radix_hist_kernel<<<(unsigned)ntiles, kSortThreads, 0, s>>>(a, N, shift, hist, ntiles);
      ScanInput si;
      si.u32 = hist;
      long long tot = 0;
      if ((rc = exclusive_scan(si, hsize, hoff, s, &tot))) return cleanup(), cudaFree(off), rc;
      radix_scatter_kernel<<<(unsigned)ntiles, kSortThreads, 0, s>>>(a, b, N, shift, hoff, ntiles);
      uint64_t* t = a;
      a = b;
      b = t;
    }
    // a holds the sorted keys
    cudaFree(hist);
    hist = nullptr;
    cudaFree(hoff);
    hoff = nullptr;
    if ((rc = dev_alloc((void**)&pos, sizeof(int64_t) * N, "dedup positions"))) return cleanup(), cudaFree(off), rc;
    ScanInput fi;
    fi.keys = a;
    if ((rc = exclusive_scan(fi, N, pos, s, &nnz))) return cleanup(), cudaFree(off), rc;
    if ((rc = dev_alloc((void**)&adj, sizeof(int32_t) * (nnz > 0 ? nnz : 1), "CSR adjacency")))
      return cleanup(), cudaFree(off), rc;
    emit_csr_kernel<<<di.sm_count * 8, 256, 0, s>>>(a, pos, N, vbits, n, nnz, off, adj);
  } else {
    if ((rc = dev_alloc((void**)&adj, sizeof(int32_t), "CSR adjacency"))) return cleanup(), cudaFree(off), rc;
    fill_offsets_kernel<<<di.sm_count, 256, 0, s>>>(off, n, 0);
  }
  err = cudaGetLastError();
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  cleanup();
  if (err != cudaSuccess) {
    cudaFree(off);
    cudaFree(adj);
    return cuda_fail(err, "CSR construction");
  }
  *d_off_out = off;
  *d_adj_out = adj;
  *nnz_out = nnz;
  return BFS_OK;
}

int compute_dead_bits(const int64_t* d_off, int32_t n, uint32_t* d_dead, cudaStream_t s) {
  DeviceInfo di;
  if (int e = current_device_info(&di)) return e;
  dead_bits_kernel<<<di.sm_count * 4, 256, 0, s>>>(d_off, n, ((long long)n + 31) / 32, d_dead);
  BFS_CUDA_TRY(cudaGetLastError());
  return BFS_OK;
}

int build_big_chunks(const int64_t* d_off, int32_t n, int64_t nnz, cudaStream_t s, int64_t** items_out,
                     int64_t* count_out) {
  DeviceInfo di;
  if (int e = current_device_info(&di)) return e;
  const long long cap = 2 * (nnz / kChunkEdges) + 2;  // sum of ceil(deg / C) over rows with deg > C
  int64_t* items = nullptr;
  unsigned long long* d_count = nullptr;
  if (int e = dev_alloc((void**)&items, sizeof(int64_t) * cap, "high-degree row chunks")) return e;
  if (int e = dev_alloc((void**)&d_count, sizeof(unsigned long long), "chunk count")) {
    cudaFree(items);
    return e;
  }
  unsigned long long cnt = 0;
  cudaError_t err = cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), s);
  if (err == cudaSuccess) {
    big_chunks_kernel<<<di.sm_count * 4, 256, 0, s>>>(d_off, n, items, d_count);
    err = cudaGetLastError();
  }
  if (err == cudaSuccess) err = cudaMemcpyAsync(&cnt, d_count, sizeof(cnt), cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  cudaFree(d_count);
  if (err != cudaSuccess) {
    cudaFree(items);
    return cuda_fail(err, "high-degree row chunks");
  }
  *items_out = items;
  *count_out = (int64_t)cnt;
  return BFS_OK;
}

int union_shift(int64_t* off, int32_t* adj, int64_t n_part, int64_t nnz_part, int64_t off_shift, int32_t id_shift,
                cudaStream_t s) {
  DeviceInfo di;
  if (int e = current_device_info(&di)) return e;
  shift_kernel<<<di.sm_count * 4, 256, 0, s>>>(off, adj, n_part, nnz_part, off_shift, id_shift);
  BFS_CUDA_TRY(cudaGetLastError());
  return BFS_OK;
}

int build_transpose(const int64_t* d_off, const int32_t* d_adj, int32_t n, int64_t nnz, cudaStream_t s,
                    int64_t** d_toff, int32_t** d_tadj) {
  DeviceInfo di;
  if (int e = current_device_info(&di)) return e;
  int32_t* src = nullptr;
  if (int e = dev_alloc((void**)&src, sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1), "arc tails")) return e;
  expand_rows_kernel<<<di.sm_count * 8, 256, 0, s>>>(d_off, n, nnz, src);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) {
    cudaFree(src);
    return cuda_fail(err, "arc tails");
  }
  int64_t tnnz = 0;
  const int rc = build_csr_from_edges(src, d_adj, nnz, n, 2, s, d_toff, d_tadj, &tnnz);
  cudaFree(src);
  if (rc) return rc;
  if (tnnz != nnz) {
    cudaFree(*d_toff);
    cudaFree(*d_tadj);
    return fail(BFS_ERR_INVALID_GRAPH, "transpose: the CSR has repeated arcs or self-loops");
  }
  return BFS_OK;
}

int check_offsets(const int64_t* d_off, int32_t n, int64_t nnz, int* d_flag, cudaStream_t s, int* ok) {
  DeviceInfo di;
  if (int e = current_device_info(&di)) return e;
  int bad = 0;
  cudaError_t err = cudaMemsetAsync(d_flag, 0, sizeof(int), s);
  if (err == cudaSuccess) {
    offsets_kernel<<<di.sm_count * 4, 256, 0, s>>>(d_off, n, nnz, d_flag);
    err = cudaGetLastError();
  }
  if (err == cudaSuccess) err = cudaMemcpyAsync(&bad, d_flag, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  if (err != cudaSuccess) return cuda_fail(err, "row offset check");
  *ok = bad == 0;
  return BFS_OK;
}

int validate_csr(const int64_t* d_off, const int32_t* d_adj, int32_t n, int64_t nnz, bool symmetric, cudaStream_t s,
                 int* ok) {
  DeviceInfo di;
  if (int e = current_device_info(&di)) return e;
  int* d_bad = nullptr;
  if (int e = dev_alloc((void**)&d_bad, sizeof(int), "validation flag")) return e;
  int bad = 0;
  cudaError_t err = cudaMemsetAsync(d_bad, 0, sizeof(int), s);
  if (err == cudaSuccess) {
    validate_kernel<<<di.sm_count * 4, 256, 0, s>>>(d_off, d_adj, n, nnz, symmetric ? 1 : 0, d_bad);
    err = cudaGetLastError();
  }
  if (err == cudaSuccess) err = cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  cudaFree(d_bad);
  if (err != cudaSuccess) return cuda_fail(err, "CSR validation");
  *ok = bad == 0;
  return BFS_OK;
}

}  // namespace bfsint
