// Stored transition tables: the per-edge precomputation that Fast-Node2Vec
// avoids (Section 3.2, Eq. 1).  For every directed edge t -> v the table holds
// the cumulative weights C_j = sum_{i <= j} w(v, x_i) * alpha(t, x_i) over
// N(v) for one fixed (p, q): one uint64 per (edge, neighbour) pair, so the
// space is 8 * sum over edges of deg(target), which is 8 * sum_i d_i^2 on an
// undirected graph (Eq. 1).  A step then needs one binary search of the
// stored C for r = floor(u * T / 2^64), the same choice the on-the-fly
// sampler makes, so the rows are identical.
//
// Layout of the caller's table buffer (256-byte aligned pieces):
//   header   StoredHeader
//   off      int64 [nnz + 1]   first entry of edge e's C (exclusive scan of deg(col[e]))
//   sums     int64 [tiles]     scratch of the build's scan
//   cdf      uint64 [entries]
#include <string.h>

#include <algorithm>

#include "n2v_step.cuh"

namespace n2v {

constexpr uint64_t kStoredMagic = 0x31424154324e3253ull;  // tag of a built table
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int64_t kScanTile = (int64_t)kScanThreads * kScanItems;

struct StoredHeader {
  uint64_t magic;
  uint32_t a_p, a_q;
  int64_t n, nnz, entries;
  uint64_t col_addr;  // the graph the table was built for
  uint32_t weighted, pad;
};

struct StoredLayout {
  size_t off, sums, cdf, total;
  int64_t tiles;
};

static size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

static StoredLayout stored_layout(int64_t nnz, int64_t entries) {
  StoredLayout L;
  L.tiles = (nnz + 1 + kScanTile - 1) / kScanTile;
  L.off = up256(sizeof(StoredHeader));
  L.sums = up256(L.off + sizeof(int64_t) * (size_t)(nnz + 1));
  L.cdf = up256(L.sums + sizeof(int64_t) * (size_t)L.tiles);
  L.total = L.cdf + sizeof(uint64_t) * (size_t)entries;
  return L;
}

// sum over edges of deg(col[e])
__global__ void __launch_bounds__(256) k_stored_entries(GraphView g, unsigned long long* sum) {
  unsigned long long acc = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < g.nnz; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = __ldg(g.col + e);
    acc += (unsigned long long)(__ldg(g.rp + v + 1) - __ldg(g.rp + v));
  }
  acc = warp_sum_u64(acc);
  if ((threadIdx.x & 31) == 0 && acc) atomicAdd(sum, acc);
}

// off[e] = deg(col[e]) for e < nnz, off[nnz] = 0 (the scan turns it into the total)
__global__ void __launch_bounds__(256) k_stored_degcol(GraphView g, int64_t* off) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e <= g.nnz; e += (int64_t)gridDim.x * blockDim.x) {
    if (e == g.nnz) {
      off[e] = 0;
    } else {
      const int32_t v = __ldg(g.col + e);
      off[e] = __ldg(g.rp + v + 1) - __ldg(g.rp + v);
    }
  }
}

// Exclusive scan of thread totals across a block of kScanThreads; returns
// this thread's exclusive prefix and the block total.
__device__ __forceinline__ int64_t block_excl_scan(int64_t x, int64_t* warp_tot, int64_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t incl = (int64_t)warp_incl_scan_u64((uint64_t)x, lane);
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    int64_t y = lane < nw ? warp_tot[lane] : 0;
    int64_t yi = (int64_t)warp_incl_scan_u64((uint64_t)y, lane);
    if (lane < nw) warp_tot[lane] = yi - y;  // exclusive
    if (lane == nw - 1) warp_tot[32] = yi;
  }
  __syncthreads();
  const int64_t r = warp_tot[warp] + incl - x;
  *total = warp_tot[32];
  __syncthreads();
  return r;
}

// phase 1: each tile of kScanTile elements scanned in place (exclusive within
// the tile); the tile's total into sums[tile]
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(int64_t* a, int64_t n, int64_t* sums) {
  __shared__ int64_t warp_tot[33];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t item[kScanItems];
  int64_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    item[i] = base + i < n ? a[base + i] : 0;
    s += item[i];
  }
  int64_t total = 0;
  int64_t run = block_excl_scan(s, warp_tot, &total);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) a[base + i] = run;
    run += item[i];
  }
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// phase 2: one block scans the tile totals (exclusive), chunk by chunk
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(int64_t* sums, int64_t tiles) {
  __shared__ int64_t warp_tot[33];
  int64_t carry = 0;
  for (int64_t c0 = 0; c0 < tiles; c0 += kScanThreads) {
    const int64_t i = c0 + threadIdx.x;
    const int64_t x = i < tiles ? sums[i] : 0;
    int64_t total = 0;
    const int64_t ex = block_excl_scan(x, warp_tot, &total);
    if (i < tiles) sums[i] = carry + ex;
    carry += total;
  }
}

// phase 3: add each tile's offset
__global__ void __launch_bounds__(256) k_scan_add(int64_t* a, int64_t n, const int64_t* sums) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a[i] += __ldg(sums + i / kScanTile);
}

__global__ void k_stored_header(StoredHeader* h, StoredHeader v) { *h = v; }

// C over N(v) for every edge e = t -> v: one warp per edge.  alpha(t, x) as in
// Section 2.1: a_p for x == t, one for x in N(t), a_q otherwise (Q16).
__global__ void __launch_bounds__(256) k_stored_fill(GraphView g, const int64_t* __restrict__ off,
                                                     uint64_t* __restrict__ cdf, uint32_t a_p, uint32_t a_q) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t e = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); e < g.nnz; e += nwarps) {
    // the source t of edge e: the last row starting at or before e
    int64_t lo = 0, hi = g.n;  // rp[lo] <= e < rp[hi]
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) >> 1;
      if (__ldg(g.rp + mid) <= e) lo = mid;
      else hi = mid;
    }
    const int32_t t = (int32_t)lo;
    const int32_t v = __ldg(g.col + e);
    const int64_t bv = __ldg(g.rp + v), dv = __ldg(g.rp + v + 1) - bv;
    const int64_t bt = __ldg(g.rp + t), dt = __ldg(g.rp + t + 1) - bt;
    uint64_t* C = cdf + __ldg(off + e);
    uint64_t carry = 0;
    for (int64_t j0 = 0; j0 < dv; j0 += 32) {
      const int64_t j = j0 + lane;
      uint64_t c = 0;
      if (j < dv) {
        const int32_t x = __ldg(g.col + bv + j);
        const uint64_t a = x == t ? a_p : (contains_i32(g.col + bt, dt, x) ? kAlphaOne : a_q);
        c = (g.w ? (uint64_t)__ldg(g.w + bv + j) : 1ull) * a;
      }
      const uint64_t s = warp_incl_scan_u64(c, lane) + carry;
      if (j < dv) C[j] = s;
      carry = __shfl_sync(kFull, s, 31);
    }
  }
}

// First index in [0, n) of a non-decreasing a with a[i] > key (n if none).
__device__ __forceinline__ int64_t first_above_u64(const uint64_t* __restrict__ a, int64_t n, uint64_t key) {
  int64_t lo = 0;
  while (n > 0) {
    const int64_t half = n >> 1;
    if (__ldg(a + lo + half) <= key) {
      lo += half + 1;
      n -= half + 1;
    } else {
      n = half;
    }
  }
  return lo;
}

// One thread per walker, all l steps in one launch.  The walker carries the
// CSR index e of its last edge t -> v, which names the table of the step.
__global__ void __launch_bounds__(256) k_stored_walk(GraphView g, const int64_t* __restrict__ off,
                                                     const uint64_t* __restrict__ cdf, WalkJob J) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < J.count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t wid = J.walk_begin + i;
    int32_t* row = J.walks + i * (int64_t)J.l;
    const int64_t s0 = J.starts[wid % J.n_starts];
    int k = 0;
    if (s0 < 0 || s0 >= g.n) {
      atomicOr(J.status, kStInvalidArg);
    } else {
      int64_t v = s0, e = -1;
#ifdef N2V_CHECKED
      int64_t t = -1;  // the previous vertex, for the checked build's total
#endif
      for (; k < J.l; ++k) {
        const int64_t bv = __ldg(g.rp + v), dv = __ldg(g.rp + v + 1) - bv;
        if (dv == 0) break;
        const uint64_t u = philox_draw(J.seed, (uint64_t)wid, (uint32_t)k);
        int64_t j;
        if (k == 0) {
          if (!g.w) {
            j = (int64_t)scale_draw(u, (uint64_t)dv);
          } else {
            const uint64_t T0 = __ldg(g.wpre + bv + dv - 1);
            if (T0 == 0) break;
            j = first_above_u64(g.wpre + bv, dv, scale_draw(u, T0));
          }
        } else {
          const uint64_t* C = cdf + __ldg(off + e);
          const uint64_t T = __ldg(C + dv - 1);
          // the edge's stored entries are one per neighbour of v, and its stored total is the on-the-fly one
          N2V_CHECK(g, __ldg(off + e + 1) - __ldg(off + e) == dv);
#ifdef N2V_CHECKED
          N2V_CHECK(g, T == merge_total(g.rp, g.col, g.w, t, v, J.a_p, J.a_q));
#endif
          if (T == 0) break;
          j = first_above_u64(C, dv, scale_draw(u, T));
        }
        N2V_CHECK(g, j >= 0 && j < dv);
        e = bv + j;
#ifdef N2V_CHECKED
        t = v;
#endif
        v = __ldg(g.col + e);
        row[k] = (int32_t)v;
      }
    }
    for (; k < J.l; ++k) row[k] = -1;
  }
}

static int grid_for(const n2v_graph* g, int64_t work, int threads) {
  const int64_t want = (work + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)g->sms * 16));
}

}  // namespace n2v

using namespace n2v;

extern "C" {

int n2v_stored_bytes(const n2v_graph* g, void* stream, size_t* bytes, int64_t* entries) {
  if (!g || !bytes) return N2V_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long* sum = g->scratch + kScSumDeg2;
  if (cudaMemsetAsync(sum, 0, sizeof(*sum), s) != cudaSuccess) return N2V_ERR_CUDA;
  if (g->nnz > 0) k_stored_entries<<<grid_for(g, g->nnz, 256), 256, 0, s>>>(g->view, sum);
  unsigned long long h = 0;
  if (cudaMemcpyAsync(&h, sum, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess) return N2V_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return N2V_ERR_CUDA;
  *bytes = stored_layout(g->nnz, (int64_t)h).total;
  if (entries) *entries = (int64_t)h;
  return N2V_OK;
}

int n2v_stored_build(const n2v_graph* g, double p, double q, void* table, size_t table_bytes, void* stream) {
  if (!g || !table || ((uintptr_t)table & 255)) return N2V_ERR_INVALID_ARG;
  uint32_t a_p, a_q;
  if (n2v_alpha_q16(p, q, &a_p, &a_q) != N2V_OK) return N2V_ERR_INVALID_ARG;
  const uint64_t amax = std::max<uint64_t>(std::max<uint64_t>(a_p, a_q), kAlphaOne);
  if (g->info.max_wsum > UINT64_MAX / amax) return N2V_ERR_OVERFLOW;
  size_t need = 0;
  int64_t entries = 0;
  int rc = n2v_stored_bytes(g, stream, &need, &entries);
  if (rc != N2V_OK) return rc;
  if (table_bytes < need) return N2V_ERR_NO_MEM;
  cudaStream_t s = (cudaStream_t)stream;
  const StoredLayout L = stored_layout(g->nnz, entries);
  char* base = (char*)table;
  int64_t* off = (int64_t*)(base + L.off);
  int64_t* sums = (int64_t*)(base + L.sums);
  uint64_t* cdf = (uint64_t*)(base + L.cdf);
  const int64_t n_off = g->nnz + 1;
  k_stored_degcol<<<grid_for(g, n_off, 256), 256, 0, s>>>(g->view, off);
  k_scan_tiles<<<(unsigned)L.tiles, kScanThreads, 0, s>>>(off, n_off, sums);
  k_scan_sums<<<1, kScanThreads, 0, s>>>(sums, L.tiles);
  k_scan_add<<<grid_for(g, n_off, 256), 256, 0, s>>>(off, n_off, sums);
  if (g->nnz > 0) k_stored_fill<<<grid_for(g, g->nnz * 32, 256), 256, 0, s>>>(g->view, off, cdf, a_p, a_q);
  StoredHeader h;
  memset(&h, 0, sizeof(h));
  h.magic = kStoredMagic;
  h.a_p = a_p;
  h.a_q = a_q;
  h.n = g->n;
  h.nnz = g->nnz;
  h.entries = entries;
  h.col_addr = (uint64_t)(uintptr_t)g->view.col;
  h.weighted = (uint32_t)g->weighted;
  k_stored_header<<<1, 1, 0, s>>>((StoredHeader*)base, h);
  return cudaGetLastError() == cudaSuccess ? N2V_OK : N2V_ERR_CUDA;
}

int n2v_stored_walk(const n2v_graph* g, const void* table, const int32_t* starts, int64_t n_starts, int32_t r,
                    int32_t l, uint64_t seed, int64_t walk_begin, int64_t walk_count, int32_t* walks, void* stream) {
  if (!g || !table || ((uintptr_t)table & 255) || l < 1 || r < 1 || n_starts < 1 || walk_begin < 0 || walk_count < 0)
    return N2V_ERR_INVALID_ARG;
  if (n_starts > INT64_MAX / r) return N2V_ERR_INVALID_ARG;
  const int64_t total = n_starts * (int64_t)r;
  if (walk_begin > total || walk_count > total - walk_begin) return N2V_ERR_INVALID_ARG;
  if (walk_count == 0) return N2V_OK;
  if (!starts || !walks) return N2V_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  StoredHeader h;
  if (cudaMemcpyAsync(&h, table, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess) return N2V_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return N2V_ERR_CUDA;
  if (h.magic != kStoredMagic || h.n != g->n || h.nnz != g->nnz || h.col_addr != (uint64_t)(uintptr_t)g->view.col)
    return N2V_ERR_INVALID_ARG;
  const StoredLayout L = stored_layout(h.nnz, h.entries);
  const char* base = (const char*)table;
  WalkJob J;
  memset(&J, 0, sizeof(J));
  J.starts = starts;
  J.n_starts = n_starts;
  J.walk_begin = walk_begin;
  J.count = walk_count;
  J.l = l;
  J.a_p = h.a_p;
  J.a_q = h.a_q;
  J.seed = seed;
  J.walks = walks;
  J.status = g->status;
  k_stored_walk<<<grid_for(g, walk_count, 256), 256, 0, s>>>(g->view, (const int64_t*)(base + L.off),
                                                            (const uint64_t*)(base + L.cdf), J);
  return cudaGetLastError() == cudaSuccess ? N2V_OK : N2V_ERR_CUDA;
}

}  // extern "C"
