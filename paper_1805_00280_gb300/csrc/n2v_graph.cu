// Graph residency: validation of the caller's CSR, degree statistics, the
// static weight prefix of weighted graphs and the hub neighbour-set cache.
//
// The graph arrays stay where the caller put them (device memory it owns);
// everything built here goes into the caller's auxiliary buffer.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "n2v_internal.cuh"

namespace n2v {

static inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

AuxLayout aux_layout(int64_t n, int64_t nnz, int weighted, const n2v_tune& t) {
  AuxLayout L{};
  size_t off = 0;
  L.status = off;
  off += 256;
  L.scratch = off;
  off += align256(sizeof(unsigned long long) * kScWords);
  L.wpre = off;
  if (weighted) off += align256(sizeof(uint64_t) * (size_t)nnz);
  L.hubs_cap = 0;
  L.slots_cap = 0;
  if (t.hub_count > 0 && n > 0) {
    L.hubs_cap = std::min<int64_t>(t.hub_count, n);
    int64_t budget = (int64_t)t.hub_budget_mb * (1 << 20) / (int64_t)sizeof(int2);
    L.slots_cap = std::max<int64_t>(0, std::min<int64_t>(budget, 4 * nnz + 64));
  }
  L.hub_of = off;
  if (L.hubs_cap > 0) off += align256(sizeof(int32_t) * (size_t)n);
  L.hub_off = off;
  off += align256(sizeof(int64_t) * (size_t)L.hubs_cap);
  L.hub_bits = off;
  off += align256(sizeof(uint32_t) * (size_t)L.hubs_cap);
  L.hub_vtx = off;
  off += align256(sizeof(int32_t) * (size_t)L.hubs_cap);
  L.hub_slot = off;
  off += align256(sizeof(int2) * (size_t)L.slots_cap);
  // rank bitmaps: a probe table of at least twice as many slots as hubs, the hub
  // vertices, and ceil(n/64) 16-byte entries per hub (the data area also holds the
  // degree counts of the hub selection, 4 (n + 2) bytes, before the bitmaps are built)
  L.bm_cap = t.bitmap_hubs > 0 ? std::min<int64_t>(t.bitmap_hubs, n) : 0;
  L.bm_words = (n + 63) / 64;
  L.bm_bits = 4;
  while (((int64_t)1 << L.bm_bits) < 2 * L.bm_cap) ++L.bm_bits;
  L.bm_tab = off;
  if (L.bm_cap > 0) off += align256(sizeof(int2) * ((size_t)1 << L.bm_bits));
  L.bm_vtx = off;
  off += align256(sizeof(int32_t) * (size_t)L.bm_cap);
  L.bm_data = off;
  if (L.bm_cap > 0)
    off += align256(std::max<size_t>(16 * (size_t)L.bm_cap * (size_t)L.bm_words, 4 * ((size_t)n + 2)));
  L.total = off;
  return L;
}

// ---------------------------------------------------------------------------
// kernels

// One thread per vertex: canonical-CSR checks, degree histogram, maxima and the
// row-local inclusive prefix of the weights.
__global__ void k_validate_stats(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                 const uint32_t* __restrict__ w, int64_t n, int64_t nnz,
                                 uint64_t* __restrict__ wpre, unsigned long long* __restrict__ sc) {
  __shared__ unsigned long long hist[34];
  for (int i = threadIdx.x; i < 34; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = rp[u], e = rp[u + 1];
    bool bad = (b < 0) || (e < b) || (e > nnz) || (u == 0 && b != 0) || (u == n - 1 && e != nnz);
    if (bad) {
      atomicOr(&sc[kScBad], 1ull);
      continue;
    }
    int64_t d = e - b;
    uint64_t sum = 0;
    int32_t prev = -1;
    for (int64_t j = b; j < e; ++j) {
      int32_t x = col[j];
      if (x < 0 || x >= n || x <= prev) {
        atomicOr(&sc[kScBad], 2ull);
        break;
      }
      prev = x;
      if (w) {
        sum += w[j];
        wpre[j] = sum;
        atomicMax(&sc[kScWMax], (unsigned long long)w[j]);
        atomicMax(&sc[kScWMin], (unsigned long long)(0xffffffffu - w[j]));  // max of complements = min
      }
    }
    if (!w) sum = (uint64_t)d;
    atomicMax(&sc[kScMaxDeg], (unsigned long long)d);
    atomicMax(&sc[kScMaxWsum], (unsigned long long)sum);
    int bin = d == 0 ? 0 : 64 - __clzll((unsigned long long)d);  // d in [2^(bin-1), 2^bin)
    atomicAdd(&hist[bin], 1ull);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 34; i += blockDim.x)
    if (hist[i]) atomicAdd(&sc[kScHist + i], hist[i]);
}

// count[d] += 1 for every vertex of degree d >= dmin (count lives in the hub_of area).
__global__ void k_degree_counts(const int64_t* __restrict__ rp, int64_t n, int64_t dmin, uint32_t* __restrict__ count) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
    int64_t d = rp[u + 1] - rp[u];
    if (d >= dmin) atomicAdd(&count[d], 1u);
  }
}

__host__ __device__ static inline uint32_t table_bits(int64_t d) {
  uint32_t bits = 1;
  while (((int64_t)1 << bits) < 2 * d) ++bits;
  return bits;
}

// Give every vertex with degree >= dstar a hub slot and a table.
__global__ void k_hub_assign(const int64_t* __restrict__ rp, int64_t n, int64_t dstar, int32_t* __restrict__ hub_of,
                             int64_t* __restrict__ hub_off, uint32_t* __restrict__ hub_bits,
                             int32_t* __restrict__ hub_vtx, unsigned long long* __restrict__ sc, int64_t hubs_cap,
                             int64_t slots_cap) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
    int64_t d = rp[u + 1] - rp[u];
    if (d < dstar) continue;
    uint32_t bits = table_bits(d);
    unsigned long long h = atomicAdd(&sc[kScHubCount], 1ull);
    unsigned long long off = atomicAdd(&sc[kScSlotCount], 1ull << bits);
    if ((int64_t)h >= hubs_cap || (int64_t)(off + (1ull << bits)) > slots_cap) {
      atomicOr(&sc[kScBad], 4ull);  // host-side sizing guarantees this never happens
      continue;
    }
    hub_of[u] = (int32_t)h;
    hub_off[h] = (int64_t)off;
    hub_bits[h] = bits;
    hub_vtx[h] = (int32_t)u;
  }
}

// One block per hub: insert (neighbour, index) pairs by linear probing.
__global__ void k_hub_build(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                            const int64_t* __restrict__ hub_off, const uint32_t* __restrict__ hub_bits,
                            const int32_t* __restrict__ hub_vtx, int2* __restrict__ slots,
                            unsigned long long* __restrict__ sc) {
  const int h = blockIdx.x;
  const int64_t v = hub_vtx[h];
  const int64_t b = rp[v], e = rp[v + 1];
  const uint32_t bits = hub_bits[h];
  const uint32_t mask = (1u << bits) - 1u;
  int2* tab = slots + hub_off[h];
  for (int64_t j = b + threadIdx.x; j < e; j += blockDim.x) {
    int32_t x = col[j];
    uint32_t s = hub_hash(x, bits);
    bool done = false;
    for (uint32_t probe = 0; probe <= mask && !done; ++probe) {
      int old = atomicCAS(&tab[s].x, -1, x);
      if (old == -1) {
        tab[s].y = (int32_t)(j - b);
        done = true;
      } else {
        s = (s + 1u) & mask;
      }
    }
    if (!done) atomicOr(&sc[kScBad], 8ull);
  }
}

// Give every vertex with degree >= dstar a rank bitmap: an index and a slot in
// the probe table.
__global__ void k_bm_assign(const int64_t* __restrict__ rp, int64_t n, int64_t dstar, int2* __restrict__ tab,
                            uint32_t bits, int32_t* __restrict__ bm_vtx, unsigned long long* __restrict__ sc,
                            int64_t cap) {
  const uint32_t mask = (1u << bits) - 1u;
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
    if (rp[u + 1] - rp[u] < dstar) continue;
    const unsigned long long h = atomicAdd(&sc[kScBmCount], 1ull);
    if ((int64_t)h >= cap) {
      atomicOr(&sc[kScBad], 16ull);  // host-side selection guarantees this never happens
      continue;
    }
    bm_vtx[h] = (int32_t)u;
    uint32_t s = hub_hash((int32_t)u, bits);
    bool done = false;
    for (uint32_t probe = 0; probe <= mask && !done; ++probe) {
      if (atomicCAS(&tab[s].x, -1, (int)u) == -1) {
        tab[s].y = (int32_t)h;
        done = true;
      } else {
        s = (s + 1u) & mask;
      }
    }
    if (!done) atomicOr(&sc[kScBad], 16ull);
  }
}

// One block per bitmap hub: set the bit of every neighbour.
__global__ void k_bm_fill(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                          const int32_t* __restrict__ bm_vtx, uint4* __restrict__ data, int64_t words) {
  const int64_t v = bm_vtx[blockIdx.x];
  uint4* d = data + (int64_t)blockIdx.x * words;
  for (int64_t j = rp[v] + threadIdx.x; j < rp[v + 1]; j += blockDim.x) {
    const int32_t x = col[j];
    atomicOr((unsigned long long*)(d + (x >> 6)), 1ull << (x & 63));
  }
}

// One block per bitmap hub: .z of every entry = neighbours in the entries before
// it (a block-wide exclusive scan of the entries' population counts).
__global__ void __launch_bounds__(1024) k_bm_rank(uint4* __restrict__ data, int64_t words) {
  __shared__ uint32_t part[1024];
  uint4* d = data + (int64_t)blockIdx.x * words;
  const int64_t per = (words + blockDim.x - 1) / blockDim.x;
  const int64_t b = threadIdx.x * per, e = min(words, b + per);
  uint32_t sum = 0;
  for (int64_t i = b; i < e; ++i) sum += __popc(d[i].x) + __popc(d[i].y);
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int o = 1; o < (int)blockDim.x; o <<= 1) {  // inclusive scan (Hillis-Steele)
    const uint32_t add = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0u;
    __syncthreads();
    part[threadIdx.x] += add;
    __syncthreads();
  }
  uint32_t run = part[threadIdx.x] - sum;
  for (int64_t i = b; i < e; ++i) {
    uint4 x = d[i];
    x.z = run;
    x.w = 0u;
    run += __popc(x.x) + __popc(x.y);
    d[i] = x;
  }
}

// Build (or rebuild) the rank bitmaps under g->tune.  Synchronises the stream.
static int build_bitmaps(n2v_graph* g, const AuxLayout& L, cudaStream_t s) {
  g->view.bm_data = nullptr;
  g->view.bm_tab = nullptr;
  g->view.bm_words = L.bm_words;
  g->view.bm_bits = L.bm_bits;
  g->view.bm_min_deg = INT64_MAX;
  g->info.bitmap_hubs = 0;
  g->info.bitmap_min_degree = 0;
  if (L.bm_cap <= 0) return N2V_OK;
  const int64_t n = g->n;
  const int64_t maxd = g->info.max_degree;
  const int64_t dmin = std::max<int64_t>(1, g->tune.hub_min_degree);
  const int64_t cap = std::min<int64_t>(L.bm_cap, g->tune.bitmap_hubs);
  if (maxd < dmin || cap <= 0) return N2V_OK;
  char* aux = (char*)g->aux;
  uint32_t* count = (uint32_t*)(aux + L.bm_data);  // 4 (maxd + 1) <= 4 (n + 2) bytes
  const int threads = 256, blocks = g->sms * 8;
  if (cudaMemsetAsync(count, 0, sizeof(uint32_t) * (size_t)(maxd + 1), s) != cudaSuccess) return N2V_ERR_CUDA;
  k_degree_counts<<<blocks, threads, 0, s>>>(g->view.rp, n, dmin, count);
  std::vector<uint32_t> hc((size_t)(maxd + 1 - dmin));
  if (cudaMemcpyAsync(hc.data(), count + dmin, sizeof(uint32_t) * hc.size(), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return N2V_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return N2V_ERR_CUDA;
  int64_t hubs = 0, dstar = -1;  // largest degrees first, whole degree classes
  for (int64_t d = maxd; d >= dmin; --d) {
    const int64_t c = hc[(size_t)(d - dmin)];
    if (!c) continue;
    if (hubs + c > cap) break;
    hubs += c;
    dstar = d;
  }
  if (dstar < 0 || hubs == 0) return N2V_OK;
  unsigned long long* sc = g->scratch;
  cudaError_t e = cudaMemsetAsync(aux + L.bm_tab, 0xff, sizeof(int2) * ((size_t)1 << L.bm_bits), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(aux + L.bm_data, 0, 16 * (size_t)hubs * (size_t)L.bm_words, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(sc + kScBmCount, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return N2V_ERR_CUDA;
  k_bm_assign<<<blocks, threads, 0, s>>>(g->view.rp, n, dstar, (int2*)(aux + L.bm_tab), L.bm_bits,
                                         (int32_t*)(aux + L.bm_vtx), sc, hubs);
  k_bm_fill<<<(unsigned)hubs, 256, 0, s>>>(g->view.rp, g->view.col, (const int32_t*)(aux + L.bm_vtx),
                                           (uint4*)(aux + L.bm_data), L.bm_words);
  k_bm_rank<<<(unsigned)hubs, 1024, 0, s>>>((uint4*)(aux + L.bm_data), L.bm_words);
  unsigned long long bad = 0;
  if (cudaMemcpyAsync(&bad, sc + kScBad, sizeof(bad), cudaMemcpyDeviceToHost, s) != cudaSuccess) return N2V_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return N2V_ERR_CUDA;
  if (bad) return N2V_ERR_CUDA;
  g->view.bm_data = (const uint4*)(aux + L.bm_data);
  g->view.bm_tab = (const int2*)(aux + L.bm_tab);
  g->view.bm_min_deg = dstar;
  g->info.bitmap_hubs = (int32_t)hubs;
  g->info.bitmap_min_degree = dstar;
  return N2V_OK;
}

// Build (or rebuild) the hub cache under g->tune.  Synchronises the stream.
static int build_hubs(n2v_graph* g, const AuxLayout& L, cudaStream_t s) {
  g->view.hub_of = nullptr;
  g->view.hub_off = nullptr;
  g->view.hub_bits = nullptr;
  g->view.hub_slot = nullptr;
  g->view.hub_min_deg = INT64_MAX;
  g->info.hub_count = 0;
  g->info.hub_min_degree = 0;
  g->info.hub_slots = 0;
  // the current tuning's caps, inside the layout's (which may be the larger loaded one)
  const int64_t hubs_cap = std::min<int64_t>(L.hubs_cap, g->tune.hub_count);
  const int64_t slots_cap =
      std::min<int64_t>(L.slots_cap, (int64_t)g->tune.hub_budget_mb * (1 << 20) / (int64_t)sizeof(int2));
  if (hubs_cap <= 0 || slots_cap <= 0) return N2V_OK;
  const int64_t n = g->n;
  const int64_t maxd = g->info.max_degree;
  const int64_t dmin = std::max<int64_t>(1, g->tune.hub_min_degree);
  if (maxd < dmin) return N2V_OK;
  char* aux = (char*)g->aux;
  uint32_t* count = (uint32_t*)(aux + L.hub_of);
  int threads = 256, blocks = g->sms * 8;
  if (cudaMemsetAsync(count, 0, sizeof(uint32_t) * (size_t)(maxd + 1), s) != cudaSuccess) return N2V_ERR_CUDA;
  k_degree_counts<<<blocks, threads, 0, s>>>(g->view.rp, n, dmin, count);
  std::vector<uint32_t> hc((size_t)(maxd + 1 - dmin));
  if (cudaMemcpyAsync(hc.data(), count + dmin, sizeof(uint32_t) * hc.size(), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return N2V_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return N2V_ERR_CUDA;
  // largest degrees first, whole degree classes, within the hub and slot caps
  int64_t hubs = 0, slots = 0, dstar = -1;
  for (int64_t d = maxd; d >= dmin; --d) {
    int64_t c = hc[(size_t)(d - dmin)];
    if (!c) continue;
    int64_t add = c * ((int64_t)1 << table_bits(d));
    if (hubs + c > hubs_cap || slots + add > slots_cap) break;
    hubs += c;
    slots += add;
    dstar = d;
  }
  if (dstar < 0 || hubs == 0) return N2V_OK;
  unsigned long long* sc = g->scratch;
  cudaError_t e = cudaSuccess;
  e = cudaMemsetAsync(aux + L.hub_of, 0xff, sizeof(int32_t) * (size_t)n, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(aux + L.hub_slot, 0xff, sizeof(int2) * (size_t)slots, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(sc + kScHubCount, 0, 2 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return N2V_ERR_CUDA;
  k_hub_assign<<<blocks, threads, 0, s>>>(g->view.rp, n, dstar, (int32_t*)(aux + L.hub_of), (int64_t*)(aux + L.hub_off),
                                          (uint32_t*)(aux + L.hub_bits), (int32_t*)(aux + L.hub_vtx), sc, L.hubs_cap,
                                          L.slots_cap);
  k_hub_build<<<(unsigned)hubs, 256, 0, s>>>(g->view.rp, g->view.col, (const int64_t*)(aux + L.hub_off),
                                             (const uint32_t*)(aux + L.hub_bits), (const int32_t*)(aux + L.hub_vtx),
                                             (int2*)(aux + L.hub_slot), sc);
  unsigned long long bad = 0;
  if (cudaMemcpyAsync(&bad, sc + kScBad, sizeof(bad), cudaMemcpyDeviceToHost, s) != cudaSuccess) return N2V_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return N2V_ERR_CUDA;
  if (bad) return N2V_ERR_CUDA;
  g->view.hub_of = (const int32_t*)(aux + L.hub_of);
  g->view.hub_off = (const int64_t*)(aux + L.hub_off);
  g->view.hub_bits = (const uint32_t*)(aux + L.hub_bits);
  g->view.hub_slot = (const int2*)(aux + L.hub_slot);
  g->view.hub_min_deg = dstar;
  g->info.hub_count = (int32_t)hubs;
  g->info.hub_min_degree = dstar;
  g->info.hub_slots = slots;
  return N2V_OK;
}

static bool tune_ok(const n2v_tune& t) {
  if (t.block_threads < 64 || t.block_threads > 256 || t.block_threads % 32) return false;
  if (t.blocks_per_sm < 0 || t.thread_max_deg < 0 || t.smem_specials < 32 || t.smem_specials > 8192) return false;
  if (t.hub_count < 0 || t.hub_min_degree < 0 || t.chunk_walkers < 0 || t.hub_budget_mb < 0) return false;
  if (t.stage_window != 0 && (t.stage_window < 64 || t.stage_window > 4096 || (t.stage_window & (t.stage_window - 1))))
    return false;
  if (t.stream_ratio < 0 || t.stream_ratio > 1000000 || t.spill_specials < 0 || t.spill_specials > (1 << 24)) return false;
  if (t.smem_specials % 32) return false;
  if (t.stage_buffers != 2 && t.stage_buffers != 4) return false;
  if (t.bitmap_hubs < 0 || t.bitmap_hubs > 4096 || t.block_min_deg < 0) return false;
  if (t.merge_ratio < 0 || t.merge_ratio > 1000000 || t.l2_persist_mb < 0 || t.l2_persist_mb > 4096) return false;
  if (t.reserved[0]) return false;
  return true;
}

}  // namespace n2v

using namespace n2v;

extern "C" {

void n2v_tune_default(n2v_tune* t) {
  if (!t) return;
  memset(t, 0, sizeof(*t));
  t->block_threads = 128;
  t->blocks_per_sm = 0;
  t->thread_max_deg = 16;
  t->smem_specials = 256;
  t->hub_count = 0;
  t->hub_min_degree = 256;
  t->chunk_walkers = 0;
  t->hub_budget_mb = 1024;
  t->stage_window = 1024;
  t->stream_ratio = 40;
  t->spill_specials = 4096;
  t->stage_buffers = 2;
  t->merge_ratio = 0;
}

int n2v_graph_aux_bytes(int64_t n, int64_t nnz, int weighted, const n2v_tune* t, size_t* bytes) {
  if (!bytes || n < 1 || nnz < 0 || n > INT32_MAX) return N2V_ERR_INVALID_ARG;
  n2v_tune d;
  n2v_tune_default(&d);
  const n2v_tune& tt = t ? *t : d;
  if (!tune_ok(tt)) return N2V_ERR_INVALID_ARG;
  *bytes = aux_layout(n, nnz, weighted ? 1 : 0, tt).total;
  return N2V_OK;
}

int n2v_graph_load(const int64_t* row_ptr, const int32_t* col, const uint32_t* w, int64_t n, int64_t nnz, void* aux,
                   size_t aux_bytes, const n2v_tune* t, void* stream, n2v_graph** out) {
  if (!out) return N2V_ERR_INVALID_ARG;
  *out = nullptr;
  if (!row_ptr || (!col && nnz > 0) || !aux || n < 1 || nnz < 0 || n > INT32_MAX) return N2V_ERR_INVALID_ARG;
  if (((uintptr_t)aux & 255) != 0 || ((uintptr_t)col & 15) != 0) return N2V_ERR_INVALID_ARG;
  n2v_tune tt;
  n2v_tune_default(&tt);
  if (t) tt = *t;
  if (!tune_ok(tt)) return N2V_ERR_INVALID_ARG;
  const int weighted = w ? 1 : 0;
  AuxLayout L = aux_layout(n, nnz, weighted, tt);
  if (aux_bytes < L.total) return N2V_ERR_NO_MEM;
  cudaStream_t s = (cudaStream_t)stream;

  n2v_graph* g = (n2v_graph*)calloc(1, sizeof(n2v_graph));
  if (!g) return N2V_ERR_NO_MEM;
  g->n = n;
  g->nnz = nnz;
  g->weighted = weighted;
  g->aux = aux;
  g->aux_bytes = aux_bytes;
  g->tune = tt;
  g->tune_loaded = tt;
  char* a = (char*)aux;
  g->status = (uint32_t*)(a + L.status);
  g->scratch = (unsigned long long*)(a + L.scratch);
  if (cudaGetDevice(&g->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, g->device) != cudaSuccess) {
    free(g);
    return N2V_ERR_CUDA;
  }
  g->view.rp = row_ptr;
  g->view.col = col;
  g->view.w = w;
  g->view.wpre = weighted ? (const uint64_t*)(a + L.wpre) : nullptr;
  g->view.n = n;
  g->view.nnz = nnz;
  g->view.status = g->status;

  int rc = N2V_OK;
  unsigned long long sc[kScWords];
  if (cudaMemsetAsync(a, 0, L.scratch + sizeof(unsigned long long) * kScWords, s) != cudaSuccess) rc = N2V_ERR_CUDA;
  if (rc == N2V_OK) {
    k_validate_stats<<<g->sms * 8, 256, 0, s>>>(row_ptr, col, w, n, nnz, (uint64_t*)g->view.wpre, g->scratch);
    if (cudaMemcpyAsync(sc, g->scratch, sizeof(sc), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      rc = N2V_ERR_CUDA;
  }
  if (rc == N2V_OK && sc[kScBad]) rc = N2V_ERR_INVALID_GRAPH;
  // the samplers pack a neighbour's index into 30 bits
  if (rc == N2V_OK && sc[kScMaxDeg] >= (1ull << 30)) rc = N2V_ERR_INVALID_ARG;
  if (rc == N2V_OK) {
    g->info.n = n;
    g->info.nnz = nnz;
    g->info.weighted = weighted;
    g->info.max_degree = (int64_t)sc[kScMaxDeg];
    g->info.max_wsum = (uint64_t)sc[kScMaxWsum];
    g->info.w_min = weighted && nnz > 0 ? 0xffffffffu - (uint32_t)sc[kScWMin] : 1u;
    g->info.w_max = weighted && nnz > 0 ? (uint32_t)sc[kScWMax] : 1u;
    for (int i = 0; i < 34; ++i) g->info.deg_hist[i] = (int64_t)sc[kScHist + i];
    rc = build_hubs(g, L, s);
    if (rc == N2V_OK) rc = build_bitmaps(g, L, s);
  }
  if (rc == N2V_OK) {
    g->graph_cache = new_graph_cache();
    if (!g->graph_cache) rc = N2V_ERR_NO_MEM;
  }
  if (rc != N2V_OK) {
    free(g);
    return rc;
  }
  *out = g;
  return N2V_OK;
}

int n2v_graph_info_get(const n2v_graph* g, n2v_graph_info* info) {
  if (!g || !info) return N2V_ERR_INVALID_ARG;
  *info = g->info;
  return N2V_OK;
}

int n2v_graph_retune(n2v_graph* g, const n2v_tune* t, void* stream) {
  if (!g || !t || !tune_ok(*t)) return N2V_ERR_INVALID_ARG;
  AuxLayout L = aux_layout(g->n, g->nnz, g->weighted, *t);
  if (L.total > g->aux_bytes) return N2V_ERR_NO_MEM;
  clear_graph_cache(g);
  const bool same_hubs = t->hub_count == g->tune.hub_count && t->hub_min_degree == g->tune.hub_min_degree &&
                         t->hub_budget_mb == g->tune.hub_budget_mb;
  const bool same_bm = t->bitmap_hubs == g->tune.bitmap_hubs && t->hub_min_degree == g->tune.hub_min_degree;
  // the caches must be built at the layout the graph was loaded with (aux offsets do not move)
  const AuxLayout L0 = aux_layout(g->n, g->nnz, g->weighted, g->tune_loaded);
  if (t->hub_count > g->tune_loaded.hub_count || t->hub_budget_mb > g->tune_loaded.hub_budget_mb ||
      t->bitmap_hubs > g->tune_loaded.bitmap_hubs)
    return N2V_ERR_NO_MEM;
  (void)L;
  g->tune = *t;
  int rc = same_hubs ? N2V_OK : build_hubs(g, L0, (cudaStream_t)stream);
  if (rc == N2V_OK && !same_bm) rc = build_bitmaps(g, L0, (cudaStream_t)stream);
  return rc;
}

void n2v_graph_free(n2v_graph* g) {
  if (!g) return;
  free_graph_cache(g);
  free(g);
}

}  // extern "C"
