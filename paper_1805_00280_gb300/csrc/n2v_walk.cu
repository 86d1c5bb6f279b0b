// The three samplers (plain, binned, persistent), their launch logic, the
// CUDA-graph recording of a call's launch sequence, and the walk-traffic
// counter.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "n2v_step.cuh"

namespace n2v {

// ---------------------------------------------------------------------------
// Plain: one thread per walker, one launch per step k.  The walker's state is
// read back from its own output row (v = row[k-1], t = row[k-2] or the start).
__global__ void __launch_bounds__(256) k_plain_step(GraphView g, WalkJob J, int k) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= J.count) return;
  const int64_t wid = J.walk_begin + i;
  int32_t* row = J.walks + i * (int64_t)J.l;
  const int64_t s0 = J.starts[wid % J.n_starts];
  if (s0 < 0 || s0 >= g.n) {
    if (k == 0) atomicOr(J.status, kStInvalidArg);
    row[k] = -1;
    return;
  }
  int64_t v, t;
  if (k == 0) {
    v = s0;
    t = -1;
  } else {
    v = row[k - 1];
    if (v < 0) {
      row[k] = -1;
      return;
    }
    t = (k == 1) ? s0 : row[k - 2];
  }
  const uint64_t u = philox_draw(J.seed, (uint64_t)wid, (uint32_t)k);
  if (J.approx && k > 0) {
    const int64_t bv = g.rp[v], ev = g.rp[v + 1];
    if (approx_here(J, k, ev - bv, g.rp[t + 1] - g.rp[t])) {
      row[k] = static_step(g, bv, ev, u);
      return;
    }
  }
  row[k] = thread_step(g, t, v, k, u, J.a_p, J.a_q);
}

// ---------------------------------------------------------------------------
// Binned: one launch per step k; warp w owns walkers [32w, 32w + 32) and bins
// each of their steps by degree (own lane, or the whole warp).
__global__ void __launch_bounds__(256) k_binned_step(GraphView g, WalkJob J, int k, LaunchCfg L) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t base = ((int64_t)blockIdx.x * (blockDim.x >> 5) + warp) * 32;
  if (base >= J.count) return;  // uniform per warp
  WarpSmem sm = warp_smem(smem_raw, warp, L, nullptr);
  warp_smem_init(sm, lane);
  const int64_t i = base + lane;
  const bool mine = i < J.count;
  const int64_t wid = J.walk_begin + i;
  int32_t* row = J.walks + i * (int64_t)J.l;
  bool alive = false;
  int64_t v = -1, t = -1;
  if (mine) {
    const int64_t s0 = J.starts[wid % J.n_starts];
    if (s0 >= 0 && s0 < g.n) {
      if (k == 0) {
        v = s0;
        alive = true;
      } else {
        v = row[k - 1];
        t = (k == 1) ? s0 : row[k - 2];
        alive = v >= 0;
      }
    } else if (k == 0) {
      atomicOr(J.status, kStInvalidArg);
    }
  }
  const int32_t x = warp_binned_step(g, alive, t, v, k, (uint64_t)wid, J, L.thread_max_deg, sm, L.stream_ratio, lane);
  if (mine) row[k] = alive ? x : -1;
  if (sm.timed_out && lane == 0) atomicOr(J.status, kStTimeout);
}

// ---------------------------------------------------------------------------
// Persistent: one launch for all l steps.  Each warp takes 32 walkers at a
// time from a device counter and runs them to the end; every step is binned
// by degree as above.  Walkers are independent (FN-Multi's observation,
// Section 3.4), so the order in which warps take them does not change any row.
// KIND selects the full or a lean instance (PersistKind).
template <int MINB, int KIND>
__global__ void __launch_bounds__(kPersistThreads, MINB)
    k_persistent(GraphView g, WalkJob J, unsigned long long* __restrict__ counter, LaunchCfg L,
                 uint32_t* __restrict__ spill) {
  constexpr bool FULL = KIND == kPersistFull;
  if (KIND == kPersistLeanUnw) fold_unweighted(g);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  WarpSmem sm = warp_smem(smem_raw, warp, L, spill ? spill + gw * (int64_t)L.spill_specials : nullptr);
  warp_smem_init(sm, lane);
#ifdef N2V_STATS
  const long long t_kernel = clock64();
#endif
  while (!sm.timed_out) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(counter, 32ull);
    base = __shfl_sync(kFull, base, 0);
    if ((int64_t)base >= J.count) break;
    const int64_t i = (int64_t)base + lane;
    const bool mine = i < J.count;
    const int64_t wid = J.walk_begin + i;
    int32_t* row = J.walks + i * (int64_t)J.l;
    int64_t t = -1, v = -1;
    bool alive = false;
    if (mine) {
      const int64_t s0 = J.starts[wid % J.n_starts];
      if (s0 >= 0 && s0 < g.n) {
        v = s0;
        alive = true;
      } else {
        atomicOr(J.status, kStInvalidArg);
      }
    }
    int k = 0;
    for (; k < J.l; ++k) {
      if (sm.timed_out || !__any_sync(kFull, alive)) break;
      const int32_t x = warp_binned_step<FULL>(g, alive, t, v, k, (uint64_t)wid, J, L.thread_max_deg, sm,
                                               L.stream_ratio, lane);
      N2V_CHECK(g, !alive || (x >= -1 && x < g.n));
      if (mine) row[k] = alive ? x : -1;
      if (alive) {
        if (x < 0) {
          alive = false;
        } else {
          t = v;
          v = x;
        }
      }
    }
    if (mine)
      for (int kk = k; kk < J.l; ++kk) row[kk] = -1;
  }
#ifdef N2V_STATS
  if (lane == 0) N2V_STAT(kStatKernelCycles, clock64() - t_kernel);
#endif
  if (sm.timed_out && lane == 0) atomicOr(J.status, kStTimeout);
}

// ---------------------------------------------------------------------------
// Persistent with a block tier: each block takes 128 walkers at a time and
// advances them together, one step at a time; every step is binned into the
// lane, warp and block tiers through the block's shared-memory work queue
// (block_binned_step), which lives after the four warps' areas.
template <int MINB>
__global__ void __launch_bounds__(kPersistThreads, MINB)
    k_persistent_blk(GraphView g, WalkJob J, unsigned long long* __restrict__ counter, LaunchCfg L,
                     uint32_t* __restrict__ spill) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t gw = (int64_t)blockIdx.x * (kPersistThreads / 32) + warp;
  WarpSmem sm = warp_smem(smem_raw, warp, L, spill ? spill + gw * (int64_t)L.spill_specials : nullptr);
  BlockQueue* bq = reinterpret_cast<BlockQueue*>(smem_raw + (size_t)(kPersistThreads / 32) * warp_smem_bytes(L));
  warp_smem_init(sm, lane);
  for (;;) {
    if (tid == 0) {
      bq->base = atomicAdd(counter, (unsigned long long)kPersistThreads);
      bq->nb[0] = bq->nb[1] = 0;
      bq->nw[0] = bq->nw[1] = 0;
      bq->pull[0] = bq->pull[1] = 0;
    }
    __syncthreads();
    const int64_t base = (int64_t)bq->base;
    if (base >= J.count) break;  // uniform: every thread read the same base
    const int64_t i = base + tid;
    const bool mine = i < J.count;
    const int64_t wid = J.walk_begin + i;
    int32_t* row = J.walks + i * (int64_t)J.l;
    int64_t t = -1, v = -1;
    bool alive = false;
    if (mine) {
      const int64_t s0 = J.starts[wid % J.n_starts];
      if (s0 >= 0 && s0 < g.n) {
        v = s0;
        alive = true;
      } else {
        atomicOr(J.status, kStInvalidArg);
      }
    }
    int k = 0;
    for (; k < J.l; ++k) {
      if (sm.timed_out) alive = false;  // a warp whose bounded wait gave up stops its walkers
      if (!__syncthreads_or(alive)) break;
      const int32_t x = block_binned_step(g, alive, t, v, k, (uint64_t)wid, J, L, sm, bq, warp, lane, tid);
      N2V_CHECK(g, !alive || (x >= -1 && x < g.n));
      if (mine) row[k] = alive ? x : -1;
      if (alive) {
        if (x < 0) {
          alive = false;
        } else {
          t = v;
          v = x;
        }
      }
    }
    if (mine)
      for (int kk = k; kk < J.l; ++kk) row[kk] = -1;
    if (__syncthreads_or(sm.timed_out)) break;  // also: nobody reads bq before thread 0 rewrites it
  }
  if (sm.timed_out && lane == 0) atomicOr(J.status, kStTimeout);
}

// ---------------------------------------------------------------------------
// Traffic counter: one thread per row.
__global__ void k_traffic(const int64_t* __restrict__ rp, int weighted, const int32_t* __restrict__ starts,
                          int64_t n_starts, int64_t walk_begin, int64_t count, int32_t l,
                          const int32_t* __restrict__ walks, unsigned long long* __restrict__ out3) {
  unsigned long long steps = 0, bytes = 0, lower = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t* row = walks + i * (int64_t)l;
    const int64_t s0 = starts[(walk_begin + i) % n_starts];
    int64_t t = -1, v = s0;
    for (int k = 0; k < l; ++k) {
      const int32_t x = row[k];
      if (x < 0 || v < 0) break;
      const unsigned long long b = 16 + 4ull * (unsigned long long)(rp[v + 1] - rp[v]) * (weighted ? 2 : 1) + 4;
      steps += 1;
      lower += b;
      bytes += b + (k >= 1 ? 16 + 4ull * (unsigned long long)(rp[t + 1] - rp[t]) : 0ull);
      t = v;
      v = x;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    steps += __shfl_xor_sync(kFull, steps, o);
    bytes += __shfl_xor_sync(kFull, bytes, o);
    lower += __shfl_xor_sync(kFull, lower, o);
  }
  if ((threadIdx.x & 31) == 0 && (steps || bytes)) {
    atomicAdd(&out3[0], steps);
    atomicAdd(&out3[1], bytes);
    atomicAdd(&out3[2], lower);
  }
}

// ---------------------------------------------------------------------------
// Self-test of the bounded waits: one warp waits on an mbarrier that nothing
// arrives on, with the samplers' wait routine and a short limit, then records
// the timeout in the status word and returns (no copy is in flight).
__global__ void k_selftest_wait(uint32_t* status, long long limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncwarp();
  const bool ok = mbar_wait_bounded(&bar, 0u, limit);
  if (!ok && threadIdx.x == 0) atomicOr(status, kStTimeout);
}

// ---------------------------------------------------------------------------
// launch configuration

static int smem_per_block(const LaunchCfg& c) {
  return (c.block_threads / 32) * warp_smem_bytes(c) + (c.block_min_deg > 0 ? (int)sizeof(BlockQueue) : 0);
}

// The persistent kernel is compiled for 4, 5, 6 or 8 resident blocks of 128
// threads per SM: 128, 96, 80 or 64 registers a thread (each of the SM's four
// schedulers holds one warp of every block in its 16384 registers).  Fewer
// registers than the code wants spill to local memory; more warps hide more
// latency.
static int persistent_minb(int per_sm) { return per_sm <= 4 ? 4 : per_sm <= 5 ? 5 : per_sm <= 6 ? 6 : 8; }

static const void* persistent_fn(int minb, bool blk, int kind) {
  if (blk) {
    switch (minb) {
      case 4: return (const void*)k_persistent_blk<4>;
      case 6: return (const void*)k_persistent_blk<6>;
      case 8: return (const void*)k_persistent_blk<8>;
      default: return (const void*)k_persistent_blk<5>;
    }
  }
  if (kind == kPersistLeanUnw) {
    switch (minb) {
      case 4: return (const void*)k_persistent<4, kPersistLeanUnw>;
      case 6: return (const void*)k_persistent<6, kPersistLeanUnw>;
      case 8: return (const void*)k_persistent<8, kPersistLeanUnw>;
      default: return (const void*)k_persistent<5, kPersistLeanUnw>;
    }
  }
  if (kind == kPersistLean) {
    switch (minb) {
      case 4: return (const void*)k_persistent<4, kPersistLean>;
      case 6: return (const void*)k_persistent<6, kPersistLean>;
      case 8: return (const void*)k_persistent<8, kPersistLean>;
      default: return (const void*)k_persistent<5, kPersistLean>;
    }
  }
  switch (minb) {
    case 4: return (const void*)k_persistent<4, kPersistFull>;
    case 6: return (const void*)k_persistent<6, kPersistFull>;
    case 8: return (const void*)k_persistent<8, kPersistFull>;
    default: return (const void*)k_persistent<5, kPersistFull>;
  }
}

// The instance a persistent launch takes: block batches when the block tier is
// on; else a lean instance unless the call needs FN-Approx, the graph's view
// carries a hub cache, or the merge form is on (the unweighted one for a graph
// without weights).
static const void* persistent_fn(const LaunchCfg& L, const GraphView& g, const WalkJob& J) {
  const bool blk = L.block_min_deg > 0;
  return persistent_fn(L.minb, blk, blk || J.approx ? kPersistFull : persist_kind(L, g));
}

// One persistent launch.  With L.l2_persist_bytes > 0 (warp batches only) the
// first that many bytes of col are marked persisting in L2 (access-policy
// window; the rest of the kernel's accesses stream as usual).
static void launch_persistent(const LaunchCfg& L, int smem, cudaStream_t s, GraphView g, WalkJob J,
                              unsigned long long* counter, uint32_t* spill) {
  LaunchCfg Lc = L;
  void* args[] = {&g, &J, &counter, &Lc, &spill};
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)L.blocks);
  cfg.blockDim = dim3((unsigned)L.block_threads);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = s;
  if (L.l2_persist_bytes > 0 && L.block_min_deg == 0) {
    attr[0].id = cudaLaunchAttributeAccessPolicyWindow;
    attr[0].val.accessPolicyWindow.base_ptr = (void*)g.col;
    attr[0].val.accessPolicyWindow.num_bytes = L.l2_persist_bytes;
    attr[0].val.accessPolicyWindow.hitRatio = 1.0f;
    attr[0].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
    attr[0].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  cudaLaunchKernelExC(&cfg, persistent_fn(L, g, J), args);
}

// The persisting L2 window over the start of col: the tuning's size, capped by
// the device's largest window and by col itself.  The context's persisting
// set-aside is raised to the window once per device (a limit of this process's
// context, gone with it).  Returns 0 when the device offers none.
static std::mutex g_l2_mu;
static size_t g_l2_set[64];

static size_t l2_persist_window(const n2v_graph* g) {
  int max_win = 0, max_persist = 0;
  if (cudaDeviceGetAttribute(&max_win, cudaDevAttrMaxAccessPolicyWindowSize, g->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, g->device) != cudaSuccess)
    return 0;
  size_t bytes = (size_t)g->tune.l2_persist_mb << 20;
  bytes = std::min(bytes, (size_t)max_win);
  bytes = std::min(bytes, (size_t)max_persist);
  bytes = std::min(bytes, sizeof(int32_t) * (size_t)g->nnz);
  if (bytes == 0 || g->device < 0 || g->device >= 64) return 0;
  std::lock_guard<std::mutex> lock(g_l2_mu);
  if (g_l2_set[g->device] < bytes) {
    if (cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, bytes) != cudaSuccess) return 0;
    g_l2_set[g->device] = bytes;
  }
  return bytes;
}

LaunchCfg resolve_launch(const n2v_graph* g, int variant) {
  LaunchCfg c{};
  c.block_threads = g->tune.block_threads;
  c.thread_max_deg = g->tune.thread_max_deg;
  c.smem_specials = g->tune.smem_specials;
  c.stage_window = g->tune.stage_window;
  c.stream_ratio = g->tune.stream_ratio;
  c.spill_specials = g->tune.spill_specials;
  c.stage_buffers = g->tune.stage_buffers;
  c.merge_ratio = g->tune.merge_ratio;
  c.block_min_deg = 0;
  c.l2_persist_bytes = 0;
  if (g->tune.l2_persist_mb > 0 && variant == N2V_PERSISTENT) c.l2_persist_bytes = l2_persist_window(g);
  if (variant == N2V_PERSISTENT) {
    // 128-thread blocks; the tuning's resident warps per SM (20 by default),
    // as many as shared memory holds
    c.block_threads = kPersistThreads;
    c.block_min_deg = g->tune.block_min_deg;
    const int warps = g->tune.blocks_per_sm > 0 ? g->tune.blocks_per_sm * (g->tune.block_threads / 32) : 20;
    int per_sm = std::max(1, (warps + 3) / 4);
    const int smem = smem_per_block(c);
    const void* fn = persistent_fn(8, c.block_min_deg > 0, kPersistFull);  // the fewest registers: only shared memory limits it
    if (smem > 48 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, c.block_threads, smem) == cudaSuccess && occ > 0)
      per_sm = std::min(per_sm, occ);
    c.minb = persistent_minb(per_sm);
    c.blocks = g->sms * per_sm;
    return c;
  }
  const int smem = smem_per_block(c);
  int per_sm = g->tune.blocks_per_sm;
  if (per_sm <= 0) {
    per_sm = 1;
    const void* fn = (const void*)k_binned_step;
    if (smem > 48 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, c.block_threads, smem) == cudaSuccess && occ > 0)
      per_sm = occ;
  }
  c.blocks = g->sms * per_sm;
  return c;
}

static int64_t n_chunks(const n2v_graph* g, int64_t count) {
  const int64_t cw = g->tune.chunk_walkers;
  if (cw <= 0 || count <= 0) return 1;
  return (count + cw - 1) / cw;
}

static size_t counter_bytes(int64_t chunks) { return (sizeof(unsigned long long) * (size_t)chunks + 255) & ~(size_t)255; }

struct WalkCall {
  const int32_t* starts;
  int64_t n_starts;
  int32_t l;
  uint32_t a_p, a_q;
  uint64_t seed;
  int64_t walk_begin, count;
  int32_t* walks;
  void* ws;
  int variant;
  int approx;  // FN-Approx parameters (approx == 0: exact walks)
  double approx_eps;
  int64_t approx_popular;
};

// Enqueue the launches of one call on stream s.
static cudaError_t issue(const n2v_graph* g, const WalkCall& c, cudaStream_t s) {
  WalkJob J;
  J.starts = c.starts;
  J.n_starts = c.n_starts;
  J.walk_begin = c.walk_begin;
  J.count = c.count;
  J.l = c.l;
  J.a_p = c.a_p;
  J.a_q = c.a_q;
  J.seed = c.seed;
  J.walks = c.walks;
  J.status = g->status;
  J.approx = c.approx;
  J.approx_eps = c.approx_eps;
  J.approx_popular = c.approx_popular;
  J.w_min = g->info.w_min;
  J.w_max = g->info.w_max;
  const int base = c.variant & 0xff;
  if (base == N2V_PLAIN) {
    const unsigned blocks = (unsigned)((c.count + 255) / 256);
    for (int k = 0; k < c.l; ++k) k_plain_step<<<blocks, 256, 0, s>>>(g->view, J, k);
    return cudaGetLastError();
  }
  const LaunchCfg L = resolve_launch(g, base);
  const int smem = smem_per_block(L);
  if (base == N2V_BINNED) {
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_binned_step, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    const int64_t warps = (c.count + 31) / 32;
    const int wpb = L.block_threads / 32;
    const unsigned blocks = (unsigned)((warps + wpb - 1) / wpb);
    for (int k = 0; k < c.l; ++k)
      k_binned_step<<<blocks, L.block_threads, smem, s>>>(g->view, J, k, L);
    return cudaGetLastError();
  }
  // persistent
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(persistent_fn(L, g->view, J), cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  const int64_t chunks = n_chunks(g, c.count);
  unsigned long long* counters = (unsigned long long*)c.ws;
  cudaError_t e = cudaMemsetAsync(counters, 0, sizeof(unsigned long long) * (size_t)chunks, s);
  if (e != cudaSuccess) return e;
  const int64_t per = chunks == 1 ? c.count : g->tune.chunk_walkers;
  uint32_t* spill = L.spill_specials > 0 ? (uint32_t*)((char*)c.ws + counter_bytes(chunks)) : nullptr;
  for (int64_t ci = 0; ci < chunks; ++ci) {
    WalkJob Jc = J;
    const int64_t lo = ci * per;
    Jc.walk_begin = c.walk_begin + lo;
    Jc.count = std::min<int64_t>(per, c.count - lo);
    Jc.walks = c.walks + lo * (int64_t)c.l;
    launch_persistent(L, smem, s, g->view, Jc, counters + ci, spill);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// CUDA-graph recording of a call's launch sequence, keyed by every argument.

struct GraphEntry {
  WalkCall key;
  cudaGraphExec_t exec;
};
struct GraphCache {
  std::mutex mu;
  std::vector<GraphEntry> entries;
};

static bool same_call(const WalkCall& a, const WalkCall& b) { return memcmp(&a, &b, sizeof(WalkCall)) == 0; }

// The cache is created with the handle (n2v_graph_load), so that calls from
// several threads never race to create it; retuning only empties it.
void* new_graph_cache() { return new (std::nothrow) GraphCache(); }

void clear_graph_cache(n2v_graph* g) {
  GraphCache* gc = (GraphCache*)g->graph_cache;
  if (!gc) return;
  std::lock_guard<std::mutex> lock(gc->mu);
  for (auto& e : gc->entries) cudaGraphExecDestroy(e.exec);
  gc->entries.clear();
}

void free_graph_cache(n2v_graph* g) {
  clear_graph_cache(g);
  delete (GraphCache*)g->graph_cache;
  g->graph_cache = nullptr;
}

static int issue_graph(n2v_graph* g, const WalkCall& c, cudaStream_t s) {
  if (!s) return N2V_ERR_INVALID_ARG;  // the legacy stream cannot be recorded
  GraphCache* gc = (GraphCache*)g->graph_cache;
  if (!gc) return N2V_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(gc->mu);
  for (auto& e : gc->entries)
    if (same_call(e.key, c)) return cudaGraphLaunch(e.exec, s) == cudaSuccess ? N2V_OK : N2V_ERR_CUDA;
  // make sure lazy function attributes are set before recording
  if ((c.variant & 0xff) != N2V_PLAIN) resolve_launch(g, c.variant & 0xff);
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return N2V_ERR_CUDA;
  cudaError_t e1 = issue(g, c, s);
  cudaError_t e2 = cudaStreamEndCapture(s, &graph);
  if (e1 != cudaSuccess || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return N2V_ERR_CUDA;
  }
  cudaGraphExec_t exec = nullptr;
  cudaError_t e3 = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e3 != cudaSuccess) return N2V_ERR_CUDA;
  if (gc->entries.size() >= 16) {
    cudaGraphExecDestroy(gc->entries.front().exec);
    gc->entries.erase(gc->entries.begin());
  }
  gc->entries.push_back({c, exec});
  return cudaGraphLaunch(exec, s) == cudaSuccess ? N2V_OK : N2V_ERR_CUDA;
}

}  // namespace n2v

using namespace n2v;

extern "C" {

int n2v_alpha_q16(double p, double q, uint32_t* a_p, uint32_t* a_q) {
  if (!a_p || !a_q) return N2V_ERR_INVALID_ARG;
  if (!isfinite(p) || !isfinite(q) || !(p > 0.0) || !(q > 0.0)) return N2V_ERR_INVALID_ARG;
  // one rounding, to nearest with ties to even, of the IEEE double quotient
  const double xp = nearbyint(65536.0 / p), xq = nearbyint(65536.0 / q);
  if (!(xp >= 1.0 && xp <= 16777216.0 && xq >= 1.0 && xq <= 16777216.0)) return N2V_ERR_INVALID_ARG;
  *a_p = (uint32_t)xp;
  *a_q = (uint32_t)xq;
  return N2V_OK;
}

int n2v_walk_ws_bytes(const n2v_graph* g, int64_t walk_count, int32_t l, int variant, size_t* bytes) {
  if (!g || !bytes || walk_count < 0 || l < 1) return N2V_ERR_INVALID_ARG;
  const int base = variant & 0xff;
  if (base != N2V_PLAIN && base != N2V_BINNED && base != N2V_PERSISTENT) return N2V_ERR_INVALID_ARG;
  size_t b = 0;
  if (base == N2V_PERSISTENT) {
    const LaunchCfg L = resolve_launch(g, base);
    b = counter_bytes(n_chunks(g, walk_count));
    b += sizeof(uint32_t) * (size_t)L.blocks * (size_t)(L.block_threads / 32) * (size_t)L.spill_specials;
  }
  *bytes = b;
  return N2V_OK;
}

static int walk_impl(const n2v_graph* g, const int32_t* starts, int64_t n_starts, int32_t r, int32_t l, double p,
                     double q, uint64_t seed, int64_t walk_begin, int64_t walk_count, int32_t* walks, void* ws,
                     size_t ws_bytes, int variant, int approx, double eps, int64_t popular, void* stream);

int n2v_walk(const n2v_graph* g, const int32_t* starts, int64_t n_starts, int32_t r, int32_t l, double p, double q,
             uint64_t seed, int64_t walk_begin, int64_t walk_count, int32_t* walks, void* ws, size_t ws_bytes,
             int variant, void* stream) {
  return walk_impl(g, starts, n_starts, r, l, p, q, seed, walk_begin, walk_count, walks, ws, ws_bytes, variant, 0, 0.0,
                   0, stream);
}

int n2v_walk_approx(const n2v_graph* g, const int32_t* starts, int64_t n_starts, int32_t r, int32_t l, double p,
                    double q, uint64_t seed, int64_t walk_begin, int64_t walk_count, int32_t* walks, void* ws,
                    size_t ws_bytes, int variant, double eps, int64_t popular_degree, void* stream) {
  if (!(eps >= 0.0) || !isfinite(eps) || popular_degree < 1) return N2V_ERR_INVALID_ARG;
  return walk_impl(g, starts, n_starts, r, l, p, q, seed, walk_begin, walk_count, walks, ws, ws_bytes, variant, 1, eps,
                   popular_degree, stream);
}

static int walk_impl(const n2v_graph* g, const int32_t* starts, int64_t n_starts, int32_t r, int32_t l, double p,
                     double q, uint64_t seed, int64_t walk_begin, int64_t walk_count, int32_t* walks, void* ws,
                     size_t ws_bytes, int variant, int approx, double eps, int64_t popular, void* stream) {
  if (!g || l < 1 || r < 1 || n_starts < 1 || walk_begin < 0 || walk_count < 0) return N2V_ERR_INVALID_ARG;
  const int base = variant & 0xff;
  if (base != N2V_PLAIN && base != N2V_BINNED && base != N2V_PERSISTENT) return N2V_ERR_INVALID_ARG;
  if ((variant & ~0xff) & ~N2V_FLAG_CUDA_GRAPH) return N2V_ERR_INVALID_ARG;
  if (n_starts > INT64_MAX / r) return N2V_ERR_INVALID_ARG;
  const int64_t total = n_starts * (int64_t)r;
  if (walk_begin > total || walk_count > total - walk_begin) return N2V_ERR_INVALID_ARG;
  uint32_t a_p, a_q;
  if (n2v_alpha_q16(p, q, &a_p, &a_q) != N2V_OK) return N2V_ERR_INVALID_ARG;
  const uint64_t amax = std::max<uint64_t>(std::max<uint64_t>(a_p, a_q), kAlphaOne);
  if (g->info.max_wsum > UINT64_MAX / amax) return N2V_ERR_OVERFLOW;
  if (walk_count == 0) return N2V_OK;
  if (!starts || !walks) return N2V_ERR_INVALID_ARG;
  size_t need = 0;
  n2v_walk_ws_bytes(g, walk_count, l, variant, &need);
  if (need > 0 && (!ws || ws_bytes < need)) return N2V_ERR_NO_MEM;
  if (ws && ((uintptr_t)ws & 255) != 0) return N2V_ERR_INVALID_ARG;
  WalkCall c;
  memset(&c, 0, sizeof(c));
  c.starts = starts;
  c.n_starts = n_starts;
  c.l = l;
  c.a_p = a_p;
  c.a_q = a_q;
  c.seed = seed;
  c.walk_begin = walk_begin;
  c.count = walk_count;
  c.walks = walks;
  c.ws = ws;
  c.variant = base;
  c.approx = approx;
  c.approx_eps = eps;
  c.approx_popular = popular;
  cudaStream_t s = (cudaStream_t)stream;
  if (variant & N2V_FLAG_CUDA_GRAPH) return issue_graph(const_cast<n2v_graph*>(g), c, s);
  return issue(g, c, s) == cudaSuccess ? N2V_OK : N2V_ERR_CUDA;
}

int n2v_walk_stream(const n2v_graph* g, const int32_t* starts, int64_t n_starts, int32_t r, int32_t l, double p,
                    double q, uint64_t seed, int64_t walk_begin, int64_t walk_count, int32_t* host_walks,
                    int32_t* dev_ring, int64_t ring_walks, int32_t ring_slots, void* ws, size_t ws_bytes,
                    int variant, void* stream, void* copy_stream) {
  if (!g || l < 1 || r < 1 || n_starts < 1 || walk_begin < 0 || walk_count < 0) return N2V_ERR_INVALID_ARG;
  if (ring_walks < 1 || ring_slots < 1 || ring_slots > 8 || (variant & N2V_FLAG_CUDA_GRAPH)) return N2V_ERR_INVALID_ARG;
  if (walk_count == 0) return N2V_OK;
  if (!host_walks || !dev_ring || !starts) return N2V_ERR_INVALID_ARG;
  if (n_starts > INT64_MAX / r || walk_begin + walk_count > n_starts * (int64_t)r) return N2V_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream, cs = copy_stream ? (cudaStream_t)copy_stream : s;
  cudaEvent_t ready[8], copied[8];
  int made = 0, rc = N2V_OK;
  for (; made < ring_slots; ++made) {
    if (cudaEventCreateWithFlags(&ready[made], cudaEventDisableTiming) != cudaSuccess) break;
    if (cudaEventCreateWithFlags(&copied[made], cudaEventDisableTiming) != cudaSuccess) {
      cudaEventDestroy(ready[made]);
      break;
    }
  }
  if (made < ring_slots) rc = N2V_ERR_CUDA;
  const int64_t chunks = (walk_count + ring_walks - 1) / ring_walks;
  const size_t slot_elems = (size_t)ring_walks * (size_t)l;
  for (int64_t ci = 0; ci < chunks && rc == N2V_OK; ++ci) {
    const int b = (int)(ci % ring_slots);
    const int64_t lo = ci * ring_walks, cnt = std::min<int64_t>(ring_walks, walk_count - lo);
    int32_t* slot = dev_ring + (size_t)b * slot_elems;
    // the slot's previous rows must have reached the host before they are overwritten
    if (ci >= ring_slots && cs != s && cudaStreamWaitEvent(s, copied[b], 0) != cudaSuccess) rc = N2V_ERR_CUDA;
    if (rc == N2V_OK)
      rc = n2v_walk(g, starts, n_starts, r, l, p, q, seed, walk_begin + lo, cnt, slot, ws, ws_bytes, variant, stream);
    if (rc == N2V_OK && cudaEventRecord(ready[b], s) != cudaSuccess) rc = N2V_ERR_CUDA;
    if (rc == N2V_OK && cs != s && cudaStreamWaitEvent(cs, ready[b], 0) != cudaSuccess) rc = N2V_ERR_CUDA;
    if (rc == N2V_OK &&
        cudaMemcpyAsync(host_walks + (size_t)lo * (size_t)l, slot, sizeof(int32_t) * (size_t)cnt * (size_t)l,
                        cudaMemcpyDeviceToHost, cs) != cudaSuccess)
      rc = N2V_ERR_CUDA;
    if (rc == N2V_OK && cudaEventRecord(copied[b], cs) != cudaSuccess) rc = N2V_ERR_CUDA;
  }
  // `stream` reaches the end of the call only after the last copies
  if (rc == N2V_OK && cs != s)
    for (int64_t ci = std::max<int64_t>(0, chunks - ring_slots); ci < chunks && rc == N2V_OK; ++ci)
      if (cudaStreamWaitEvent(s, copied[ci % ring_slots], 0) != cudaSuccess) rc = N2V_ERR_CUDA;
  for (int i = 0; i < made; ++i) {  // released once the work recorded on them completes
    cudaEventDestroy(ready[i]);
    cudaEventDestroy(copied[i]);
  }
  return rc;
}

int n2v_walk_traffic(const n2v_graph* g, const int32_t* starts, int64_t n_starts, int64_t walk_begin,
                     int64_t walk_count, int32_t l, const int32_t* walks, uint64_t* out3, void* stream) {
  if (!g || !out3 || l < 1 || n_starts < 1 || walk_begin < 0 || walk_count < 0) return N2V_ERR_INVALID_ARG;
  if (walk_count > 0 && (!starts || !walks)) return N2V_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(out3, 0, 3 * sizeof(uint64_t), s) != cudaSuccess) return N2V_ERR_CUDA;
  if (walk_count == 0) return N2V_OK;
  const unsigned blocks = (unsigned)std::min<int64_t>((walk_count + 255) / 256, (int64_t)g->sms * 16);
  k_traffic<<<blocks, 256, 0, s>>>(g->view.rp, g->weighted, starts, n_starts, walk_begin, walk_count, l, walks,
                                   (unsigned long long*)out3);
  return cudaGetLastError() == cudaSuccess ? N2V_OK : N2V_ERR_CUDA;
}

int n2v_selftest_timeout(const n2v_graph* g, int64_t limit_cycles, void* stream) {
  if (!g || limit_cycles < 1 || limit_cycles > (1ll << 34)) return N2V_ERR_INVALID_ARG;
  k_selftest_wait<<<1, 32, 0, (cudaStream_t)stream>>>(g->status, (long long)limit_cycles);
  return cudaGetLastError() == cudaSuccess ? N2V_OK : N2V_ERR_CUDA;
}

int n2v_stream_status(const n2v_graph* g, void* stream) {
  if (!g) return N2V_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t st = 0;
  if (cudaStreamSynchronize(s) != cudaSuccess) return N2V_ERR_CUDA;
  if (cudaMemcpy(&st, g->status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess) return N2V_ERR_CUDA;
  if (st && cudaMemset(g->status, 0, sizeof(st)) != cudaSuccess) return N2V_ERR_CUDA;
  if (st & kStTimeout) return N2V_ERR_TIMEOUT;
  if (st & kStInternal) return N2V_ERR_INTERNAL;
  if (st & kStInvalidArg) return N2V_ERR_INVALID_ARG;
  return N2V_OK;
}

const char* n2v_strerror(int code) {
  switch (code) {
    case N2V_OK: return "ok";
    case N2V_ERR_INVALID_ARG: return "invalid argument";
    case N2V_ERR_INVALID_GRAPH: return "invalid graph (CSR not canonical)";
    case N2V_ERR_OVERFLOW: return "weighted totals could overflow 64 bits for these p, q";
    case N2V_ERR_NO_MEM: return "caller buffer too small";
    case N2V_ERR_TIMEOUT: return "bounded device wait timed out";
    case N2V_ERR_CUDA: return "CUDA runtime error";
    case N2V_ERR_INTERNAL: return "a device self-check of the checked build failed";
    default: return "unknown status";
  }
}

int n2v_step_stats(uint64_t* out, int32_t n, int32_t reset) {
  if (!out || n < 1 || n > kStatWords) return N2V_ERR_INVALID_ARG;
#ifdef N2V_STATS
  if (cudaDeviceSynchronize() != cudaSuccess) return N2V_ERR_CUDA;
  if (cudaMemcpyFromSymbol(out, g_step_stats, sizeof(uint64_t) * (size_t)n) != cudaSuccess) return N2V_ERR_CUDA;
  if (reset) {
    static const unsigned long long zero[kStatWords] = {};
    if (cudaMemcpyToSymbol(g_step_stats, zero, sizeof(zero)) != cudaSuccess) return N2V_ERR_CUDA;
  }
  return N2V_OK;
#else
  (void)reset;
  memset(out, 0, sizeof(uint64_t) * (size_t)n);
  return N2V_ERR_INVALID_ARG;  // not the stats build
#endif
}

int n2v_launch_shape(const n2v_graph* g, int32_t* sms, int32_t* blocks, int32_t* threads) {
  if (!g) return N2V_ERR_INVALID_ARG;
  LaunchCfg L = resolve_launch(g, N2V_PERSISTENT);
  if (sms) *sms = g->sms;
  if (blocks) *blocks = L.blocks;
  if (threads) *threads = L.block_threads;
  return N2V_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free variant of the persistent sampler.
//
// Some callers cannot allocate device memory at the point where they need
// walks: code running inside a memory pool or arena that another runtime owns,
// plugins handed only a stream and the input/output buffers, or real-time
// paths where an allocation could block or fail.  For them the persistent
// sampler can run on a scratch area that lives inside this library: a
// file-scope device array of kNoAllocScratchBytes, reserved on every GPU that
// loads the library until the process exits.  The scratch holds the work
// counters (one per persistent launch) and the per-warp spill area for
// special neighbours; the spill area is only a cache, so a smaller one
// changes speed, never results.

namespace n2v {

constexpr size_t kNoAllocScratchBytes = (size_t)4 << 20;  // 4 MiB per device
constexpr size_t kNoAllocCounterBytes = 4096;              // room for 512 launch counters
constexpr int64_t kNoAllocMaxLaunches = (int64_t)(kNoAllocCounterBytes / sizeof(unsigned long long));
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch per device.  In host code the symbol
// is only a host-side stand-in; the address comes from cudaGetSymbolAddress
// with the device current, once per device.
static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[kNoAllocMaxDevices];

static int noalloc_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return N2V_ERR_CUDA;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return N2V_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return N2V_ERR_CUDA;
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return N2V_OK;
}

}  // namespace n2v

extern "C" int n2v_walk_noalloc(const n2v_graph* g, const int32_t* starts, int64_t n_starts, int32_t r, int32_t l,
                                double p, double q, uint64_t seed, int64_t walk_begin, int64_t walk_count,
                                int32_t* walks, void* stream) {
  using namespace n2v;
  if (!g || l < 1 || r < 1 || n_starts < 1 || walk_begin < 0 || walk_count < 0) return N2V_ERR_INVALID_ARG;
  if (n_starts > INT64_MAX / r) return N2V_ERR_INVALID_ARG;
  const int64_t total = n_starts * (int64_t)r;
  if (walk_begin > total || walk_count > total - walk_begin) return N2V_ERR_INVALID_ARG;
  uint32_t a_p, a_q;
  if (n2v_alpha_q16(p, q, &a_p, &a_q) != N2V_OK) return N2V_ERR_INVALID_ARG;
  const uint64_t amax = std::max<uint64_t>(std::max<uint64_t>(a_p, a_q), kAlphaOne);
  if (g->info.max_wsum > UINT64_MAX / amax) return N2V_ERR_OVERFLOW;
  if (walk_count == 0) return N2V_OK;
  if (!starts || !walks) return N2V_ERR_INVALID_ARG;
  const int64_t chunks = n_chunks(g, walk_count);
  if (chunks > kNoAllocMaxLaunches) return N2V_ERR_NO_MEM;  // more launch counters than the scratch holds
  // the scratch used is the current device's: it must be the graph's device
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return N2V_ERR_CUDA;
  if (cur != g->device) return N2V_ERR_INVALID_ARG;
  void* scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc != N2V_OK) return rc;

  LaunchCfg L = resolve_launch(g, N2V_PERSISTENT);
  const int smem = smem_per_block(L);
  // the spill area is whatever the scratch has left, shared evenly by the warps
  const int64_t warps = (int64_t)L.blocks * (L.block_threads / 32);
  const int64_t per_warp = (int64_t)((kNoAllocScratchBytes - kNoAllocCounterBytes) / sizeof(uint32_t)) / warps;
  L.spill_specials = (int)std::min<int64_t>(L.spill_specials, per_warp);
  unsigned long long* counters = (unsigned long long*)scratch;
  uint32_t* spill = L.spill_specials > 0 ? (uint32_t*)((char*)scratch + kNoAllocCounterBytes) : nullptr;

  cudaStream_t s = (cudaStream_t)stream;
  // the scratch keeps the previous call's contents: the counters must start at 0
  if (cudaMemsetAsync(counters, 0, sizeof(unsigned long long) * (size_t)chunks, s) != cudaSuccess)
    return N2V_ERR_CUDA;
  WalkJob J;
  J.starts = starts;
  J.n_starts = n_starts;
  J.l = l;
  J.a_p = a_p;
  J.a_q = a_q;
  J.seed = seed;
  J.status = g->status;
  J.approx = 0;
  J.approx_eps = 0.0;
  J.approx_popular = 0;
  J.w_min = g->info.w_min;
  J.w_max = g->info.w_max;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(persistent_fn(L, g->view, J), cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  const int64_t per = chunks == 1 ? walk_count : g->tune.chunk_walkers;
  for (int64_t ci = 0; ci < chunks; ++ci) {
    const int64_t lo = ci * per;
    J.walk_begin = walk_begin + lo;
    J.count = std::min<int64_t>(per, walk_count - lo);
    J.walks = walks + lo * (int64_t)l;
    launch_persistent(L, smem, s, g->view, J, counters + ci, spill);
  }
  return cudaGetLastError() == cudaSuccess ? N2V_OK : N2V_ERR_CUDA;
}
