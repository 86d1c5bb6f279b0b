// Internal declarations and device primitives of the GB300 node2vec sampler.
//
// Shared by the graph set-up, the samplers and the serving loop.  Nothing here
// is visible through the C ABI (include/n2v.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "n2v.h"

namespace n2v {

constexpr uint32_t kAlphaOne = 65536u;  // alpha = 1 in Q16
constexpr unsigned kFull = 0xffffffffu;

// device status word bits
constexpr uint32_t kStInvalidArg = 1u;
constexpr uint32_t kStTimeout = 2u;
constexpr uint32_t kStInternal = 4u;  // a self-check of the checked build failed

// Device self-checks of the checked build (compiled with -DN2V_CHECKED):
// a failed check sets kStInternal in the status word of the graph and the
// kernel carries on -- no trap, no assert.  Compiled out otherwise.
#ifdef N2V_CHECKED
#define N2V_CHECK(g, cond)                                       \
  do {                                                           \
    if (!(cond)) atomicOr((g).status, ::n2v::kStInternal);      \
  } while (0)
#else
#define N2V_CHECK(g, cond) \
  do {                     \
  } while (0)
#endif

// Step statistics of the stats build (compiled with -DN2V_STATS): lane 0 of a
// warp adds counts, SM clock cycles and list lengths per kind of step to a
// device array that n2v_step_stats reads.  Compiled out otherwise.
enum : int {
  kStatLaneSteps = 0,    // warp-batches of lane-tier work, and their cycles
  kStatLaneCycles = 1,
  kStatFirst = 2,        // first steps (k = 0) on a warp, and cycles
  kStatFirstCycles = 3,
  kStatMode = 4,         // + 4m: warp steps of generator mode m (0..4), cycles, shorter and longer lengths
  kStatSegments = 24,    // re-enumerations of a step's specials (segments beyond the first)
  kStatSpilled = 25,     // steps whose specials overflowed shared memory
  kStatKernelCycles = 26,  // sum over warps of their time in the persistent loop
  kStatChunks = 27,        // staged steps: chunks of 64 keys
  kStatWindows = 28,       // staged steps: windows landed
  kStatSearches = 29,      // staged steps: window searches (a chunk's keys in one window)
  kStatWords = 32
};
#ifdef N2V_STATS
// one array per translation unit (no relocatable device code); n2v_step_stats reads the samplers'
static __device__ unsigned long long g_step_stats[kStatWords];
#define N2V_STAT(i, x) atomicAdd(&::n2v::g_step_stats[(i)], (unsigned long long)(x))
#else
#define N2V_STAT(i, x) \
  do {                  \
  } while (0)
#endif

// Read-only view of a resident graph plus its auxiliary structures.
struct GraphView {
  const int64_t* __restrict__ rp;      // [n+1]
  const int32_t* __restrict__ col;     // [nnz]
  const uint32_t* __restrict__ w;      // [nnz] or null (unweighted)
  const uint64_t* __restrict__ wpre;   // [nnz] row-local inclusive prefix of w (weighted only)
  int64_t n;
  int64_t nnz;
  // hashed neighbour sets of hub vertices (FN-Cache analogue); hub_of null = none
  const int32_t* __restrict__ hub_of;    // [n] hub slot or -1
  const int64_t* __restrict__ hub_off;   // [H] first slot of the hub's table
  const uint32_t* __restrict__ hub_bits; // [H] log2 of the table size
  const int2* __restrict__ hub_slot;     // [slots] (neighbour id or -1 if empty, index in the hub's row)
  int64_t hub_min_deg;                   // smallest degree of a hub with a hashed set
  // rank bitmaps of the largest hubs (FN-Cache analogue); bm_data null = none.  Entry
  // bm_data[h * bm_words + (x >> 6)] holds bits 64*(x>>6) .. +63 of N(hub h) as a
  // 64-bit mask (.x low, .y high) and in .z the number of neighbours below 64*(x>>6).
  const uint4* __restrict__ bm_data;     // [bitmap hubs][bm_words]
  const int2* __restrict__ bm_tab;       // [2^bm_bits] (hub vertex or -1, bitmap index)
  int64_t bm_words;                      // ceil(n / 64)
  int64_t bm_min_deg;                    // smallest degree of a bitmap hub
  uint32_t bm_bits;
  uint32_t* status;                      // the graph's device status word (self-checks)
};

// One walk job slice, as every sampler sees it.
struct WalkJob {
  const int32_t* starts;
  int64_t n_starts;
  int64_t walk_begin;  // first walk id of this slice
  int64_t count;       // walks in this slice
  int32_t l;
  uint32_t a_p, a_q;
  uint64_t seed;
  int32_t* walks;      // [count][l]
  uint32_t* status;
  // FN-Approx (Section 3.4): off when approx == 0
  int approx;
  double approx_eps;
  int64_t approx_popular;  // popular: degree >= this
  uint32_t w_min, w_max;   // extreme edge weights of the graph
};

// Threads per block of the persistent kernels (the sampler and the serving tick).
constexpr int kPersistThreads = 128;

// Tuning resolved for a launch.
struct LaunchCfg {
  int block_threads;
  int blocks;
  int thread_max_deg;
  int smem_specials;   // per warp
  int stage_window;    // per warp: elements of each of the two staging windows (0 = no staging)
  int stream_ratio;    // x10
  int spill_specials;  // per warp, in the device workspace (persistent sampler only)
  int stage_buffers;   // staging windows per warp (2 or 4)
  int minb;            // persistent kernel instance: resident 128-thread blocks per SM it is compiled for
  int block_min_deg;   // persistent sampler: 0 = warps independent; > 0 = block batches with a block tier
  int merge_ratio;     // x10, merge form of short steps (0: off)
  size_t l2_persist_bytes;  // bytes at the start of col marked persisting in L2 (0: off)
};

// Instances of the persistent kernels.  The lean ones run exact walks without
// hub caches or the merge form, so that the step they inline carries only the
// probe and staged generators (fewer live registers, fewer spills);
// kPersistLeanUnw is for graphs without weights and knows that at compile time.
enum PersistKind { kPersistFull = 0, kPersistLean = 1, kPersistLeanUnw = 2 };

// The instance an exact-walk launch under L over graph view g can take.
__host__ __forceinline__ int persist_kind(const LaunchCfg& L, const GraphView& g) {
  if (L.merge_ratio != 0 || g.hub_of != nullptr || g.bm_data != nullptr) return kPersistFull;
  return g.w ? kPersistLean : kPersistLeanUnw;
}

// Inside a kPersistLeanUnw kernel: the view's weights are null already (the
// host picks that instance only then); stating it lets the compiler drop the
// weighted code paths.
__device__ __forceinline__ void fold_unweighted(GraphView& g) {
  g.w = nullptr;
  g.wpre = nullptr;
}

// Shared memory of one warp: four mbarrier slots (32 bytes), the specials
// buffer (smem_specials uint32), then stage_buffers staging windows of
// stage_window + 8 int32 each (16-byte aligned).
__host__ __device__ __forceinline__ int warp_smem_bytes(const LaunchCfg& c) {
  const int win = c.stage_window > 0 ? c.stage_buffers * (c.stage_window + 8) * 4 : 0;
  return 32 + c.smem_specials * 4 + win;
}

// ---------------------------------------------------------------------------
// mbarrier and TMA bulk-copy primitives (inline PTX, sm_90+ / sm_103a).

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
// One-dimensional bulk copy global -> shared, completing `bytes` transactions
// on `bar`.  dst, src and bytes must be multiples of 16.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase with the given parity to complete, giving up after
// `limit` SM clock cycles (default about two seconds; returns false then).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit = (1ll << 32)) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}

// Drop the 128-byte L2 line at p (128-byte aligned) without writing it back:
// its data becomes undefined.  For scratch that is dead once read.
__device__ __forceinline__ void discard_l2_line(const void* p) {
  asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the
// multiply-xor bijection with the key advanced by the Weyl increments between
// rounds.  Key = (lo32 seed, hi32 seed); counter = (k, lo32 id, hi32 id, 0);
// the 64-bit draw is out[1] << 32 | out[0].
__device__ __forceinline__ uint64_t philox_draw(uint64_t seed, uint64_t walk_id, uint32_t k) {
  uint32_t x0 = k, x1 = (uint32_t)walk_id, x2 = (uint32_t)(walk_id >> 32), x3 = 0u;
  uint32_t key0 = (uint32_t)seed, key1 = (uint32_t)(seed >> 32);
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
    uint32_t hi0 = __umulhi(m0, x0), lo0 = m0 * x0;
    uint32_t hi1 = __umulhi(m1, x2), lo1 = m1 * x2;
    uint32_t y0 = hi1 ^ x1 ^ key0;
    uint32_t y2 = hi0 ^ x3 ^ key1;
    x0 = y0;
    x1 = lo1;
    x2 = y2;
    x3 = lo0;
    key0 += 0x9E3779B9u;
    key1 += 0xBB67AE85u;
  }
  return ((uint64_t)x1 << 32) | (uint64_t)x0;
}

// floor(u * T / 2^64)
__device__ __forceinline__ uint64_t scale_draw(uint64_t u, uint64_t T) { return __umul64hi(u, T); }

// First index i in [0, n) with a[i] >= key (n if none).
__device__ __forceinline__ int64_t lower_bound_i32(const int32_t* __restrict__ a, int64_t n, int32_t key) {
  int64_t lo = 0;
  while (n > 0) {
    int64_t half = n >> 1;
    if (__ldg(a + lo + half) < key) {
      lo += half + 1;
      n -= half + 1;
    } else {
      n = half;
    }
  }
  return lo;
}

__device__ __forceinline__ bool contains_i32(const int32_t* __restrict__ a, int64_t n, int32_t key) {
  int64_t i = lower_bound_i32(a, n, key);
  return i < n && __ldg(a + i) == key;
}

// T = sum over N(v) of w(v,x) * alpha(t,x) by a merge over N(v) and N(t) (one
// lane, O(deg v + deg t)): the checked build recomputes stored totals with it.
__device__ __forceinline__ uint64_t merge_total(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                const uint32_t* __restrict__ w, int64_t t, int64_t v, uint32_t a_p,
                                                uint32_t a_q) {
  const int64_t bv = rp[v], ev = rp[v + 1], bt = rp[t], et = rp[t + 1];
  uint64_t T = 0;
  int64_t pt = bt;
  for (int64_t j = bv; j < ev; ++j) {
    const int32_t x = col[j];
    while (pt < et && col[pt] < x) ++pt;
    const uint32_t a = (int64_t)x == t ? a_p : ((pt < et && col[pt] == x) ? 65536u : a_q);
    T += (uint64_t)(w ? w[j] : 1u) * a;
  }
  return T;
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}

__device__ __forceinline__ uint64_t warp_incl_scan_u64(uint64_t x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint64_t y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// First index j in [lo, hi] with a[j] > key, given a non-decreasing a and
// a[hi] > key.  Whole warp, 32-ary search.
__device__ __forceinline__ int64_t warp_first_above_u64(const uint64_t* __restrict__ a, int64_t lo,
                                                        int64_t hi, uint64_t key, int lane) {
  while (hi - lo + 1 > 32) {
    int64_t step = (hi - lo + 32) / 32;  // ceil(len / 32)
    int64_t p = lo + (int64_t)(lane + 1) * step - 1;
    if (p > hi) p = hi;
    unsigned m = __ballot_sync(kFull, __ldg(a + p) > key);
    if (!m) return hi;     // lane 31 probes hi, so this only happens if a[hi] <= key
    int f = __ffs(m) - 1;
    int64_t pf = __shfl_sync(kFull, p, f);
    int64_t pprev = __shfl_sync(kFull, p, f > 0 ? f - 1 : 0);
    hi = pf;
    if (f > 0) lo = pprev + 1;
  }
  int64_t p = lo + lane;
  unsigned m = __ballot_sync(kFull, p <= hi && __ldg(a + p) > key);
  return m ? lo + (__ffs(m) - 1) : hi;
}

}  // namespace n2v

// Host-side handle.
struct n2v_graph {
  n2v::GraphView view;
  int64_t n, nnz;
  int weighted;
  void* aux;
  size_t aux_bytes;
  uint32_t* status;        // device status word
  unsigned long long* scratch;  // device scratch words inside aux
  n2v_tune tune;
  n2v_tune tune_loaded;    // the tuning aux was laid out for (n2v_graph_load)
  n2v_graph_info info;
  int device;
  int sms;
  void* graph_cache;       // recorded CUDA graphs (opaque, see n2v_walk.cu)
};

namespace n2v {

// Fibonacci hashing of a vertex id into a table of 2^bits slots.
__host__ __device__ __forceinline__ uint32_t hub_hash(int32_t x, uint32_t bits) {
  return ((uint32_t)x * 2654435769u) >> (32u - bits);
}

// Index of x inside the CSR row of hub h, or -1 when x is not a neighbour.
// Linear probing over a table at most half full; every probe sequence ends at
// an empty slot or at x, and is additionally bounded by the table size.
__device__ __forceinline__ int32_t hub_find(const GraphView& g, int32_t h, int32_t x) {
  const int2* __restrict__ tab = g.hub_slot + g.hub_off[h];
  const uint32_t bits = g.hub_bits[h];
  const uint32_t mask = (1u << bits) - 1u;
  uint32_t s = hub_hash(x, bits);
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    int2 e = __ldg(tab + s);
    if (e.x == x) return e.y;
    if (e.x < 0) return -1;
    s = (s + 1u) & mask;
  }
  return -1;
}

// Bitmap index of hub vertex v, or -1 (open addressing, table at most half full).
__device__ __forceinline__ int32_t bm_find(const GraphView& g, int32_t v) {
  const uint32_t mask = (1u << g.bm_bits) - 1u;
  uint32_t s = hub_hash(v, g.bm_bits);
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    const int2 e = __ldg(g.bm_tab + s);
    if (e.x == v) return e.y;
    if (e.x < 0) return -1;
    s = (s + 1u) & mask;
  }
  return -1;
}

// Index of x inside the CSR row of bitmap hub h, or -1 when x is not a
// neighbour: one 16-byte load, a bit test and a population count.
__device__ __forceinline__ int32_t bm_pos(const GraphView& g, int32_t h, int32_t x) {
  const uint4 e = __ldg(g.bm_data + (int64_t)h * g.bm_words + (x >> 6));
  const uint64_t bits = ((uint64_t)e.y << 32) | (uint64_t)e.x;
  const int b = x & 63;
  if (!((bits >> b) & 1ull)) return -1;
  return (int32_t)e.z + __popcll(bits & ((1ull << b) - 1ull));
}

// Layout of the caller's auxiliary buffer (byte offsets, 256-aligned).
struct AuxLayout {
  size_t status, scratch, wpre, hub_of, hub_off, hub_bits, hub_vtx, hub_slot, bm_tab, bm_vtx, bm_data, total;
  int64_t hubs_cap, slots_cap, bm_cap, bm_words;
  uint32_t bm_bits;
};
AuxLayout aux_layout(int64_t n, int64_t nnz, int weighted, const n2v_tune& t);

// scratch word indices (unsigned long long) inside the aux scratch block
enum : int {
  kScBad = 0,
  kScMaxDeg = 1,
  kScMaxWsum = 2,
  kScHubCount = 3,
  kScSlotCount = 4,
  kScHist = 8,  // 34 words
  kScWMin = 42,
  kScWMax = 43,
  kScSumDeg2 = 44,  // sum over edges of deg(target): entries of a stored transition table
  kScBmCount = 45,  // bitmap hubs assigned
  kScWords = 64
};

// FN-Approx decision (Section 3.4, Eq. 2-3) for a step at v (degree dv)
// reached from t (degree dt): bounds on the probability of any x != t,
// evaluated in IEEE double with one rounding per operation in a fixed order
// (the _rn intrinsics forbid contraction), so that every implementation of
// the same formula takes the same branch.  The bounds assume t is a
// neighbour of v (undirected graphs).
__device__ __forceinline__ bool approx_decide(int64_t dv, int64_t dt, uint32_t a_p, uint32_t a_q, uint32_t w_min,
                                              uint32_t w_max, double eps) {
  const double ip = __ddiv_rn((double)a_p, 65536.0);
  const double iq = __ddiv_rn((double)a_q, 65536.0);
  const double wmin = (double)w_min, wmax = (double)w_max;
  const double others = (double)(dv - 1);
  const double cmax = (double)(dt < dv - 1 ? dt : dv - 1);
  const double num_min = __dmul_rn(wmin, iq < 1.0 ? iq : 1.0);
  const double num_max = __dmul_rn(wmax, iq < 1.0 ? 1.0 : iq);
  const double all_q = __dadd_rn(ip, __dmul_rn(others, iq));
  const double most_1 = __dadd_rn(__dadd_rn(ip, cmax), __dmul_rn(__dsub_rn(others, cmax), iq));
  const double den_min = __dmul_rn(wmin, iq >= 1.0 ? most_1 : all_q);
  const double den_max = __dmul_rn(wmax, iq >= 1.0 ? all_q : most_1);
  const double lb = __ddiv_rn(num_min, den_max);
  const double ub = __ddiv_rn(num_max, den_min);
  return __dsub_rn(ub, lb) < eps;
}

// n2v_walk.cu
LaunchCfg resolve_launch(const n2v_graph* g, int variant);
void* new_graph_cache();
void clear_graph_cache(n2v_graph* g);
void free_graph_cache(n2v_graph* g);
}  // namespace n2v
