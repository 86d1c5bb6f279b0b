// Exact node2vec step functions (device side).
//
// Every function here returns the same vertex for the same (t, v, k, u): the
// first neighbour x of v in CSR order whose inclusive prefix of
// c_x = w(v,x) * alpha(t,x) exceeds r = floor(u * T / 2^64), T = sum of c_x
// (Section 2.1 model, Section 3.2 on-demand computation), or -1 when T == 0.
// They differ only in how much of N(v) and N(t) they touch.
#pragma once

#include "n2v_internal.cuh"

namespace n2v {

// ---------------------------------------------------------------------------
// One lane, full scan (the form of Section 3.2: scan N(v), test each x for
// membership in N(t)).  Both lists are sorted, so the membership test is a
// merge pointer that walks N(t) once: O(deg v + deg t) per pass, two passes
// (total, then selection).
__device__ __forceinline__ int32_t thread_step(const GraphView& g, int64_t t, int64_t v, int k, uint64_t u,
                                               uint32_t a_p, uint32_t a_q) {
  const int64_t bv = g.rp[v], ev = g.rp[v + 1];
  if (ev == bv) return -1;
  const int32_t* __restrict__ col = g.col;
  if (k == 0) {
    if (!g.w) return __ldg(col + bv + (int64_t)scale_draw(u, (uint64_t)(ev - bv)));
    uint64_t T = 0;
    for (int64_t j = bv; j < ev; ++j) T += __ldg(g.w + j);
    if (T == 0) return -1;
    const uint64_t r = scale_draw(u, T);
    uint64_t C = 0;
    for (int64_t j = bv; j < ev; ++j) {
      C += __ldg(g.w + j);
      if (C > r) return __ldg(col + j);
    }
    return -1;
  }
  const int64_t bt = g.rp[t], et = g.rp[t + 1];
  uint64_t T = 0;
  int64_t pt = bt;
  for (int64_t j = bv; j < ev; ++j) {
    const int32_t x = __ldg(col + j);
    while (pt < et && __ldg(col + pt) < x) ++pt;
    const uint32_t a = ((int64_t)x == t) ? a_p : ((pt < et && __ldg(col + pt) == x) ? kAlphaOne : a_q);
    T += (uint64_t)(g.w ? __ldg(g.w + j) : 1u) * a;
  }
  if (T == 0) return -1;
  const uint64_t r = scale_draw(u, T);
  uint64_t C = 0;
  pt = bt;
  for (int64_t j = bv; j < ev; ++j) {
    const int32_t x = __ldg(col + j);
    while (pt < et && __ldg(col + pt) < x) ++pt;
    const uint32_t a = ((int64_t)x == t) ? a_p : ((pt < et && __ldg(col + pt) == x) ? kAlphaOne : a_q);
    C += (uint64_t)(g.w ? __ldg(g.w + j) : 1u) * a;
    if (C > r) return x;
  }
  return -1;
}

// ---------------------------------------------------------------------------
// Whole warp, one step.  All 32 lanes must call it with the same arguments.
//
// Only the "special" neighbours of v -- x == t (alpha = 1/p) and x in N(t)
// (alpha = 1) -- differ from the default alpha = 1/q.  Writing
//   C_j = a_q * W_j + D_j,   W_j = static prefix of w over N(v) up to j,
//   D_j = sum over specials s <= j of (alpha_s - a_q) * w_s   (mod 2^64),
// the total is T = a_q * W_last + D_last, and between two specials C is a_q
// times the static prefix plus a constant, so the first j with C_j > r is
// found from the specials alone plus one division (unweighted) or one search
// of the static prefix (weighted).  All arithmetic is modulo 2^64; every true
// prefix lies in [0, T] < 2^64, so the modular values are the exact ones.
//
// The specials are N(v) intersected with S = N(t) + {t}.  A generator emits
// them in increasing position, 32 candidates per call of its callback (one
// per lane), in one of two ways:
//   probe -- walk the shorter list; find each element in the longer one by
//            binary search in global memory (or the hashed set of a hub):
//            about ceil(short/32) * log2(long) dependent loads;
//   stage -- stream the longer list through two shared-memory windows filled
//            by TMA bulk copies (double-buffered) and binary-search the
//            shorter list's elements inside the resident window: the bytes
//            of the longer list move without instructions, and every probe is
//            a shared-memory access.
// Both give the same specials, so the choice only changes speed.

struct WarpSmem {
  uint64_t* bar;     // one mbarrier per staging window
  uint32_t* spec;    // cap entries: pos | class << 30
  int cap;
  int32_t* win;      // nbuf windows of (wlen + 8) int32, 16-byte aligned
  int wlen;          // elements per window (0 = no staging)
  int nbuf;          // windows in flight (2 or 4)
  uint32_t* spill;   // per-warp device workspace for specials beyond cap (may be null)
  int spill_cap;
  uint32_t parity;   // bit b: parity of the next phase of bar[b]
  bool timed_out;    // a bounded wait gave up
  int merge_ratio;   // x10: merge both lists when deg v + deg t <= merge_ratio/10 * the probe cost (0: never)
  uint32_t inv_q;    // the a_q that aq_inv belongs to (0: none yet)
  uint64_t aq_inv;   // floor((2^64 - 1) / inv_q)
};

// floor(x / d) for d = sm.inv_q, by a multiply with the cached reciprocal
// floor((2^64 - 1) / d): the estimate umulhi(x, inv) is floor(x / d) or one
// less, and one comparison corrects it.  The reciprocal is computed once per
// warp and value of d (uniform in the warp).
__device__ __forceinline__ uint64_t div_aq(WarpSmem& sm, uint64_t x, uint32_t d) {
  if (sm.inv_q != d) {
    sm.inv_q = d;
    sm.aq_inv = ~0ull / (uint64_t)d;
  }
  uint64_t q = __umul64hi(x, sm.aq_inv);
  if (x - q * (uint64_t)d >= (uint64_t)d) ++q;
  return q;
}

__device__ __forceinline__ WarpSmem warp_smem(unsigned char* base, int warp, const LaunchCfg& L, uint32_t* spill) {
  WarpSmem w;
  unsigned char* p = base + (size_t)warp * warp_smem_bytes(L);
  w.bar = (uint64_t*)p;
  w.spec = (uint32_t*)(p + 32);
  w.cap = L.smem_specials;
  w.win = (int32_t*)(p + 32 + L.smem_specials * 4);
  w.wlen = L.stage_window;
  w.nbuf = L.stage_buffers;
  w.spill = spill;
  w.spill_cap = spill ? L.spill_specials : 0;
  w.parity = 0;
  w.timed_out = false;
  w.merge_ratio = L.stage_window > 0 ? L.merge_ratio : 0;
  w.inv_q = 0;
  w.aq_inv = 0;
  return w;
}

// Initialise this warp's mbarriers (once per kernel, whole warp).
__device__ __forceinline__ void warp_smem_init(WarpSmem& w, int lane) {
  if (w.wlen > 0 && lane == 0) {
    for (int b = 0; b < w.nbuf; ++b) mbar_init(&w.bar[b], 1);
    fence_mbar_init();
  }
  __syncwarp();
}

struct StepCtx {
  const GraphView* g;
  int64_t bv;
  int dv, dt;      // degrees (< 2^31: col is indexed by int32 vertex ids)
  const int32_t* __restrict__ nv;
  const int32_t* __restrict__ nt;
  int32_t t32;
  int ins;         // index of t inside S = N(t) + {t}
  bool has_self;   // t already in N(t) (self-loop at t)
  int slen;        // |S|
  // the candidates a generator walks, [cb, ce) of the shorter list (ce < 0: to its end),
  // and the part [lb, le) of the longer list a staging generator streams (le < 0: to its end)
  int cb, ce, lb, le;
};

// i-th element of S = N(t) + {t} (sorted, no duplicate)
__device__ __forceinline__ int32_t s_at(const StepCtx& c, int i) {
  if (c.has_self || i < c.ins) return __ldg(c.nt + i);
  return i == c.ins ? c.t32 : __ldg(c.nt + i - 1);
}

__device__ __forceinline__ int ceil_log2(int x) { return x <= 1 ? 0 : 32 - __clz(x - 1); }

// First index i in [0, n) with a[i] >= key (n if none); 32-bit lengths.
__device__ __forceinline__ int lower_bound32(const int32_t* __restrict__ a, int n, int32_t key) {
  int lo = 0;
  while (n > 0) {
    const int half = n >> 1;
    if (__ldg(a + lo + half) < key) {
      lo += half + 1;
      n -= half + 1;
    } else {
      n = half;
    }
  }
  return lo;
}

// Element offset of L[wi * wlen] inside its staging buffer (the copy starts at
// the 16-byte boundary below it).
__device__ __forceinline__ int stage_off(const WarpSmem& sm, const int32_t* L, int wi) {
  return (int)(((uintptr_t)(L + wi * sm.wlen) & 15) >> 2);
}

// 32-bit load from a shared-memory byte address.
__device__ __forceinline__ int32_t lds32(uint32_t addr) {
  int32_t v;
  asm volatile("ld.shared.s32 %0, [%1];" : "=r"(v) : "r"(addr));
  return v;
}

// One level of two interleaved fixed-depth searches: the positions are kept as
// shared addresses, and the level's probe offset 4 (ST - 1) is an immediate of
// the load, so that a level is one load, one compare and one add per key.
template <int ST>
struct WindowLevels {
  __device__ __forceinline__ static void run(uint32_t& p0, uint32_t& p1, int32_t key0, int32_t key1) {
    int32_t v0, v1;
    asm volatile("ld.shared.s32 %0, [%1+%2];" : "=r"(v0) : "r"(p0), "n"(4 * (ST - 1)));
    asm volatile("ld.shared.s32 %0, [%1+%2];" : "=r"(v1) : "r"(p1), "n"(4 * (ST - 1)));
    p0 += v0 < key0 ? 4u * ST : 0u;
    p1 += v1 < key1 ? 4u * ST : 0u;
    WindowLevels<ST / 2>::run(p0, p1, key0, key1);
  }
};
template <>
struct WindowLevels<0> {
  __device__ __forceinline__ static void run(uint32_t&, uint32_t&, int32_t, int32_t) {}
};

// Number of window slots below key0 and key1 among the first W - 1 of a sorted
// window of W slots (W a power of two; slots past the data hold +inf) at shared
// address base: two interleaved fixed-depth searches, fully unrolled.
template <int W>
__device__ __forceinline__ void window_rank2(uint32_t base, int32_t key0, int32_t key1, int& lo0, int& lo1) {
  uint32_t p0 = base, p1 = base;
  WindowLevels<W / 2>::run(p0, p1, key0, key1);
  lo0 = (int)((p0 - base) >> 2);
  lo1 = (int)((p1 - base) >> 2);
}

// The same search over a window of depth slots (a power of two): unrolled for
// full 1024-element windows, a loop for every other depth.
__device__ __forceinline__ void window_rank2_any(int depth, uint32_t base, int32_t key0, int32_t key1, int& lo0,
                                                 int& lo1) {
  if (depth == 1024) {
    window_rank2<1024>(base, key0, key1, lo0, lo1);
    return;
  }
  int a = 0, b = 0;
  for (int st = depth >> 1; st > 0; st >>= 1) {
    const int32_t v0 = lds32(base + 4u * (uint32_t)(a + st - 1));
    const int32_t v1 = lds32(base + 4u * (uint32_t)(b + st - 1));
    a += v0 < key0 ? st : 0;
    b += v1 < key1 ? st : 0;
  }
  lo0 = a;
  lo1 = b;
}

// Fill staging buffer b with src[0, cnt) (0 < cnt <= wlen): the 16-byte-aligned
// body by one TMA bulk copy, the ragged tail that would read past the
// 16-byte-aligned end of col by plain loads.  The data starts at element
// ((uintptr_t)src & 15) / 4 of the buffer; the copy completes on bar[b].
__device__ __forceinline__ void stage_fill(WarpSmem& sm, const GraphView& g, const int32_t* src, int cnt, int b,
                                           int lane) {
  int32_t* buf = sm.win + b * (sm.wlen + 8);
  const uintptr_t a = (uintptr_t)src, e = (uintptr_t)(src + cnt);
  const uintptr_t a16 = a & ~(uintptr_t)15;
  uintptr_t e16 = (e + 15) & ~(uintptr_t)15;
  const uintptr_t lim = (uintptr_t)(g.col + g.nnz) & ~(uintptr_t)15;  // never read past the end of col
  if (e16 > lim) e16 = lim;
  const uint32_t bytes = e16 > a16 ? (uint32_t)(e16 - a16) : 0u;
  const int off = (int)((a - a16) >> 2);
  const int tail0 = bytes ? (int)((e16 - a) >> 2) : 0;  // first element not covered by the copy
  N2V_CHECK(g, bytes <= (uint32_t)(sm.wlen + 8) * 4u && off + cnt <= sm.wlen + 8 && cnt > 0);
  for (int i = tail0 + lane; i < cnt; i += 32) buf[off + i] = __ldg(src + i);
  __syncwarp();
  if (lane == 0) {
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&sm.bar[b], bytes);
    if (bytes) bulk_copy_g2s(buf, (const void*)a16, bytes, &sm.bar[b]);
  }
}

// Fill staging window wi of list L (length llen) into buffer wi % nbuf.
__device__ __forceinline__ void stage_issue(WarpSmem& sm, const GraphView& g, const int32_t* L, int llen, int wi,
                                            int lane) {
  stage_fill(sm, g, L + wi * sm.wlen, min(sm.wlen, llen - wi * sm.wlen), wi & (sm.nbuf - 1), lane);
}

__device__ __forceinline__ void stage_wait(WarpSmem& sm, int b) {
  if (!mbar_wait_bounded(&sm.bar[b], (sm.parity >> b) & 1u)) sm.timed_out = true;
  sm.parity ^= 1u << b;
  __syncwarp();
}

// Where the specials of a step go: ordinals [skip, skip + cap + spill_cap)
// are kept (shared memory first, then the warp's spill area); every special
// adds its correction (alpha - a_q) * w to the lane's partial sum.
struct SpecialSink {
  int cnt;          // specials seen so far (uniform)
  int ord_t;        // ordinal of the special x == t (class 2), or -1
  uint64_t dpart;   // this lane's share of sum (alpha - a_q) * w
  int skip;
  int cap;          // shared-memory slots
  int keep;         // cap + spill slots
  int lim;          // deg v: positions lie in [0, lim)
};

__device__ __forceinline__ uint64_t special_delta(const GraphView& g, int64_t bv, int32_t pos, uint32_t cls, uint32_t a_p,
                                                  uint32_t a_q) {
  if (!cls) return 0ull;
  const uint64_t a = cls == 2u ? (uint64_t)a_p : (uint64_t)kAlphaOne;
  const uint64_t wt = g.w ? (uint64_t)__ldg(g.w + bv + pos) : 1ull;
  return (a - (uint64_t)a_q) * wt;
}

__device__ __forceinline__ void sink_emit(SpecialSink& k, WarpSmem& sm, const GraphView& g, int64_t bv, int32_t pos,
                                          uint32_t cls, uint32_t a_p, uint32_t a_q, int lane) {
  // unweighted: a special's correction depends only on its class, so the
  // total comes from the class counts instead of a per-lane sum
  if (g.w) k.dpart += special_delta(g, bv, pos, cls, a_p, a_q);
  const unsigned m = __ballot_sync(kFull, cls != 0u);
  const unsigned m2 = __ballot_sync(kFull, cls == 2u);
  if (m2) k.ord_t = k.cnt + __popc(m & ((1u << (__ffs(m2) - 1)) - 1u));
  if (cls) {
    const int ord = k.cnt + __popc(m & lanemask_lt()) - k.skip;
    N2V_CHECK(g, pos >= 0 && pos < k.lim);
    if (ord >= 0 && ord < k.keep) {
      const uint32_t e = (uint32_t)pos | (cls << 30);
      if (ord < k.cap) {
        sm.spec[ord] = e;
      } else {
        N2V_CHECK(g, sm.spill != nullptr && ord - k.cap < sm.spill_cap);
        sm.spill[ord - k.cap] = e;
      }
    }
  }
  k.cnt += __popc(m);
}

// Keep special `pos` (class cls) at ordinal ord of the step (before the skip).
__device__ __forceinline__ void sink_store(SpecialSink& k, WarpSmem& sm, const GraphView& g, int32_t pos,
                                           uint32_t cls, int ord) {
  ord -= k.skip;
  N2V_CHECK(g, pos >= 0 && pos < k.lim);
  if (ord >= 0 && ord < k.keep) {
    const uint32_t e = (uint32_t)pos | (cls << 30);
    if (ord < k.cap) {
      sm.spec[ord] = e;
    } else {
      N2V_CHECK(g, sm.spill != nullptr && ord - k.cap < sm.spill_cap);
      sm.spill[ord - k.cap] = e;
    }
  }
}

// sink_emit for the two candidate sets of a chunk at once (set 1 follows set 0
// in position order; has1: set 1 exists, uniform).  The x == t special can be
// in the chunk only when maybe_t (uniform); then one vote finds it.
__device__ __forceinline__ void sink_emit2(SpecialSink& k, WarpSmem& sm, const GraphView& g, int64_t bv, int32_t pos0,
                                           uint32_t cls0, int32_t pos1, uint32_t cls1, bool has1, bool maybe_t,
                                           uint32_t a_p, uint32_t a_q, int lane) {
  if (g.w) k.dpart += special_delta(g, bv, pos0, cls0, a_p, a_q) + special_delta(g, bv, pos1, cls1, a_p, a_q);
  const unsigned m0 = __ballot_sync(kFull, cls0 != 0u);
  const unsigned m1 = has1 ? __ballot_sync(kFull, cls1 != 0u) : 0u;
  const int n0 = __popc(m0);
  if (maybe_t) {
    const unsigned t0 = __ballot_sync(kFull, cls0 == 2u), t1 = __ballot_sync(kFull, cls1 == 2u);
    if (t0) k.ord_t = k.cnt + __popc(m0 & ((1u << (__ffs(t0) - 1)) - 1u));
    else if (t1) k.ord_t = k.cnt + n0 + __popc(m1 & ((1u << (__ffs(t1) - 1)) - 1u));
  }
  const unsigned lt = lanemask_lt();
  if (cls0) sink_store(k, sm, g, pos0, cls0, k.cnt + __popc(m0 & lt));
  if (cls1) sink_store(k, sm, g, pos1, cls1, k.cnt + n0 + __popc(m1 & lt));
  k.cnt += n0 + __popc(m1);
}

// Enumerate the specials of the step in increasing position into `k`.
// mode 0: probe over N(v) (membership in N(t)); 1: probe over S (position in
// N(v)); 2: stage N(v), candidates S; 3: stage N(t), candidates N(v).
// hub >= 0: the longer list is that hub's hashed set; bm >= 0: it has a rank
// bitmap (the probe modes only).
__device__ __forceinline__ void gen_specials(StepCtx& c, int mode, int32_t hub, int32_t bm, WarpSmem& sm,
                                             SpecialSink& k, uint32_t a_p, uint32_t a_q, int lane) {
  const GraphView& g = *c.g;
  if (mode == 0 && bm >= 0) {
    // N(t) is a bitmap hub: two independent one-load membership tests per lane and chunk
    const int ce = c.ce < 0 ? c.dv : c.ce;
    for (int c0 = c.cb; c0 < ce; c0 += 64) {
      const int i0 = c0 + lane, i1 = c0 + 32 + lane;
      const int32_t x0 = i0 < ce ? __ldg(c.nv + i0) : 0;
      const int32_t x1 = i1 < ce ? __ldg(c.nv + i1) : 0;
      const bool in0 = i0 < ce && bm_pos(g, bm, x0) >= 0;
      const bool in1 = i1 < ce && bm_pos(g, bm, x1) >= 0;
      const bool sp0 = i0 < ce && (x0 == c.t32 || in0);
      const bool sp1 = i1 < ce && (x1 == c.t32 || in1);
      sink_emit(k, sm, g, c.bv, sp0 ? i0 : -1, sp0 ? (x0 == c.t32 ? 2u : 1u) : 0u, a_p, a_q, lane);
      if (c0 + 32 < ce) sink_emit(k, sm, g, c.bv, sp1 ? i1 : -1, sp1 ? (x1 == c.t32 ? 2u : 1u) : 0u, a_p, a_q, lane);
    }
    return;
  }
  if (mode == 1 && bm >= 0) {
    // N(v) is a bitmap hub: each element of S = N(t) + {t} finds its index in N(v) by one load
    const int ce = c.ce < 0 ? c.slen : c.ce;
    for (int c0 = c.cb; c0 < ce; c0 += 64) {
      const int i0 = c0 + lane, i1 = c0 + 32 + lane;
      const int32_t y0 = i0 < ce ? s_at(c, i0) : 0;
      const int32_t y1 = i1 < ce ? s_at(c, i1) : 0;
      const int32_t p0 = i0 < ce ? bm_pos(g, bm, y0) : -1;
      const int32_t p1 = i1 < ce ? bm_pos(g, bm, y1) : -1;
      sink_emit(k, sm, g, c.bv, p0, p0 >= 0 ? (y0 == c.t32 ? 2u : 1u) : 0u, a_p, a_q, lane);
      if (c0 + 32 < ce) sink_emit(k, sm, g, c.bv, p1, p1 >= 0 ? (y1 == c.t32 ? 2u : 1u) : 0u, a_p, a_q, lane);
    }
    return;
  }
  if (mode == 0) {
    // two candidates per lane and chunk: two independent searches in flight
    auto member = [&](int32_t x) -> bool {
      if (x == c.t32) return true;
      if (hub >= 0) return hub_find(g, hub, x) >= 0;
      const int p = lower_bound32(c.nt, c.dt, x);
      return p < c.dt && __ldg(c.nt + p) == x;
    };
    const int ce = c.ce < 0 ? c.dv : c.ce;
    for (int c0 = c.cb; c0 < ce; c0 += 64) {
      const int i0 = c0 + lane, i1 = c0 + 32 + lane;
      const int32_t x0 = i0 < ce ? __ldg(c.nv + i0) : -1;
      const int32_t x1 = i1 < ce ? __ldg(c.nv + i1) : -1;
      bool sp0 = false, sp1 = false;
      if (hub < 0) {
        // interleaved lower bounds over N(t)
        int lo0 = 0, n0 = c.dt, lo1 = 0, n1 = c.dt;
        while (n0 > 0 || n1 > 0) {
          const int h0 = n0 >> 1, h1 = n1 >> 1;
          const bool a0 = n0 > 0 && __ldg(c.nt + lo0 + h0) < x0;
          const bool a1 = n1 > 0 && __ldg(c.nt + lo1 + h1) < x1;
          if (n0 > 0) {
            lo0 = a0 ? lo0 + h0 + 1 : lo0;
            n0 = a0 ? n0 - h0 - 1 : h0;
          }
          if (n1 > 0) {
            lo1 = a1 ? lo1 + h1 + 1 : lo1;
            n1 = a1 ? n1 - h1 - 1 : h1;
          }
        }
        sp0 = i0 < ce && (x0 == c.t32 || (lo0 < c.dt && __ldg(c.nt + lo0) == x0));
        sp1 = i1 < ce && (x1 == c.t32 || (lo1 < c.dt && __ldg(c.nt + lo1) == x1));
      } else {
        sp0 = i0 < ce && member(x0);
        sp1 = i1 < ce && member(x1);
      }
      sink_emit(k, sm, g, c.bv, sp0 ? i0 : -1, sp0 ? (x0 == c.t32 ? 2u : 1u) : 0u, a_p, a_q, lane);
      if (c0 + 32 < ce) sink_emit(k, sm, g, c.bv, sp1 ? i1 : -1, sp1 ? (x1 == c.t32 ? 2u : 1u) : 0u, a_p, a_q, lane);
    }
    return;
  }
  if (mode == 1) {
    const int ce = c.ce < 0 ? c.slen : c.ce;
    for (int c0 = c.cb; c0 < ce; c0 += 32) {
      const int i = c0 + lane;
      int32_t pos = -1;
      uint32_t cls = 0;
      if (i < ce) {
        const int32_t y = s_at(c, i);
        int p;
        if (hub >= 0) {
          p = hub_find(g, hub, y);
        } else {
          p = lower_bound32(c.nv, c.dv, y);
          if (p >= c.dv || __ldg(c.nv + p) != y) p = -1;
        }
        if (p >= 0) {
          pos = p;
          cls = y == c.t32 ? 2u : 1u;
        }
      }
      sink_emit(k, sm, g, c.bv, pos, cls, a_p, a_q, lane);
    }
    return;
  }
  // stage: the longer list flows through the two windows; the candidates of
  // each chunk are searched in the resident window
  const bool stage_v = mode == 2;
  const int32_t* L = (stage_v ? c.nv : c.nt) + c.lb;
  const int llen = (c.le < 0 ? (stage_v ? c.dv : c.dt) : c.le) - c.lb;  // > 0 (the callers ensure it)
  const int W = sm.wlen;
  const int nwin = (llen + W - 1) / W;
  const int ahead = min(sm.nbuf, nwin);
  for (int q = 0; q < ahead; ++q) stage_issue(sm, g, L, llen, q, lane);
  if (stage_v && c.ins < 0) {  // t's slot in S = N(t) + {t}, searched while the copies fly
    c.ins = lower_bound32(c.nt, c.dt, c.t32);
    c.has_self = c.ins < c.dt && __ldg(c.nt + c.ins) == c.t32;
    c.slen = c.dt + (c.has_self ? 0 : 1);
  }
  const int nkeys = c.ce < 0 ? (stage_v ? c.slen : c.dv) : c.ce;  // keys [c.cb, nkeys)
  int wi = 0;
  // two keys per lane and chunk (keys kc + lane and kc + 32 + lane): two
  // independent search chains in flight per lane
  // key i (clamped into the list: keys past the end are never searched), without branches:
  // element i of S = N(t) + {t} is t at t's slot, else N(t)[i] or N(t)[i - 1]
  const int ins_e = c.has_self ? INT32_MAX : c.ins;
  auto key_at = [&](int i) -> int32_t {
    const int j = min(i, nkeys - 1);
    if (!stage_v) return __ldg(c.nv + j);
    const int32_t x = __ldg(c.nt + min(j - (j > ins_e ? 1 : 0), c.dt - 1));
    return j == ins_e ? c.t32 : x;
  };
  // search depth of a window holding cnt elements: the next power of two
  auto depth_of = [](int cnt) { return cnt <= 1 ? 1 : 1 << (32 - __clz(cnt - 1)); };
  // after a window lands: the last window is padded with +inf up to and including
  // its search depth, so that the fixed-depth search needs no bounds test and the
  // slot after any search result reads +inf (every other window is full, and a
  // key searched in it is at most its last element)
  auto land = [&](int wj) {
    if (lane == 0) N2V_STAT(kStatWindows, 1);
    stage_wait(sm, wj & (sm.nbuf - 1));
    if (wj == nwin - 1) {
      const int cnt = llen - wj * W;
      const int depth = depth_of(cnt);
      int32_t* w = sm.win + (wj & (sm.nbuf - 1)) * (sm.wlen + 8) + stage_off(sm, L, wj);
      for (int q = cnt + lane; q <= depth; q += 32) w[q] = INT32_MAX;
      __syncwarp();
    }
  };
  // keys two chunks ahead are in flight while a chunk is searched
  // the resident window: shared address, length, last element (+inf for the last window)
  uint32_t wbase = 0;
  int wcnt = 0, wdepth = 0;
  int32_t wlast = 0;
  bool wlast_inf = false;
  auto set_window = [&](int wj) {
    wbase = smem_addr(sm.win + (wj & (sm.nbuf - 1)) * (sm.wlen + 8) + stage_off(sm, L, wj));
    wcnt = min(W, llen - wj * W);
    wdepth = depth_of(wcnt);
    wlast_inf = wj == nwin - 1;
    wlast = lds32(wbase + 4u * (uint32_t)(wcnt - 1));
  };
  int32_t next0 = key_at(c.cb + lane), next1 = key_at(c.cb + 32 + lane);
  int32_t after0 = key_at(c.cb + 64 + lane), after1 = key_at(c.cb + 96 + lane);
  land(0);
  set_window(0);
  for (int kc = c.cb; kc < nkeys; kc += 64) {
    if (lane == 0) N2V_STAT(kStatChunks, 1);
    const int i0 = kc + lane, i1 = kc + 32 + lane;
    const int32_t key0 = next0, key1 = next1;
    next0 = after0;
    next1 = after1;
    after0 = key_at(i0 + 128);
    after1 = key_at(i1 + 128);
    // an element of N(v) equal to t is special whatever N(t) holds
    const bool is_t0 = i0 < nkeys && !stage_v && key0 == c.t32;
    const bool is_t1 = i1 < nkeys && !stage_v && key1 == c.t32;
    bool pend0 = i0 < nkeys && !is_t0, pend1 = i1 < nkeys && !is_t1;
    int at0 = -1, at1 = -1;  // index of the key inside L, or -1
    for (;;) {
      const bool go0 = pend0 && (wlast_inf || key0 <= wlast);
      const bool go1 = pend1 && (wlast_inf || key1 <= wlast);
      if (lane == 0) N2V_STAT(kStatSearches, 1);
      if (go0 || go1) {
        // fixed-depth searches over the power-of-two window (slots [wcnt, wdepth) hold +inf)
        int lo0, lo1;
        window_rank2_any(wdepth, wbase, key0, key1, lo0, lo1);
        N2V_CHECK(g, lo0 >= 0 && lo0 < wdepth && lo1 >= 0 && lo1 < wdepth && wcnt <= W);
        // the lower bound is lo or lo + 1: both slots in one round trip (slot lo + 1 holds
        // data, or +inf past the end of the last window)
        const int32_t x0 = lds32(wbase + 4u * lo0), y0 = lds32(wbase + 4u * (lo0 + 1));
        const int32_t x1 = lds32(wbase + 4u * lo1), y1 = lds32(wbase + 4u * (lo1 + 1));
        if (go0 && (x0 == key0 || (x0 < key0 && y0 == key0))) at0 = c.lb + wi * W + lo0 + (x0 == key0 ? 0 : 1);
        if (go1 && (x1 == key1 || (x1 < key1 && y1 == key1))) at1 = c.lb + wi * W + lo1 + (x1 == key1 ? 0 : 1);
        pend0 = pend0 && !go0;
        pend1 = pend1 && !go1;
      }
      if (!__any_sync(kFull, pend0 || pend1)) break;
      __syncwarp();
      if (wi + sm.nbuf < nwin) stage_issue(sm, g, L, llen, wi + sm.nbuf, lane);
      ++wi;
      land(wi);
      set_window(wi);
    }
    // stage N(v): the key's index in N(v), class 2 for the key t; stage N(t): the key's own
    // index, class 2 for the key t (special whatever N(t) holds)
    const bool f0 = stage_v ? at0 >= 0 : (is_t0 || at0 >= 0);
    const bool f1 = stage_v ? at1 >= 0 : (is_t1 || at1 >= 0);
    const int32_t pos0 = f0 ? (stage_v ? at0 : i0) : -1, pos1 = f1 ? (stage_v ? at1 : i1) : -1;
    const uint32_t cls0 = f0 ? (key0 == c.t32 ? 2u : 1u) : 0u, cls1 = f1 ? (key1 == c.t32 ? 2u : 1u) : 0u;
    // the key t lies in this chunk: stage N(v) knows its slot in S; stage N(t) asks the lanes
    // (t's index in S is c.ins, also when t is in N(t) through a self-loop)
    const bool maybe_t = stage_v ? (c.ins >= kc && c.ins < kc + 64) : __any_sync(kFull, is_t0 || is_t1);
    sink_emit2(k, sm, g, c.bv, pos0, cls0, pos1, cls1, kc + 32 < nkeys, maybe_t, a_p, a_q, lane);
  }
  // the windows after the current one may still be in flight
  for (int q = wi + 1; q < nwin && q <= wi + sm.nbuf - 1; ++q) stage_wait(sm, q & (sm.nbuf - 1));
}

// Static prefix W_j = sum of w over N(v) up to position j (W_{-1} = 0).
__device__ __forceinline__ uint64_t static_prefix(const GraphView& g, int64_t bv, int j) {
  return j < 0 ? 0ull : (g.w ? __ldg(g.wpre + bv + j) : (uint64_t)(j + 1));
}

// ---------------------------------------------------------------------------
// Merge form of a step (k >= 1) whose lists both fit a staging window: N(v)
// and N(t) land in two shared-memory windows by TMA bulk copies and the warp
// merges them along the merge path (A = N(v) wins ties): lane k takes the
// diagonal segment [k (a+b) / 32, (k+1) (a+b) / 32) of the merged order,
// found by one binary search, and walks it; an element x of N(v) is special
// when it equals the first unconsumed element of N(t) (x in N(t)) or t.  The
// per-lane corrections sum (warp scan) to T; the lane whose segment contains
// the first inclusive prefix above r walks its segment again to find it.
// Nothing is stored per special: O((deg v + deg t) / 32) per lane.
__device__ __forceinline__ void sts32(uint32_t addr, int32_t v) {
  asm volatile("st.shared.s32 [%0], %1;" ::"r"(addr), "r"(v));
}

__device__ __forceinline__ int32_t merge_step(const StepCtx& c, WarpSmem& sm, uint64_t u, uint32_t a_p, uint32_t a_q,
                                              int lane) {
  const GraphView& g = *c.g;
  const int a = c.dv, b = c.dt;  // 1 <= a, b <= wlen
  stage_fill(sm, g, c.nv, a, 0, lane);
  stage_fill(sm, g, c.nt, b, 1, lane);
  stage_wait(sm, 0);
  stage_wait(sm, 1);
  const uint32_t A = smem_addr(sm.win + (((uintptr_t)c.nv & 15) >> 2));
  const uint32_t B = smem_addr(sm.win + (sm.wlen + 8) + (((uintptr_t)c.nt & 15) >> 2));
  // +inf after each list (the windows have slack): the walk needs no bounds tests
  if (lane == 0) {
    sts32(A + 4u * (uint32_t)a, INT32_MAX);
    sts32(B + 4u * (uint32_t)b, INT32_MAX);
  }
  __syncwarp();
  const int tot = a + b;
  const int d0 = (int)(((int64_t)lane * tot) >> 5), d1 = (int)(((int64_t)(lane + 1) * tot) >> 5);
  // merge-path split: A elements among the first d0 of the merged order
  int lo = max(0, d0 - b), hi = min(d0, a);
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (lds32(A + 4u * (uint32_t)mid) <= lds32(B + 4u * (uint32_t)(d0 - mid - 1))) lo = mid + 1;
    else hi = mid;
  }
  const int i0 = lo, j0 = d0 - lo;
  const int i1n = __shfl_down_sync(kFull, i0, 1);
  const int i1 = lane == 31 ? a : i1n;  // first A element of the next segment
  const uint64_t d1c = (uint64_t)kAlphaOne - (uint64_t)a_q, d2c = (uint64_t)a_p - (uint64_t)a_q;
  uint64_t corr = 0;
  {
    int i = i0, j = j0;
    int32_t av = lds32(A + 4u * (uint32_t)i), bv = lds32(B + 4u * (uint32_t)j);
    for (int st = d0; st < d1; ++st) {
      const bool ta = av <= bv;  // the next merged element is A's (ties: A first)
      const bool sp = ta && (av == c.t32 || av == bv);
      if (g.w) {
        if (sp) corr += (av == c.t32 ? d2c : d1c) * (uint64_t)__ldg(g.w + c.bv + i);
      } else {
        corr += sp ? (av == c.t32 ? d2c : d1c) : 0ull;
      }
      i += ta ? 1 : 0;
      j += ta ? 0 : 1;
      const int32_t nx = lds32(ta ? A + 4u * (uint32_t)i : B + 4u * (uint32_t)j);
      av = ta ? nx : av;
      bv = ta ? bv : nx;
    }
  }
  const uint64_t incl = warp_incl_scan_u64(corr, lane);
  const uint64_t T = (uint64_t)a_q * static_prefix(g, c.bv, a - 1) + __shfl_sync(kFull, incl, 31);
  if (T == 0) return -1;
  const uint64_t r = scale_draw(u, T);
  const uint64_t C_end = (uint64_t)a_q * static_prefix(g, c.bv, i1 - 1) + incl;
  const int f = __ffs(__ballot_sync(kFull, C_end > r)) - 1;  // lane 31's C_end is T > r
  // the answer is among positions [p0, p1) of segment f: the warp takes them 32 at a time,
  // each lane one position (x special when x == t or x is in N(t), by a search of B)
  const int p0 = __shfl_sync(kFull, i0, f), p1 = __shfl_sync(kFull, i1, f);
  uint64_t D = __shfl_sync(kFull, incl - corr, f);
  int chosen = -1;
  for (int q0 = p0; q0 < p1 && chosen < 0; q0 += 32) {
    const int p = q0 + lane;
    uint64_t dl = 0;
    if (p < p1) {
      const int32_t x = lds32(A + 4u * (uint32_t)p);
      int l2 = 0, n2 = b;  // lower bound of x in B
      while (n2 > 0) {
        const int h2 = n2 >> 1;
        const bool lt = lds32(B + 4u * (uint32_t)(l2 + h2)) < x;
        l2 = lt ? l2 + h2 + 1 : l2;
        n2 = lt ? n2 - h2 - 1 : h2;
      }
      const bool sp = x == c.t32 || lds32(B + 4u * (uint32_t)l2) == x;  // B[b] is +inf
      dl = sp ? (x == c.t32 ? d2c : d1c) * (g.w ? (uint64_t)__ldg(g.w + c.bv + p) : 1ull) : 0ull;
    }
    const uint64_t inc = warp_incl_scan_u64(dl, lane) + D;
    const bool hit = p < p1 && (uint64_t)a_q * static_prefix(g, c.bv, p) + inc > r;
    const unsigned hm = __ballot_sync(kFull, hit);
    if (hm) chosen = q0 + __ffs(hm) - 1;
    D = __shfl_sync(kFull, inc, 31);
  }
  N2V_CHECK(g, chosen >= 0 && chosen < a);
  return lds32(A + 4u * (uint32_t)chosen);
}

// How a step enumerates its specials (the generator modes of gen_specials) and
// which hub structure, if any, serves its longer list.
struct StepPlan {
  int mode;
  int32_t hub, bm;
};

// Identical in every lane (and in every warp of a block that shares the step).
// FULL = false: the instance without hub caches and without the merge form
// (those generators are then not compiled into the caller at all).
template <bool FULL = true>
__device__ __forceinline__ StepPlan plan_step(StepCtx& c, const GraphView& g, int64_t t, int64_t v,
                                              const WarpSmem& sm, int stream_ratio, int merge_ratio) {
  const bool v_short = c.dv <= c.slen;
  const int shorter = v_short ? c.dv : c.slen;
  const int longer = v_short ? c.dt : c.dv;  // the list that would be staged
  const int64_t probe_cost = 32ll * ((shorter + 31) / 32) * (ceil_log2(longer + 1) + 1);
  StepPlan pl;
  pl.hub = -1;
  pl.bm = -1;
  // a longer list with a rank bitmap or a hashed set is always probed: about one load per
  // candidate instead of a search
  const int64_t lv = v_short ? t : v;
  if (FULL && g.bm_data && longer >= g.bm_min_deg) pl.bm = bm_find(g, (int32_t)lv);
  if (FULL && pl.bm < 0 && g.hub_of && longer >= g.hub_min_deg) pl.hub = __ldg(g.hub_of + lv);
  if (pl.bm >= 0 || pl.hub >= 0) {
    pl.mode = v_short ? 0 : 1;
  } else if (FULL && merge_ratio > 0 && c.dv <= sm.wlen && c.dt <= sm.wlen &&
             (int64_t)(c.dv + c.dt) * 10 <= (int64_t)merge_ratio * probe_cost) {
    pl.mode = 4;  // both lists fit a window: merge them
  } else if (sm.wlen > 0 && longer > 64 && longer * 10 <= (int64_t)stream_ratio * probe_cost) {
    pl.mode = v_short ? 3 : 2;
  } else {
    pl.mode = v_short ? 0 : 1;
  }
  return pl;
}

// t's slot in S = N(t) + {t} (the modes that walk S need it).
__device__ __forceinline__ void find_t_slot(StepCtx& c) {
  c.ins = lower_bound32(c.nt, c.dt, c.t32);
  c.has_self = c.ins < c.dt && __ldg(c.nt + c.ins) == c.t32;
  c.slen = c.dt + (c.has_self ? 0 : 1);
}

__device__ __forceinline__ SpecialSink new_sink(const WarpSmem& sm, int dv) {
  SpecialSink sk;
  sk.lim = dv;
  sk.cnt = 0;
  sk.ord_t = -1;
  sk.dpart = 0;
  sk.skip = 0;
  sk.cap = sm.cap;  // positions are packed in 30 bits: degrees < 2^30 (checked at load)
  sk.keep = sk.cap + sm.spill_cap;
  return sk;
}

// Sum of (alpha - a_q) * w over the specials the sink saw (whole warp).
__device__ __forceinline__ uint64_t sink_correction(const GraphView& g, const SpecialSink& sk, uint32_t a_p,
                                                    uint32_t a_q) {
  if (g.w) return warp_sum_u64(sk.dpart);
  const uint64_t d1 = (uint64_t)kAlphaOne - (uint64_t)a_q, d2 = (uint64_t)a_p - (uint64_t)a_q;
  return (uint64_t)(sk.cnt - (sk.ord_t >= 0 ? 1 : 0)) * d1 + (sk.ord_t >= 0 ? d2 : 0ull);
}

// The chosen position, given that it lies in the position range (prev0, hi]
// of N(v) and that C_j = a_q W_j + D_j with D = D0 just before the range.
// Pass 1 enumerates the range's specials, keeping ordinals [0, keep): done by
// the caller when first_done (with r given), else here, where its corrections
// give T = Tbase + their sum and r = floor(u T / 2^64) (-2 is returned when
// T == 0: a dead end).  Pass 2 walks the kept specials in position order; if
// the answer lies beyond them, the range is enumerated again keeping the next
// segment, and the walk continues from where it stopped.  The generator has
// one call site here, so the step's largest code is inlined once.
__device__ __forceinline__ int select_range(StepCtx& c, const StepPlan& pl, WarpSmem& sm, SpecialSink& sk,
                                            bool first_done, uint64_t& r, uint64_t u, uint64_t Tbase, uint64_t D0,
                                            int prev0, int hi_pos, uint32_t a_p, uint32_t a_q, int lane) {
  const GraphView& g = *c.g;
  const int64_t bv = c.bv;
  uint64_t D = D0;
  int prev = prev0, chosen = -1;
  bool found = false;
  const uint64_t d1 = (uint64_t)kAlphaOne - (uint64_t)a_q, d2 = (uint64_t)a_p - (uint64_t)a_q;
  for (int seg = 0;; seg += sk.keep) {
    if (seg > 0 || !first_done) {
      if (seg > 0 && lane == 0) N2V_STAT(kStatSegments, 1);
      sk.cnt = 0;
      sk.ord_t = -1;
      sk.skip = seg;
      gen_specials(c, pl.mode, pl.hub, pl.bm, sm, sk, a_p, a_q, lane);
      if (seg == 0) {
        const uint64_t T = Tbase + sink_correction(g, sk, a_p, a_q);
        if (T == 0) return -2;
        r = scale_draw(u, T);
        if (lane == 0 && sk.cnt > sk.cap) N2V_STAT(kStatSpilled, 1);
      }
    }
    __syncwarp();
    __threadfence_block();  // spilled specials are read back by other lanes
    if (!g.w && sk.cnt <= sk.keep) {
      // Unweighted, all specials kept: the correction after special m is
      // (m + 1) d1 plus (d2 - d1) once the x == t special is passed, so
      // C at special m is known without a scan and the first special with
      // C > r is found by a 32-way search over the ordinals.
      auto spec_at = [&](int m) -> int { return (int)((m < sk.cap ? sm.spec[m] : sm.spill[m - sk.cap]) & 0x3fffffffu); };
      auto Dm = [&](int m) -> uint64_t {
        return m < 0 ? D0 : D0 + (uint64_t)(m + 1) * d1 + ((sk.ord_t >= 0 && m >= sk.ord_t) ? d2 - d1 : 0ull);
      };
      int lo = 0, hi = sk.cnt;  // first m in [lo, hi) with C(pos_m) > r, hi if none
      while (hi - lo > 0) {
        const int span = hi - lo;
        const int step = (span + 31) / 32;
        const int m = lo + lane * step;
        const bool ok = m < hi && (uint64_t)a_q * (uint64_t)(spec_at(m) + 1) + Dm(m) > r;
        const unsigned bal = __ballot_sync(kFull, ok);
        if (step == 1) {
          hi = bal ? lo + __ffs(bal) - 1 : hi;
          break;
        }
        if (!bal) {
          lo += ((hi - 1 - lo) / step) * step + 1;  // past the last probe below hi
          continue;
        }
        const int f = __ffs(bal) - 1;
        hi = lo + f * step;  // m = hi satisfies
        if (f > 0) lo = lo + (f - 1) * step + 1;
      }
      if (hi < sk.cnt) {
        const int fpos = spec_at(hi);
        prev = hi > 0 ? spec_at(hi - 1) : prev0;
        D = Dm(hi - 1);
        if ((uint64_t)a_q * (uint64_t)fpos + D > r) {
          chosen = fpos - 1;  // in the gap (prev, fpos - 1]
        } else {
          chosen = fpos;
          found = true;
        }
      } else {
        prev = sk.cnt > 0 ? spec_at(sk.cnt - 1) : prev0;
        D = Dm(sk.cnt - 1);
      }
      break;
    }
    const int n_in = min(sk.cnt - seg, sk.keep);
    for (int c0 = 0; c0 < n_in; c0 += 32) {
      int32_t pos = -1;
      uint32_t cls = 0;
      const int i = c0 + lane;
      if (i < n_in) {
        const uint32_t e = i < sk.cap ? sm.spec[i] : sm.spill[i - sk.cap];
        pos = (int32_t)(e & 0x3fffffffu);
        cls = e >> 30;
      }
#ifdef N2V_CHECKED
      {  // kept specials come in strictly increasing position, after the ones already passed
        const int ppos = __shfl_up_sync(kFull, pos, 1);
        N2V_CHECK(g, cls == 0u || pos > (lane == 0 ? prev : ppos));
        N2V_CHECK(g, cls == 0u || pos <= hi_pos);
      }
#endif
      const uint64_t dl = special_delta(g, bv, pos, cls, a_p, a_q);
      const uint64_t incl = warp_incl_scan_u64(dl, lane) + D;
      const uint64_t excl = incl - dl;
      const uint64_t Wp = pos < 0 ? 0ull : static_prefix(g, bv, pos);
      const bool hit = cls != 0u && ((uint64_t)a_q * Wp + incl > r);
      const unsigned hm = __ballot_sync(kFull, hit);
      const unsigned smask = __ballot_sync(kFull, cls != 0u);
      if (hm) {
        const int f = __ffs(hm) - 1;
        const int fpos = __shfl_sync(kFull, pos, f);
        const uint64_t fexcl = __shfl_sync(kFull, excl, f);
        const unsigned below = smask & ((1u << f) - 1u);
        const int pp = __shfl_sync(kFull, pos, below ? 31 - __clz(below) : 0);
        const int gap_lo = below ? pp : prev;
        const uint64_t Wb = static_prefix(g, bv, fpos - 1);
        if ((uint64_t)a_q * Wb + fexcl > r) {
          prev = gap_lo;
          D = fexcl;
          chosen = fpos - 1;  // the answer lies in (gap_lo, fpos - 1]
        } else {
          chosen = fpos;
          found = true;
        }
        break;
      }
      if (smask) {
        D = __shfl_sync(kFull, incl, 31);
        prev = __shfl_sync(kFull, pos, 31 - __clz(smask));
      }
    }
    if (found || chosen >= 0 || seg + sk.keep >= sk.cnt) break;
  }
  if (!found) {
    // first j in (prev, hi] with a_q * W_j + D > r
    const int hi = chosen >= 0 ? chosen : hi_pos;
    const uint64_t m = div_aq(sm, r - D, a_q);
    if (!g.w) {
      chosen = m > (uint64_t)hi ? hi : (int)m;
      if (chosen <= prev) chosen = prev + 1;
    } else {
      chosen = (int)warp_first_above_u64(g.wpre + bv, prev + 1, hi, m, lane);
    }
  }
  N2V_CHECK(g, chosen > prev0 && chosen <= hi_pos && chosen < c.dv);
  // the spilled specials are dead: drop their L2 lines instead of letting them be written back
  // (only lines wholly inside this warp's used part of its spill area)
  if (sm.spill && sk.cnt > sk.cap) {
    const uintptr_t b0 = (uintptr_t)sm.spill;
    const uintptr_t e0 = b0 + 4u * (uintptr_t)(min(sk.cnt, sk.keep) - sk.cap);
    const uintptr_t first = (b0 + 127u) & ~(uintptr_t)127u, last = e0 & ~(uintptr_t)127u;
    __syncwarp();
    for (uintptr_t a = first + 128u * (uintptr_t)lane; a < last; a += 128u * 32u) discard_l2_line((const void*)a);
  }
  return chosen;
}

__device__ __forceinline__ StepCtx step_ctx(const GraphView& g, int64_t t, int64_t bv, int64_t ev, int64_t bt,
                                            int64_t et) {
  StepCtx c;
  c.g = &g;
  c.bv = bv;
  c.dv = (int)(ev - bv);
  c.dt = (int)(et - bt);
  c.nv = g.col + bv;
  c.nt = g.col + bt;
  c.t32 = (int32_t)t;
  c.ins = -1;          // t's slot in S: found only by the modes that walk S
  c.has_self = false;
  c.slen = c.dt + 1;   // |S| unless t has a self-loop; fixed where S is walked
  c.cb = 0;
  c.ce = -1;
  c.lb = 0;
  c.le = -1;
  return c;
}

// bv, ev: row bounds of v; bt, et: row bounds of t (k >= 1)
template <bool FULL = true>
__device__ __forceinline__ int32_t warp_step(const GraphView& g, int64_t t, int64_t v, int64_t bv, int64_t ev,
                                             int64_t bt, int64_t et, int k, uint64_t u, uint32_t a_p, uint32_t a_q,
                                             WarpSmem& sm, int stream_ratio, int lane) {
  const int64_t dv = ev - bv;
  if (dv == 0) return -1;
  const int32_t* __restrict__ nv = g.col + bv;
  if (k == 0) {
    if (!g.w) return __ldg(nv + (int64_t)scale_draw(u, (uint64_t)dv));
    const uint64_t T0 = __ldg(g.wpre + ev - 1);
    if (T0 == 0) return -1;
    return __ldg(nv + warp_first_above_u64(g.wpre + bv, 0, dv - 1, scale_draw(u, T0), lane));
  }
#ifdef N2V_STATS
  const long long t_enter = clock64();
#endif
  StepCtx c = step_ctx(g, t, bv, ev, bt, et);
  const StepPlan pl = plan_step<FULL>(c, g, t, v, sm, stream_ratio, sm.merge_ratio);
#ifdef N2V_STATS
  auto stat = [&]() {
    if (lane == 0) {
      const int sh = c.dv <= c.dt + 1 ? c.dv : c.dt + 1, lg = c.dv <= c.dt + 1 ? c.dt : c.dv;
      N2V_STAT(kStatMode + 4 * pl.mode, 1);
      N2V_STAT(kStatMode + 4 * pl.mode + 1, clock64() - t_enter);
      N2V_STAT(kStatMode + 4 * pl.mode + 2, sh);
      N2V_STAT(kStatMode + 4 * pl.mode + 3, lg);
    }
  };
#endif
  if (FULL && pl.mode == 4) {
    const int32_t x = merge_step(c, sm, u, a_p, a_q, lane);
#ifdef N2V_STATS
    stat();
#endif
    return x;
  }
  if (pl.mode == 1) find_t_slot(c);  // walks S in order (mode 2 finds t's slot while its copies fly)
  // every special (their corrections give T), then the selection
  SpecialSink sk = new_sink(sm, c.dv);
  uint64_t r = 0;
  const int chosen = select_range(c, pl, sm, sk, false, r, u, (uint64_t)a_q * static_prefix(g, bv, c.dv - 1), 0ull,
                                  -1, c.dv - 1, a_p, a_q, lane);
  if (chosen < 0) return -1;  // T == 0
  __syncwarp();
#ifdef N2V_STATS
  stat();
#endif
  return __ldg(nv + chosen);
}

// ---------------------------------------------------------------------------
// Whole block (four warps), one step.  Every thread of the block must call it
// with the same arguments; it synchronises the block twice.
//
// The candidates of the step (the shorter list, as in warp_step) are split
// into four contiguous quarters, one per warp.  Because both lists are sorted,
// the specials warp w finds all lie in a position range [P_w, P_{w+1}) of
// N(v), and the four ranges tile N(v) in order.  Each warp enumerates its
// quarter into its own shared-memory specials (staging only the part of the
// longer list its quarter can meet); a block-wide exclusive scan of the four
// corrections gives T and, per range, D just before it.  The range whose end
// value C exceeds r = floor(u T / 2^64) while the value before it does not
// holds the answer, and its warp finishes the step as warp_step does.
struct BlockScratch {
  uint64_t corr[4];
  int32_t pos[4];   // P_w
  int32_t result;
};

__device__ __forceinline__ int32_t block_step(const GraphView& g, int64_t t, int64_t v, int k, uint64_t u,
                                              uint32_t a_p, uint32_t a_q, WarpSmem& sm, BlockScratch* bs, int wib,
                                              int stream_ratio, int lane) {
  const int64_t bv = g.rp[v], ev = g.rp[v + 1];
  const int64_t dv = ev - bv;
  if (dv == 0) return -1;
  if (k == 0) return warp_step(g, t, v, bv, ev, 0, 0, 0, u, a_p, a_q, sm, stream_ratio, lane);
  const int64_t bt = g.rp[t], et = g.rp[t + 1];
  StepCtx c = step_ctx(g, t, bv, ev, bt, et);
  StepPlan pl = plan_step(c, g, t, v, sm, stream_ratio, sm.merge_ratio);
  if (pl.mode == 4) return merge_step(c, sm, u, a_p, a_q, lane);  // short lists: every warp merges them alike
  const bool cand_v = pl.mode == 0 || pl.mode == 3;  // candidates: N(v) (positions) or S
  if (!cand_v) find_t_slot(c);
  const int nc = cand_v ? c.dv : c.slen;
  const int per = (((nc + 3) >> 2) + 63) & ~63;  // whole 64-candidate chunks per warp
  const int cb = min(nc, wib * per), ce = min(nc, cb + per);
  // P(i): the first position of N(v) a candidate >= the i-th can meet
  auto pos_of = [&](int i) -> int {
    if (i == 0) return 0;
    if (i >= nc) return c.dv;
    return cand_v ? i : lower_bound32(c.nv, c.dv, s_at(c, i));
  };
  const int P_lo = pos_of(cb), P_hi = pos_of(ce);
  c.cb = cb;
  c.ce = ce;
  if (pl.mode == 2) {  // stage N(v): only the positions this quarter can reach
    c.lb = P_lo;
    c.le = P_hi;
  } else if (pl.mode == 3) {  // stage N(t): only the elements this quarter's keys can equal
    c.lb = cb >= nc ? c.dt : (cb == 0 ? 0 : lower_bound32(c.nt, c.dt, __ldg(c.nv + cb)));
    c.le = ce >= nc ? c.dt : lower_bound32(c.nt, c.dt, __ldg(c.nv + ce));
  }
  if ((pl.mode == 2 || pl.mode == 3) && c.le <= c.lb) {
    pl.mode = pl.mode == 2 ? 1 : 0;  // nothing to stream: probe the whole longer list, same candidates
    c.lb = 0;
    c.le = -1;
  }
  SpecialSink sk = new_sink(sm, c.dv);
  if (cb < ce) gen_specials(c, pl.mode, pl.hub, pl.bm, sm, sk, a_p, a_q, lane);
  const uint64_t corr = sink_correction(g, sk, a_p, a_q);
  if (lane == 0) {
    bs->corr[wib] = corr;
    bs->pos[wib] = P_lo;
  }
  __syncthreads();
  uint64_t T = (uint64_t)a_q * static_prefix(g, bv, c.dv - 1), Dw = 0;
  for (int w = 0; w < 4; ++w) {
    const uint64_t cw = bs->corr[w];
    T += cw;
    if (w < wib) Dw += cw;
  }
  int32_t res = -1;
  if (T != 0) {
    const uint64_t r = scale_draw(u, T);
    const uint64_t C_before = (uint64_t)a_q * static_prefix(g, bv, P_lo - 1) + Dw;
    const uint64_t C_end = (uint64_t)a_q * static_prefix(g, bv, P_hi - 1) + Dw + corr;
#ifdef N2V_CHECKED
    {  // exactly one of the four ranges holds the draw, and they tile N(v) in order
      int claims = 0;
      uint64_t D = 0;
      for (int w = 0; w < 4; ++w) {
        const int lo = bs->pos[w], hi = w < 3 ? bs->pos[w + 1] : c.dv;
        N2V_CHECK(g, lo <= hi);
        const uint64_t cb4 = (uint64_t)a_q * static_prefix(g, bv, lo - 1) + D;
        D += bs->corr[w];
        const uint64_t ce4 = (uint64_t)a_q * static_prefix(g, bv, hi - 1) + D;
        claims += (lo < hi && cb4 <= r && r < ce4) ? 1 : 0;
      }
      N2V_CHECK(g, claims == 1 && bs->pos[0] == 0);
    }
#endif
    if (P_lo < P_hi && C_before <= r && r < C_end) {
      uint64_t rr = r;
      const int j = select_range(c, pl, sm, sk, true, rr, 0ull, 0ull, Dw, P_lo - 1, P_hi - 1, a_p, a_q, lane);
      if (lane == 0) bs->result = __ldg(c.nv + j);
    }
  }
  __syncthreads();
  if (T != 0) res = bs->result;
  return res;
}

// ---------------------------------------------------------------------------
// One lane, static weights only (superstep 0 of Algorithm 1, and the steps
// FN-Approx approximates): first j with W_j > floor(u * W_last / 2^64).
__device__ __forceinline__ int32_t static_step(const GraphView& g, int64_t bv, int64_t ev, uint64_t u) {
  const int64_t dv = ev - bv;
  if (dv <= 0) return -1;
  if (!g.w) return __ldg(g.col + bv + (int64_t)scale_draw(u, (uint64_t)dv));
  const uint64_t T = __ldg(g.wpre + ev - 1);
  if (T == 0) return -1;
  const uint64_t r = scale_draw(u, T);
  int64_t lo = 0, n = dv;  // first index with wpre > r
  while (n > 0) {
    const int64_t half = n >> 1;
    if (__ldg(g.wpre + bv + lo + half) <= r) {
      lo += half + 1;
      n -= half + 1;
    } else {
      n = half;
    }
  }
  return __ldg(g.col + bv + lo);
}

// Does FN-Approx replace this 2nd-order step by a static-weight one?
__device__ __forceinline__ bool approx_here(const WalkJob& J, int k, int64_t dv, int64_t dt) {
  return J.approx && k > 0 && dv >= J.approx_popular && dt < J.approx_popular &&
         approx_decide(dv, dt, J.a_p, J.a_q, J.w_min, J.w_max, J.approx_eps);
}

// ---------------------------------------------------------------------------
// One step for the 32 walkers a warp owns (one per lane).  Steps whose
// degrees are all <= thr run on their own lane (thread bin); the others are
// taken one after another by the whole warp (warp bin).  FULL = false: the
// instance for exact walks without hub caches or the merge form.
template <bool FULL = true>
__device__ __forceinline__ int32_t warp_binned_step(const GraphView& g, bool alive, int64_t t, int64_t v, int k,
                                                    uint64_t wid, const WalkJob& J, int thr, WarpSmem& sm,
                                                    int stream_ratio, int lane) {
  const uint64_t seed = J.seed;
  const uint32_t a_p = J.a_p, a_q = J.a_q;
  int32_t x = -1;
  bool small = false;
  uint64_t u = 0;
  int64_t bv = 0, ev = 0, bt = 0, et = 0;
#ifdef N2V_STATS
  const long long t_lane = clock64();
#endif
  if (alive) {
    // every lane fetches its own walker's row bounds: 32 independent loads
    bv = g.rp[v];
    ev = g.rp[v + 1];
    if (k > 0) {
      bt = g.rp[t];
      et = g.rp[t + 1];
    }
    u = philox_draw(seed, wid, (uint32_t)k);
    if (FULL && approx_here(J, k, ev - bv, et - bt)) {
      small = true;  // taken on this lane, by static weights
      x = static_step(g, bv, ev, u);
    } else {
      small = ev - bv <= thr && (k == 0 || et - bt <= thr);
      if (small) x = thread_step(g, t, v, k, u, a_p, a_q);
    }
  }
  unsigned wm = __ballot_sync(kFull, alive && !small);
#ifdef N2V_STATS
  {
    const long long dt_lane = clock64() - t_lane;
    const long long mx = __reduce_max_sync(kFull, (unsigned)min(dt_lane, (long long)0xffffffff));
    const bool any_alive = __any_sync(kFull, alive);  // every lane votes (never inside a lane branch)
    if (lane == 0 && any_alive) {
      N2V_STAT(k == 0 ? kStatFirst : kStatLaneSteps, 1);
      N2V_STAT(k == 0 ? kStatFirstCycles : kStatLaneCycles, mx);
    }
  }
#endif
  while (wm) {
    const int src = __ffs(wm) - 1;
    wm &= wm - 1;
    const int32_t xx = warp_step<FULL>(g, __shfl_sync(kFull, t, src), __shfl_sync(kFull, v, src),
                                 __shfl_sync(kFull, bv, src), __shfl_sync(kFull, ev, src),
                                 __shfl_sync(kFull, bt, src), __shfl_sync(kFull, et, src), k,
                                 __shfl_sync(kFull, u, src), a_p, a_q, sm, stream_ratio, lane);
    if (lane == src) x = xx;
  }
  return x;
}

}  // namespace n2v

namespace n2v {

// ---------------------------------------------------------------------------
// Block tier: the shared-memory queue of one step's work of a block.  Steps
// for the whole block fill it from the front, steps for one warp from the
// back; the warps take the latter one at a time, whichever warp is free.
struct BlockQueue {
  unsigned long long base;  // first walker of the block's current batch
  int32_t nb[2], nw[2];     // queued block steps and warp steps, by the parity of the step index
  int32_t pull[2];          // warp steps taken so far, by parity
  BlockScratch scratch;
  int32_t qt[kPersistThreads], qv[kPersistThreads];  // queued steps: t and v
  uint64_t qu[kPersistThreads];                      // and their draws
  int32_t res[kPersistThreads];                      // and their results
};

// One step for the 128 walkers of a block (one per thread): the degree-binned
// work queue of the block.  A step whose degrees are all <= thr runs on its own
// lane.  Every other step is queued in shared memory: those whose longer list
// has at least block_min_deg entries are taken one after another by the whole
// block (block_step), the rest one at a time by whichever warp is free
// (warp_step), so that one costly step does not hold three idle warps.  Every
// thread of the block must call it; it synchronises the block twice.
__device__ __forceinline__ int32_t block_binned_step(const GraphView& g, bool alive, int64_t t, int64_t v, int k,
                                                     uint64_t wid, const WalkJob& J, const LaunchCfg& L, WarpSmem& sm,
                                                     BlockQueue* bq, int wib, int lane, int tid) {
  const uint32_t a_p = J.a_p, a_q = J.a_q;
  const int par = k & 1;
  int32_t x = -1;
  bool small = false, big = false, queued = false;
  uint64_t u = 0;
  if (alive) {
    const int64_t bv = g.rp[v], ev = g.rp[v + 1];
    int64_t bt = 0, et = 0;
    if (k > 0) {
      bt = g.rp[t];
      et = g.rp[t + 1];
    }
    u = philox_draw(J.seed, wid, (uint32_t)k);
    if (approx_here(J, k, ev - bv, et - bt)) {
      small = true;
      x = static_step(g, bv, ev, u);
    } else {
      small = ev - bv <= L.thread_max_deg && (k == 0 || et - bt <= L.thread_max_deg);
      if (small) x = thread_step(g, t, v, k, u, a_p, a_q);
      else big = max(ev - bv, et - bt) >= (int64_t)L.block_min_deg;
    }
    queued = !small;
  }
  // queue: block steps at the front, warp steps at the back
  const unsigned mb = __ballot_sync(kFull, queued && big), mw = __ballot_sync(kFull, queued && !big);
  int b0 = 0, w0 = 0;
  if (lane == 0) {
    if (mb) b0 = atomicAdd(&bq->nb[par], __popc(mb));
    if (mw) w0 = atomicAdd(&bq->nw[par], __popc(mw));
  }
  b0 = __shfl_sync(kFull, b0, 0);
  w0 = __shfl_sync(kFull, w0, 0);
  int slot = -1;
  if (queued) {
    slot = big ? b0 + __popc(mb & lanemask_lt()) : kPersistThreads - 1 - (w0 + __popc(mw & lanemask_lt()));
    bq->qt[slot] = (int32_t)t;
    bq->qv[slot] = (int32_t)v;
    bq->qu[slot] = u;
  }
  __syncthreads();
  const int nb = bq->nb[par], nw = bq->nw[par];
  if (tid == 0) {  // the next step's counters (nobody touches them before the next barrier)
    bq->nb[par ^ 1] = 0;
    bq->nw[par ^ 1] = 0;
    bq->pull[par ^ 1] = 0;
  }
  for (int e = 0; e < nb; ++e) {  // uniform: every thread read the same nb
    const int32_t y = block_step(g, bq->qt[e], bq->qv[e], k, bq->qu[e], a_p, a_q, sm, &bq->scratch, wib,
                                 L.stream_ratio, lane);
    if (tid == 0) bq->res[e] = y;
  }
  for (;;) {  // warp steps, one per free warp
    int e = 0;
    if (lane == 0) e = atomicAdd(&bq->pull[par], 1);
    e = __shfl_sync(kFull, e, 0);
    if (e >= nw) break;
    const int sl = kPersistThreads - 1 - e;
    const int64_t qt = bq->qt[sl], qv = bq->qv[sl];
    const int64_t bv = g.rp[qv], ev = g.rp[qv + 1];
    const int64_t bt = k > 0 ? g.rp[qt] : 0, et = k > 0 ? g.rp[qt + 1] : 0;
    const int32_t y = warp_step(g, qt, qv, bv, ev, bt, et, k, bq->qu[sl], a_p, a_q, sm, L.stream_ratio, lane);
    if (lane == 0) bq->res[sl] = y;
  }
  __syncthreads();
  if (queued) x = bq->res[slot];
  return x;
}

}  // namespace n2v
