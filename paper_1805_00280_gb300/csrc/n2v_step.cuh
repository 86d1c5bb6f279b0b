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
// of the static prefix (weighted).  The specials are found by scanning the
// SHORTER of N(v) and N(t) and probing the longer one (binary search, or the
// hashed set of a hub): O(min(deg v, deg t) * probe) instead of
// O(deg v + deg t).  All arithmetic is modulo 2^64; every true prefix lies in
// [0, T] < 2^64, so the modular values are the exact ones.
//
// sbuf: this warp's shared-memory slots (cap entries) keep the specials of
// pass 1 for pass 2; when a step has more, pass 2 recomputes them.
__device__ __forceinline__ int32_t warp_step(const GraphView& g, int64_t t, int64_t v, int k, uint64_t u,
                                             uint32_t a_p, uint32_t a_q, uint32_t* sbuf, int cap, int lane) {
  const int64_t bv = g.rp[v], ev = g.rp[v + 1], dv = ev - bv;
  if (dv == 0) return -1;
  const int32_t* __restrict__ nv = g.col + bv;
  if (k == 0) {
    if (!g.w) return __ldg(nv + (int64_t)scale_draw(u, (uint64_t)dv));
    const uint64_t T0 = __ldg(g.wpre + ev - 1);
    if (T0 == 0) return -1;
    return __ldg(nv + warp_first_above_u64(g.wpre + bv, 0, dv - 1, scale_draw(u, T0), lane));
  }
  const int64_t bt = g.rp[t], et = g.rp[t + 1], dt = et - bt;
  const int32_t* __restrict__ nt = g.col + bt;
  const uint64_t Wv = g.w ? __ldg(g.wpre + ev - 1) : (uint64_t)dv;
  const bool scan_v = dv <= dt;
  const int32_t t32 = (int32_t)t;
  int64_t ncand, ins = 0;
  bool has_self = false;
  int32_t hub = -1;
  if (scan_v) {
    ncand = dv;
    if (g.hub_of) hub = __ldg(g.hub_of + t);
  } else {
    // candidates: N(t) with t itself merged in at its sorted place
    ins = lower_bound_i32(nt, dt, t32);
    has_self = ins < dt && __ldg(nt + ins) == t32;
    ncand = dt + (has_self ? 0 : 1);
    if (g.hub_of) hub = __ldg(g.hub_of + v);
  }
  const int cap_eff = dv < ((int64_t)1 << 30) ? cap : 0;

  // (position in N(v), class) of candidate i: class 0 = default, 1 = x in
  // N(t), 2 = x == t (which takes precedence over membership)
  auto eval = [&](int64_t i, int32_t& pos, uint32_t& cls) {
    pos = -1;
    cls = 0;
    if (i >= ncand) return;
    if (scan_v) {
      const int32_t x = __ldg(nv + i);
      bool special;
      if (x == t32) special = true;
      else if (hub >= 0) special = hub_find(g, hub, x) >= 0;
      else special = contains_i32(nt, dt, x);
      if (special) {
        pos = (int32_t)i;
        cls = (x == t32) ? 2u : 1u;
      }
    } else {
      const int32_t y = has_self ? __ldg(nt + i) : (i < ins ? __ldg(nt + i) : (i == ins ? t32 : __ldg(nt + i - 1)));
      int64_t p;
      if (hub >= 0) {
        p = hub_find(g, hub, y);
      } else {
        p = lower_bound_i32(nv, dv, y);
        if (p >= dv || __ldg(nv + p) != y) p = -1;
      }
      if (p >= 0) {
        pos = (int32_t)p;
        cls = (y == t32) ? 2u : 1u;
      }
    }
  };
  auto delta = [&](int32_t pos, uint32_t cls) -> uint64_t {
    if (!cls) return 0ull;
    const uint64_t a = cls == 2u ? (uint64_t)a_p : (uint64_t)kAlphaOne;
    const uint64_t wt = g.w ? (uint64_t)__ldg(g.w + bv + pos) : 1ull;
    return (a - (uint64_t)a_q) * wt;
  };
  auto Wat = [&](int64_t pos) -> uint64_t {
    return pos < 0 ? 0ull : (g.w ? __ldg(g.wpre + bv + pos) : (uint64_t)(pos + 1));
  };

  // pass 1: total
  uint64_t part = 0;
  int64_t cnt = 0;
  for (int64_t c0 = 0; c0 < ncand; c0 += 32) {
    int32_t pos;
    uint32_t cls;
    eval(c0 + lane, pos, cls);
    part += delta(pos, cls);
    const unsigned m = __ballot_sync(kFull, cls != 0u);
    const int64_t slot = cnt + __popc(m & lanemask_lt());
    if (cls && slot < cap_eff) sbuf[slot] = (uint32_t)pos | (cls << 30);
    cnt += __popc(m);
  }
  const uint64_t T = (uint64_t)a_q * Wv + warp_sum_u64(part);
  if (T == 0) return -1;
  const uint64_t r = scale_draw(u, T);
  __syncwarp();

  // first j in (lo_excl, hi] with a_q * W_j + base > r
  auto solve_gap = [&](int64_t lo_excl, int64_t hi, uint64_t base) -> int64_t {
    const uint64_t m = (r - base) / (uint64_t)a_q;
    if (!g.w) {
      int64_t j = (int64_t)m;
      if (j <= lo_excl) j = lo_excl + 1;
      if (j > hi) j = hi;
      return j;
    }
    return warp_first_above_u64(g.wpre + bv, lo_excl + 1, hi, m, lane);
  };

  // pass 2: walk the specials in position order, carrying the running D
  uint64_t D = 0;
  int64_t prev = -1;
  const bool stored = cnt <= cap_eff;
  const int64_t nsrc = stored ? cnt : ncand;
  for (int64_t c0 = 0; c0 < nsrc; c0 += 32) {
    int32_t pos = -1;
    uint32_t cls = 0;
    if (stored) {
      if (c0 + lane < cnt) {
        const uint32_t e = sbuf[c0 + lane];
        pos = (int32_t)(e & 0x3fffffffu);
        cls = e >> 30;
      }
    } else {
      eval(c0 + lane, pos, cls);
    }
    const uint64_t dl = delta(pos, cls);
    const uint64_t incl = warp_incl_scan_u64(dl, lane) + D;
    const uint64_t excl = incl - dl;
    const bool hit = cls != 0u && ((uint64_t)a_q * Wat(pos) + incl > r);
    const unsigned hm = __ballot_sync(kFull, hit);
    const unsigned sm = __ballot_sync(kFull, cls != 0u);
    if (hm) {
      const int f = __ffs(hm) - 1;
      const int64_t fpos = __shfl_sync(kFull, (int64_t)pos, f);
      const uint64_t fexcl = __shfl_sync(kFull, excl, f);
      const unsigned below = sm & ((1u << f) - 1u);
      const int64_t pp = __shfl_sync(kFull, (int64_t)pos, below ? 31 - __clz(below) : 0);
      const int64_t gap_lo = below ? pp : prev;
      const uint64_t before = (uint64_t)a_q * Wat(fpos - 1) + fexcl;
      const int64_t j = before > r ? solve_gap(gap_lo, fpos - 1, fexcl) : fpos;
      __syncwarp();
      return __ldg(nv + j);
    }
    if (sm) {
      D = __shfl_sync(kFull, incl, 31);
      prev = __shfl_sync(kFull, (int64_t)pos, 31 - __clz(sm));
    }
  }
  __syncwarp();
  return __ldg(nv + solve_gap(prev, dv - 1, D));
}

// ---------------------------------------------------------------------------
// One step for the 32 walkers a warp owns (one per lane).  Steps whose
// degrees are all <= thr run on their own lane (thread bin); the others are
// taken one after another by the whole warp (warp bin).
__device__ __forceinline__ int32_t warp_binned_step(const GraphView& g, bool alive, int64_t t, int64_t v, int k,
                                                    uint64_t wid, uint64_t seed, uint32_t a_p, uint32_t a_q,
                                                    int thr, uint32_t* sbuf, int cap, int lane) {
  int32_t x = -1;
  bool small = false;
  uint64_t u = 0;
  if (alive) {
    u = philox_draw(seed, wid, (uint32_t)k);
    const int64_t dv = g.rp[v + 1] - g.rp[v];
    small = dv <= thr && (k == 0 || g.rp[t + 1] - g.rp[t] <= thr);
    if (small) x = thread_step(g, t, v, k, u, a_p, a_q);
  }
  unsigned wm = __ballot_sync(kFull, alive && !small);
  while (wm) {
    const int src = __ffs(wm) - 1;
    wm &= wm - 1;
    const int64_t tt = __shfl_sync(kFull, t, src);
    const int64_t vv = __shfl_sync(kFull, v, src);
    const uint64_t uu = __shfl_sync(kFull, u, src);
    const int32_t xx = warp_step(g, tt, vv, k, uu, a_p, a_q, sbuf, cap, lane);
    if (lane == src) x = xx;
  }
  return x;
}

}  // namespace n2v
