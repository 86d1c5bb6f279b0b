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
//   probe  -- walk the shorter list; find each element in the longer one by
//             binary search (or the hashed set of a hub): about
//             ceil(short/32) * log2(long) dependent loads;
//   stream -- put the shorter list in a shared-memory hash table and stream the
//             longer one with coalesced, prefetched loads: (short + long)/32
//             independent loads.  A shorter list larger than the table is cut
//             into value ranges, each streamed against its window of the
//             longer list.
// Both give the same specials, so the choice only changes speed.

struct WarpSmem {
  uint32_t* spec;  // cap entries: pos | class << 30
  int cap;
  int2* htab;      // 2 * hcap slots (key, value); key -1 = empty
  int hcap;
};

__device__ __forceinline__ WarpSmem warp_smem(unsigned char* base, int warp, const LaunchCfg& L) {
  WarpSmem w;
  w.htab = (int2*)(base + (size_t)warp * warp_smem_bytes(L));
  w.hcap = L.hash_cap;
  w.spec = (uint32_t*)(w.htab + 2 * L.hash_cap);
  w.cap = L.smem_specials;
  return w;
}

struct StepCtx {
  const GraphView* g;
  int64_t bv, dv, bt, dt;
  const int32_t* __restrict__ nv;
  const int32_t* __restrict__ nt;
  int32_t t32;
  int64_t ins;     // index of t inside S = N(t) + {t}
  bool has_self;   // t already in N(t) (self-loop at t)
  int64_t slen;    // |S|
};

// i-th element of S = N(t) + {t} (sorted, no duplicate)
__device__ __forceinline__ int32_t s_at(const StepCtx& c, int64_t i) {
  if (c.has_self || i < c.ins) return __ldg(c.nt + i);
  return i == c.ins ? c.t32 : __ldg(c.nt + i - 1);
}
// number of elements of S below val
__device__ __forceinline__ int64_t s_lower(const StepCtx& c, int32_t val) {
  int64_t p = lower_bound_i32(c.nt, c.dt, val);
  if (!c.has_self && c.t32 < val) ++p;
  return p;
}

__device__ __forceinline__ uint32_t smem_hash(int32_t x, int bits) { return ((uint32_t)x * 2654435769u) >> (32 - bits); }

// value stored for key x, or -1; the table is at most half full
__device__ __forceinline__ int32_t smem_find(const int2* tab, int bits, int32_t x) {
  const uint32_t mask = (1u << bits) - 1u;
  uint32_t s = smem_hash(x, bits);
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    const int2 e = tab[s];
    if (e.x == x) return e.y;
    if (e.x < 0) return -1;
    s = (s + 1u) & mask;
  }
  return -1;
}

__device__ __forceinline__ void smem_insert(int2* tab, int bits, int32_t x, int32_t val) {
  const uint32_t mask = (1u << bits) - 1u;
  uint32_t s = smem_hash(x, bits);
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    if (atomicCAS(&tab[s].x, -1, x) == -1) {
      tab[s].y = val;
      return;
    }
    s = (s + 1u) & mask;
  }
}

__device__ __forceinline__ int ceil_log2(int64_t x) {
  return x <= 1 ? 0 : 64 - __clzll((unsigned long long)(x - 1));
}

// probe mode, candidates = N(v): class of x_j from a membership test in N(t)
template <class F>
__device__ __forceinline__ bool gen_probe_v(const StepCtx& c, int32_t hub_t, F&& f, int lane) {
  for (int64_t c0 = 0; c0 < c.dv; c0 += 32) {
    const int64_t i = c0 + lane;
    int32_t pos = -1;
    uint32_t cls = 0;
    if (i < c.dv) {
      const int32_t x = __ldg(c.nv + i);
      bool sp;
      if (x == c.t32) sp = true;
      else if (hub_t >= 0) sp = hub_find(*c.g, hub_t, x) >= 0;
      else sp = contains_i32(c.nt, c.dt, x);
      if (sp) {
        pos = (int32_t)i;
        cls = x == c.t32 ? 2u : 1u;
      }
    }
    if (f(pos, cls)) return true;
  }
  return false;
}

// probe mode, candidates = S: position of y in N(v)
template <class F>
__device__ __forceinline__ bool gen_probe_t(const StepCtx& c, int32_t hub_v, F&& f, int lane) {
  for (int64_t c0 = 0; c0 < c.slen; c0 += 32) {
    const int64_t i = c0 + lane;
    int32_t pos = -1;
    uint32_t cls = 0;
    if (i < c.slen) {
      const int32_t y = s_at(c, i);
      int64_t p;
      if (hub_v >= 0) {
        p = hub_find(*c.g, hub_v, y);
      } else {
        p = lower_bound_i32(c.nv, c.dv, y);
        if (p >= c.dv || __ldg(c.nv + p) != y) p = -1;
      }
      if (p >= 0) {
        pos = (int32_t)p;
        cls = y == c.t32 ? 2u : 1u;
      }
    }
    if (f(pos, cls)) return true;
  }
  return false;
}

// stream mode.  hash_s: the table holds S (value = class) and N(v) is
// streamed; otherwise the table holds N(v) (value = position) and S is
// streamed.
template <class F>
__device__ __forceinline__ bool gen_stream(const StepCtx& c, bool hash_s, const WarpSmem& sm, F&& f, int lane) {
  constexpr int U = 4;  // chunks of 32 loads in flight
  const int64_t hlen = hash_s ? c.slen : c.dv;
  const int64_t llen = hash_s ? c.dv : c.slen;
  for (int64_t h0 = 0; h0 < hlen; h0 += sm.hcap) {
    const int64_t h1 = min(h0 + (int64_t)sm.hcap, hlen);
    const int bits = max(6, ceil_log2(2 * (h1 - h0)));
    // the window of the streamed list whose values fall in this piece's range
    int64_t w0 = 0, w1 = llen;
    if (h0 > 0) {
      const int32_t lo = hash_s ? s_at(c, h0) : __ldg(c.nv + h0);
      w0 = hash_s ? lower_bound_i32(c.nv, c.dv, lo) : s_lower(c, lo);
    }
    if (h1 < hlen) {
      const int32_t hi = hash_s ? s_at(c, h1) : __ldg(c.nv + h1);
      w1 = hash_s ? lower_bound_i32(c.nv, c.dv, hi) : s_lower(c, hi);
    }
    __syncwarp();
    for (int s = lane; s < (1 << bits); s += 32) sm.htab[s] = make_int2(-1, -1);
    __syncwarp();
    for (int64_t j = h0 + lane; j < h1; j += 32) {
      if (hash_s) {
        const int32_t y = s_at(c, j);
        smem_insert(sm.htab, bits, y, y == c.t32 ? 2 : 1);
      } else {
        smem_insert(sm.htab, bits, __ldg(c.nv + j), (int32_t)j);
      }
    }
    __syncwarp();
    for (int64_t c0 = w0; c0 < w1; c0 += 32 * U) {
      int32_t e[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t i = c0 + u * 32 + lane;
        e[u] = -1;
        if (i < w1) e[u] = hash_s ? __ldg(c.nv + i) : s_at(c, i);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (c0 + u * 32 >= w1) break;  // uniform
        const int64_t i = c0 + u * 32 + lane;
        int32_t pos = -1;
        uint32_t cls = 0;
        if (i < w1) {
          const int32_t val = smem_find(sm.htab, bits, e[u]);
          if (val >= 0) {
            if (hash_s) {
              pos = (int32_t)i;
              cls = (uint32_t)val;
            } else {
              pos = val;
              cls = e[u] == c.t32 ? 2u : 1u;
            }
          }
        }
        if (f(pos, cls)) return true;
      }
    }
  }
  return false;
}

__device__ __forceinline__ int32_t warp_step(const GraphView& g, int64_t t, int64_t v, int k, uint64_t u,
                                             uint32_t a_p, uint32_t a_q, const WarpSmem& sm, int stream_ratio,
                                             int lane) {
  const int64_t bv = g.rp[v], ev = g.rp[v + 1], dv = ev - bv;
  if (dv == 0) return -1;
  const int32_t* __restrict__ nv = g.col + bv;
  if (k == 0) {
    if (!g.w) return __ldg(nv + (int64_t)scale_draw(u, (uint64_t)dv));
    const uint64_t T0 = __ldg(g.wpre + ev - 1);
    if (T0 == 0) return -1;
    return __ldg(nv + warp_first_above_u64(g.wpre + bv, 0, dv - 1, scale_draw(u, T0), lane));
  }
  StepCtx c;
  c.g = &g;
  c.bv = bv;
  c.dv = dv;
  c.bt = g.rp[t];
  c.dt = g.rp[t + 1] - c.bt;
  c.nv = nv;
  c.nt = g.col + c.bt;
  c.t32 = (int32_t)t;
  c.ins = lower_bound_i32(c.nt, c.dt, c.t32);
  c.has_self = c.ins < c.dt && __ldg(c.nt + c.ins) == c.t32;
  c.slen = c.dt + (c.has_self ? 0 : 1);
  const uint64_t Wv = g.w ? __ldg(g.wpre + ev - 1) : (uint64_t)dv;

  // mode: 0 probe over N(v), 1 probe over S, 2 stream N(v) against a hash of S,
  // 3 stream S against a hash of N(v)
  const int64_t shorter = min(dv, c.slen), longer = max(dv, c.slen);
  int mode;
  int32_t hub = -1;
  const bool v_short = dv <= c.slen;
  const int64_t probe_cost = 32 * ((shorter + 31) / 32) * (int64_t)(ceil_log2(longer + 1) + 1);
  if (longer * 10 <= (int64_t)stream_ratio * probe_cost) {
    mode = v_short ? 3 : 2;
  } else {
    mode = v_short ? 0 : 1;
    if (g.hub_of) hub = __ldg(g.hub_of + (v_short ? t : v));
  }
  const int cap_eff = dv < ((int64_t)1 << 30) ? sm.cap : 0;

  auto delta = [&](int32_t pos, uint32_t cls) -> uint64_t {
    if (!cls) return 0ull;
    const uint64_t a = cls == 2u ? (uint64_t)a_p : (uint64_t)kAlphaOne;
    const uint64_t wt = g.w ? (uint64_t)__ldg(g.w + bv + pos) : 1ull;
    return (a - (uint64_t)a_q) * wt;
  };
  auto Wat = [&](int64_t pos) -> uint64_t {
    return pos < 0 ? 0ull : (g.w ? __ldg(g.wpre + bv + pos) : (uint64_t)(pos + 1));
  };
  auto generate = [&](auto&& f) -> bool {
    switch (mode) {
      case 0: return gen_probe_v(c, hub, f, lane);
      case 1: return gen_probe_t(c, hub, f, lane);
      case 2: return gen_stream(c, true, sm, f, lane);
      default: return gen_stream(c, false, sm, f, lane);
    }
  };

  // pass 1: total, keeping the specials in shared memory while they fit
  uint64_t part = 0;
  int64_t cnt = 0;
  generate([&](int32_t pos, uint32_t cls) -> bool {
    part += delta(pos, cls);
    const unsigned m = __ballot_sync(kFull, cls != 0u);
    const int64_t slot = cnt + __popc(m & lanemask_lt());
    if (cls && slot < cap_eff) sm.spec[slot] = (uint32_t)pos | (cls << 30);
    cnt += __popc(m);
    return false;
  });
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
  int64_t prev = -1, chosen = -1;
  auto search = [&](int32_t pos, uint32_t cls) -> bool {
    const uint64_t dl = delta(pos, cls);
    const uint64_t incl = warp_incl_scan_u64(dl, lane) + D;
    const uint64_t excl = incl - dl;
    const bool hit = cls != 0u && ((uint64_t)a_q * Wat(pos) + incl > r);
    const unsigned hm = __ballot_sync(kFull, hit);
    const unsigned smask = __ballot_sync(kFull, cls != 0u);
    if (hm) {
      const int f = __ffs(hm) - 1;
      const int64_t fpos = __shfl_sync(kFull, (int64_t)pos, f);
      const uint64_t fexcl = __shfl_sync(kFull, excl, f);
      const unsigned below = smask & ((1u << f) - 1u);
      const int64_t pp = __shfl_sync(kFull, (int64_t)pos, below ? 31 - __clz(below) : 0);
      const int64_t gap_lo = below ? pp : prev;
      const uint64_t before = (uint64_t)a_q * Wat(fpos - 1) + fexcl;
      chosen = before > r ? solve_gap(gap_lo, fpos - 1, fexcl) : fpos;
      return true;
    }
    if (smask) {
      D = __shfl_sync(kFull, incl, 31);
      prev = __shfl_sync(kFull, (int64_t)pos, 31 - __clz(smask));
    }
    return false;
  };
  bool found;
  if (cnt <= cap_eff) {
    found = false;
    for (int64_t c0 = 0; c0 < cnt && !found; c0 += 32) {
      int32_t pos = -1;
      uint32_t cls = 0;
      if (c0 + lane < cnt) {
        const uint32_t e = sm.spec[c0 + lane];
        pos = (int32_t)(e & 0x3fffffffu);
        cls = e >> 30;
      }
      found = search(pos, cls);
    }
  } else {
    found = generate(search);
  }
  if (!found) chosen = solve_gap(prev, dv - 1, D);
  __syncwarp();
  return __ldg(nv + chosen);
}

// ---------------------------------------------------------------------------
// One step for the 32 walkers a warp owns (one per lane).  Steps whose
// degrees are all <= thr run on their own lane (thread bin); the others are
// taken one after another by the whole warp (warp bin).
__device__ __forceinline__ int32_t warp_binned_step(const GraphView& g, bool alive, int64_t t, int64_t v, int k,
                                                    uint64_t wid, uint64_t seed, uint32_t a_p, uint32_t a_q,
                                                    int thr, const WarpSmem& sm, int stream_ratio, int lane) {
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
    const int32_t xx = warp_step(g, tt, vv, k, uu, a_p, a_q, sm, stream_ratio, lane);
    if (lane == src) x = xx;
  }
  return x;
}

}  // namespace n2v
