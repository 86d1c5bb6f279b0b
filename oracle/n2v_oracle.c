/*
 * CPU oracle for node2vec 2nd-order walks -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, single-threaded, deliberately slow restatement of the walk model
 * of Section 2.1 / Section 3.2 (Algorithm 1) under the integer contract in
 * n2v_oracle.h.  Every step computes the full list of unnormalised weights
 * over N(v) in CSR order, the total, and then the first inclusive prefix
 * above the scaled draw.  There is no blocking, no fusion and no shortcut:
 * membership of x in N(t) is a library binary search (bsearch) over the sorted
 * adjacency list of t, which is the "is x a common neighbour of t and v" test
 * of Section 3.2 in a form that can be checked by eye.
 *
 * Nothing in the CUDA sampler includes, links or calls this file.
 */
#include "n2v_oracle.h"

#include <math.h>
#include <stdlib.h>

/* ---------------------------------------------------------------------- */
/* Philox4x32-10, from the definition in Salmon et al., SC'11:             */
/*   round: (c0,c1,c2,c3) -> (hi(M1*c2)^c1^k0, lo(M1*c2), hi(M0*c0)^c3^k1, */
/*          lo(M0*c0)); the key is bumped by the Weyl constants between    */
/*   rounds.                                                                */

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void n2v_oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    uint64_t prod0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
    uint64_t prod1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

uint64_t n2v_oracle_draw(uint64_t seed, uint64_t walk_id, uint32_t k) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t ctr[4] = {k, (uint32_t)walk_id, (uint32_t)(walk_id >> 32), 0u};
  uint32_t out[4];
  n2v_oracle_philox4x32_10(ctr, key, out);
  return ((uint64_t)out[1] << 32) | (uint64_t)out[0];
}

/* ---------------------------------------------------------------------- */
/* alpha in Q16 fixed point, rounded once: nearbyint() under the default    */
/* rounding mode is round-half-to-even on the IEEE double quotient.        */

int n2v_oracle_alpha_q16(double p, double q, uint32_t* a_p, uint32_t* a_q) {
  if (!(isfinite(p) && isfinite(q)) || !(p > 0.0) || !(q > 0.0)) return -1;
  double xp = nearbyint(65536.0 / p);
  double xq = nearbyint(65536.0 / q);
  if (!(xp >= 1.0 && xp <= 16777216.0 && xq >= 1.0 && xq <= 16777216.0)) return -1;
  *a_p = (uint32_t)xp;
  *a_q = (uint32_t)xq;
  return 0;
}

/* ---------------------------------------------------------------------- */
/* One step.                                                                */

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/* Is x an out-neighbour of t?  Binary search over the sorted list N(t). */
static int is_neighbour(const int64_t* row_ptr, const int32_t* col, int64_t t, int32_t x) {
  int64_t b = row_ptr[t], e = row_ptr[t + 1];
  if (e <= b) return 0;
  return bsearch(&x, col + b, (size_t)(e - b), sizeof(int32_t), cmp_i32) != NULL;
}

/* The Q16 return parameter alpha(t, x) of the 2nd-order model. */
static uint64_t alpha_of(const int64_t* row_ptr, const int32_t* col, int64_t t, int32_t x, uint32_t a_p,
                         uint32_t a_q) {
  if ((int64_t)x == t) return a_p;                    /* dist(t, x) = 0 */
  if (is_neighbour(row_ptr, col, t, x)) return 65536u; /* dist(t, x) = 1 */
  return a_q;                                          /* dist(t, x) = 2 */
}

int64_t n2v_oracle_step(const int64_t* row_ptr, const int32_t* col, const uint32_t* w, int64_t t,
                        int64_t v, int32_t k, uint32_t a_p, uint32_t a_q, uint64_t u, uint64_t* total) {
  int64_t b = row_ptr[v], e = row_ptr[v + 1];
  /* unnormalised weights and their total */
  uint64_t T = 0;
  for (int64_t j = b; j < e; ++j) {
    uint64_t wt = w ? (uint64_t)w[j] : 1u;
    uint64_t a = (k == 0) ? 1u : alpha_of(row_ptr, col, t, col[j], a_p, a_q);
    T += wt * a;
  }
  if (total) *total = T;
  if (T == 0) return -1;
  /* r = floor(u * T / 2^64) */
  uint64_t r = (uint64_t)(((unsigned __int128)u * (unsigned __int128)T) >> 64);
  /* first inclusive prefix above r */
  uint64_t C = 0;
  for (int64_t j = b; j < e; ++j) {
    uint64_t wt = w ? (uint64_t)w[j] : 1u;
    uint64_t a = (k == 0) ? 1u : alpha_of(row_ptr, col, t, col[j], a_p, a_q);
    C += wt * a;
    if (C > r) return j - b;
  }
  return -1; /* unreachable: C reaches T > r */
}

/* ---------------------------------------------------------------------- */
/* Whole walks (Algorithm 1: l stored steps per walk, step 0 by static      */
/* weights, then one 2nd-order step per superstep).                         */

void n2v_oracle_walk(const int64_t* row_ptr, const int32_t* col, const uint32_t* w,
                     const int32_t* starts, int64_t n_starts, int32_t l, uint32_t a_p, uint32_t a_q,
                     uint64_t seed, const int64_t* walk_ids, int64_t n_ids, int32_t* out) {
  for (int64_t i = 0; i < n_ids; ++i) {
    uint64_t wid = (uint64_t)walk_ids[i];
    int32_t* row = out + i * (int64_t)l;
    int64_t t = -1;
    int64_t v = starts[wid % (uint64_t)n_starts];
    int32_t k = 0;
    for (; k < l; ++k) {
      uint64_t u = n2v_oracle_draw(seed, wid, (uint32_t)k);
      int64_t j = n2v_oracle_step(row_ptr, col, w, t, v, k, a_p, a_q, u, NULL);
      if (j < 0) break;
      int32_t x = col[row_ptr[v] + j];
      row[k] = x;
      t = v;
      v = x;
    }
    for (; k < l; ++k) row[k] = -1;
  }
}

void n2v_oracle_traffic(const int64_t* row_ptr, int weighted, const int32_t* starts, int64_t n_starts,
                        const int64_t* walk_ids, int64_t n_ids, const int32_t* walks, int32_t l,
                        uint64_t out[3]) {
  uint64_t steps = 0, bytes = 0, lower = 0;
  for (int64_t i = 0; i < n_ids; ++i) {
    const int32_t* row = walks + i * (int64_t)l;
    int64_t s0 = starts[(uint64_t)walk_ids[i] % (uint64_t)n_starts];
    for (int32_t k = 0; k < l; ++k) {
      if (row[k] < 0) break;
      int64_t v = (k == 0) ? s0 : row[k - 1];
      uint64_t dv = (uint64_t)(row_ptr[v + 1] - row_ptr[v]);
      uint64_t b = 16 + 4 * dv * (weighted ? 2 : 1) + 4; /* N(v) read locally, output */
      lower += b;
      if (k >= 1) { /* N(t) as the NEIG message */
        int64_t t = (k == 1) ? s0 : row[k - 2];
        b += 16 + 4 * (uint64_t)(row_ptr[t + 1] - row_ptr[t]);
      }
      steps += 1;
      bytes += b;
    }
  }
  out[0] = steps;
  out[1] = bytes;
  out[2] = lower;
}

/* ---------------------------------------------------------------------- */
/* FN-Approx (Section 3.4, Eq. 2-3).                                        */
/* The bounds are those of the paper for 1/p <= 1 <= 1/q, written for any   */
/* order of 1 and 1/q: a neighbour x != t has alpha 1 (common neighbour) or  */
/* 1/q, at most min(deg t, deg v - 1) neighbours can be common, t itself     */
/* carries 1/p, and every weight lies in [w_min, w_max].                     */

int n2v_oracle_approx_decide(int64_t deg_v, int64_t deg_t, uint32_t a_p, uint32_t a_q, uint32_t w_min,
                             uint32_t w_max, double eps, double bounds[2]) {
  const double ip = (double)a_p / 65536.0; /* 1/p in Q16, exact in double */
  const double iq = (double)a_q / 65536.0; /* 1/q */
  const double wmin = (double)w_min, wmax = (double)w_max;
  const double others = (double)(deg_v - 1);
  const double cmax = (double)(deg_t < deg_v - 1 ? deg_t : deg_v - 1);
  /* numerator of P(v -> x), x != t */
  const double num_min = wmin * (iq < 1.0 ? iq : 1.0);
  const double num_max = wmax * (iq < 1.0 ? 1.0 : iq);
  /* the total over N(v) is smallest with the smaller alpha on as many
   * neighbours as allowed, largest with the larger one */
  const double all_q = ip + others * iq;                 /* no common neighbour */
  const double most_1 = (ip + cmax) + (others - cmax) * iq; /* as many as allowed */
  const double den_min = wmin * (iq >= 1.0 ? most_1 : all_q);
  const double den_max = wmax * (iq >= 1.0 ? all_q : most_1);
  const double lb = num_min / den_max;
  const double ub = num_max / den_min;
  if (bounds) {
    bounds[0] = lb;
    bounds[1] = ub;
  }
  return (ub - lb) < eps;
}

void n2v_oracle_walk_approx(const int64_t* row_ptr, const int32_t* col, const uint32_t* w,
                            const int32_t* starts, int64_t n_starts, int32_t l, uint32_t a_p, uint32_t a_q,
                            uint64_t seed, const int64_t* walk_ids, int64_t n_ids, double eps,
                            int64_t popular, uint32_t w_min, uint32_t w_max, int32_t* out, uint64_t counts[2]) {
  uint64_t n_approx = 0, n_second = 0;
  for (int64_t i = 0; i < n_ids; ++i) {
    uint64_t wid = (uint64_t)walk_ids[i];
    int32_t* row = out + i * (int64_t)l;
    int64_t t = -1;
    int64_t v = starts[wid % (uint64_t)n_starts];
    int32_t k = 0;
    for (; k < l; ++k) {
      uint64_t u = n2v_oracle_draw(seed, wid, (uint32_t)k);
      int32_t kk = k; /* the step index the weights use: 0 means static weights */
      if (k >= 1) {
        int64_t dv = row_ptr[v + 1] - row_ptr[v], dt = row_ptr[t + 1] - row_ptr[t];
        ++n_second;
        if (dv >= popular && dt < popular &&
            n2v_oracle_approx_decide(dv, dt, a_p, a_q, w_min, w_max, eps, NULL)) {
          kk = 0;
          ++n_approx;
        }
      }
      int64_t j = n2v_oracle_step(row_ptr, col, w, t, v, kk, a_p, a_q, u, NULL);
      if (j < 0) break;
      int32_t x = col[row_ptr[v] + j];
      row[k] = x;
      t = v;
      v = x;
    }
    for (; k < l; ++k) row[k] = -1;
  }
  if (counts) {
    counts[0] = n_approx;
    counts[1] = n_second;
  }
}
