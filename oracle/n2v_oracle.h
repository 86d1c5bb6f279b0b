/*
 * CPU oracle for node2vec 2nd-order walks -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this library.  The product path (the CUDA sampler) never calls it
 * and shares no code with it.
 *
 * The walk model (Section 2.1 and Section 3.2 of the paper, Algorithm 1):
 * a walker at v that arrived from t gives every out-neighbour x of v the
 * unnormalised weight w(v,x) * alpha(t,x), with alpha = 1/p when x == t,
 * 1 when x is a neighbour of t, and 1/q otherwise; the first step has no t
 * and uses w(v,x) alone (Algorithm 1, superstep 0).
 *
 * Integer contract used to make the result exact and reproducible:
 *   - alpha in Q16: a_p = round_half_even(65536/p), a_q likewise, a_1 = 65536;
 *   - c_x = w(v,x) * alpha as uint64, T = sum of c_x in CSR order;
 *   - u = 64-bit Philox4x32-10 draw keyed by (seed; step k, walk id);
 *   - r = floor(u * T / 2^64); the chosen neighbour is the first x in CSR order
 *     whose inclusive prefix C_x exceeds r;
 *   - T == 0 (no out-edges, or all weights zero) ends the walk: that step and
 *     every later one is written as -1.
 */
#ifndef N2V_ORACLE_H
#define N2V_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11). */
void n2v_oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* The 64-bit draw of walk `walk_id` at step `k`: key (lo32 seed, hi32 seed),
 * counter (k, lo32 walk_id, hi32 walk_id, 0), u = out[1] << 32 | out[0]. */
uint64_t n2v_oracle_draw(uint64_t seed, uint64_t walk_id, uint32_t k);

/* Q16 return parameters.  Returns 0, or -1 when p or q is not a positive
 * finite number or a quantised value falls outside [1, 2^24]. */
int n2v_oracle_alpha_q16(double p, double q, uint32_t* a_p, uint32_t* a_q);

/* One step at v (k >= 1: arrived from t; k == 0: t ignored) with draw u.
 * Returns the chosen CSR index j in [0, deg(v)) or -1 when T == 0; writes
 * the total T through *total when total is not NULL. */
int64_t n2v_oracle_step(const int64_t* row_ptr, const int32_t* col, const uint32_t* w, int64_t t,
                        int64_t v, int32_t k, uint32_t a_p, uint32_t a_q, uint64_t u, uint64_t* total);

/* Walks for the given walk ids.  Walk id i starts at starts[i mod n_starts]
 * (ids are round-major: id = round * n_starts + index).  out is row-major
 * [n_ids][l].  w may be NULL (every weight 1). */
void n2v_oracle_walk(const int64_t* row_ptr, const int32_t* col, const uint32_t* w,
                     const int32_t* starts, int64_t n_starts, int32_t l, uint32_t a_p, uint32_t a_q,
                     uint64_t seed, const int64_t* walk_ids, int64_t n_ids, int32_t* out);

/* FN-Approx (Section 3.4, Eq. 2-3): at a popular v (degree >= popular) reached
 * from an unpopular t (degree < popular), the bounds
 *   LB = num_min / den_max,  UB = num_max / den_min
 * on the probability of moving to any x != t are computed from deg(v), deg(t),
 * the Q16 return parameters and the extreme edge weights w_min, w_max of the
 * graph; when UB - LB < eps the step ignores the 2nd-order factor and samples
 * by static weights with the same draw.  The bounds and the comparison are
 * evaluated in IEEE double, one rounding per operation, in the order written
 * in n2v_oracle.c.  Returns 1 when the step is approximated. */
int n2v_oracle_approx_decide(int64_t deg_v, int64_t deg_t, uint32_t a_p, uint32_t a_q, uint32_t w_min,
                             uint32_t w_max, double eps, double bounds[2]);

/* n2v_oracle_walk with FN-Approx applied at the steps where it decides so.
 * counts (may be NULL) receives [approximated steps, all 2nd-order steps]. */
void n2v_oracle_walk_approx(const int64_t* row_ptr, const int32_t* col, const uint32_t* w,
                            const int32_t* starts, int64_t n_starts, int32_t l, uint32_t a_p, uint32_t a_q,
                            uint64_t seed, const int64_t* walk_ids, int64_t n_ids, double eps,
                            int64_t popular, uint32_t w_min, uint32_t w_max, int32_t* out, uint64_t counts[2]);

/* Counts of the given walk rows: out[0] = real transitions (entries != -1),
 * out[1] = adjacency bytes by the per-step model
 *   16 + 4*deg(v)*(1 + weighted) + [k >= 1] * (16 + 4*deg(t)) + 4,
 * out[2] = bytes by the lower model without the N(t) term,
 *   16 + 4*deg(v)*(1 + weighted) + 4. */
void n2v_oracle_traffic(const int64_t* row_ptr, int weighted, const int32_t* starts, int64_t n_starts,
                        const int64_t* walk_ids, int64_t n_ids, const int32_t* walks, int32_t l,
                        uint64_t out[3]);

#ifdef __cplusplus
}
#endif
#endif
