/*
 * n2v.h -- C ABI of the GB300 (sm_103a) node2vec 2nd-order walk sampler.
 *
 * The library generates node2vec biased random walks (Zhou, Niu, Chen,
 * "Efficient Graph Computation for Node2Vec", arXiv 1805.00280) with every
 * transition distribution computed on the fly at the step that needs it
 * (Section 3.2), instead of stored per edge (Eq. 1 gives the memory the stored
 * form would take: 8 * sum_i d_i^2 bytes).
 *
 * Walk model (Section 2.1 and Algorithm 1).  A walker at v that arrived from t
 * gives each out-neighbour x of v the weight w(v,x) * alpha(t,x), with
 * alpha = 1/p if x == t, 1 if x is an out-neighbour of t, and 1/q otherwise;
 * the first step (superstep 0 of Algorithm 1) has no t and uses w(v,x)
 * alone.  A walk stores its l sampled vertices (the start is not stored).
 *
 * Integer contract (the same on every variant, so results are bit-exact):
 *   - alpha in Q16 fixed point, rounded once on the host:
 *       a_p = round_half_even(65536 / p), a_q = round_half_even(65536 / q),
 *       the return-free common-neighbour value is 65536;
 *   - c_x = w(v,x) * alpha as uint64, T = sum over N(v) (w == 1 if unweighted);
 *   - u = Philox4x32-10 (Salmon et al., SC'11) with key (lo32 seed, hi32 seed)
 *     and counter (k, lo32 walk_id, hi32 walk_id, 0), u = out[1]<<32 | out[0];
 *   - r = floor(u * T / 2^64); the chosen x is the first neighbour in CSR
 *     order whose inclusive prefix sum of c exceeds r;
 *   - T == 0 (no out-edges or all weights zero) ends the walk: that step and
 *     the later ones are written as -1.
 *
 * Graph: CSR with int64 row_ptr[n+1] (row_ptr[0] == 0, non-decreasing,
 * row_ptr[n] == nnz), int32 col[nnz] strictly increasing inside every row and
 * in [0, n), optional uint32 weights w[nnz].  Directed graphs use out-lists
 * (Section 3.2 analyses the undirected case and notes that directed graphs
 * work alike).
 *
 * Memory: the library never allocates device memory.  Every device buffer
 * (graph arrays, the auxiliary buffer, walk workspace, output) is owned by the
 * caller, who must keep it alive while the library uses it.  The library
 * allocates small host structures (the graph handle) with malloc.
 *
 * Streams: `stream` arguments are cudaStream_t values passed as void*
 * (NULL = the legacy default stream).  n2v_walk is asynchronous; argument
 * errors are returned synchronously, errors found on the device (a start
 * vertex out of range) are recorded in a device status word that
 * n2v_stream_status reads.
 *
 * Thread safety: distinct graph handles may be used from distinct threads.
 * Calls on one handle that overlap in time must use one stream.
 */
#ifndef N2V_H
#define N2V_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
#define N2V_OK 0
#define N2V_ERR_INVALID_ARG (-1)   /* a bad argument (null pointer, size, p, q ...) */
#define N2V_ERR_INVALID_GRAPH (-2) /* CSR is not canonical (see above)              */
#define N2V_ERR_OVERFLOW (-3)      /* max_v sum_x w(v,x) * max(a_p, 65536, a_q) >= 2^64 */
#define N2V_ERR_NO_MEM (-4)        /* a caller buffer is smaller than required       */
#define N2V_ERR_TIMEOUT (-5)       /* a bounded device wait gave up                  */
#define N2V_ERR_CUDA (-6)          /* a CUDA runtime call failed                     */
#define N2V_ERR_INTERNAL (-7)      /* a device self-check failed (checked build only: the
                                      library compiled with -DN2V_CHECKED verifies positions,
                                      spill indices, search bounds and stored totals on the
                                      device and records failures in the status word)   */

/* ---- sampler variants (n2v_walk `variant`) ------------------------------- */
/* One thread per walker and one launch per step (the plain form). */
#define N2V_PLAIN 0
/* One launch per step; inside it each warp serves 32 walkers and hands every
 * step whose degrees exceed the thread threshold to the whole warp. */
#define N2V_BINNED 1
/* One persistent launch for all steps of all walkers: warps take batches of
 * walkers from a device work counter and run all l steps, binning each step
 * by degree (one lane, or the whole warp). */
#define N2V_PERSISTENT 2
/* Flag: record the launch sequence of the call as a CUDA graph the first time
 * a shape is seen on a handle, and replay it afterwards. */
#define N2V_FLAG_CUDA_GRAPH 0x100

/* ---- tuning ---------------------------------------------------------------- */
typedef struct n2v_tune {
  int32_t block_threads;   /* threads per block of the binned/persistent kernels (64..256, x32;
                              default 128)                                                    */
  int32_t blocks_per_sm;   /* resident blocks per SM for the persistent grid; 0 = 20 resident
                              warps per SM where block_threads divides that, else 16, capped by
                              shared memory.  The persistent kernel is compiled for 128, 96, 80
                              and 64 registers a thread; the resident warps per SM (<= 16, 20,
                              24, more) select the budget.                                    */
  int32_t thread_max_deg;  /* a step runs on one lane when deg(v) and deg(t) are <= this      */
  int32_t smem_specials;   /* per-warp shared-memory slots for the special positions of a step */
  int32_t hub_count;       /* vertices (largest degree first) with a hashed neighbour set     */
  int32_t hub_min_degree;  /* a vertex needs at least this degree to get a hashed set         */
  int32_t chunk_walkers;   /* walkers per persistent launch (0 = all in one launch)           */
  int32_t hub_budget_mb;   /* MiB of device memory for all hub hash sets (8 bytes per slot)   */
  int32_t stage_window;    /* elements per shared-memory window that stages the longer list of
                              a step by TMA bulk copies (power of two, 64..4096; 0 = never) */
  int32_t stream_ratio;    /* x10: stage the longer list when its length is at most
                              stream_ratio/10 * 32*ceil(short/32) * log2(long) (else probe it) */
  int32_t spill_specials;  /* per-warp device-workspace slots for special neighbours that do
                              not fit in shared memory (persistent sampler)                 */
  int32_t stage_buffers;   /* staging windows in flight per warp (2 or 4)                    */
  int32_t bitmap_hubs;     /* vertices (largest degree first, whole degree classes, degree >=
                              hub_min_degree) with a rank bitmap: one bit per vertex of the
                              graph and a running count per 64 bits (n/4 bytes a hub), so that
                              "is x in N(h)" and x's index in N(h) take one 16-byte load     */
  int32_t block_min_deg;   /* 0: warps run their walkers independently.  > 0: the blocks of
                              the persistent sampler advance 128 walkers together, step by step,
                              and a step whose longer list has at least this many entries is
                              taken by the whole block (four warps) instead of one warp      */
  int32_t merge_ratio;     /* x10: a step whose two lists both fit a staging window is taken by
                              a merge of the two lists in shared memory (each lane one segment
                              of the merge path) when deg v + deg t <= merge_ratio/10 *
                              32*ceil(short/32) * log2(long); 0 = never                     */
  int32_t l2_persist_mb;   /* MiB at the start of col that the persistent sampler's launches mark
                              as persisting in L2 (an access-policy window; the context's
                              persisting set-aside is raised to match, up to the device's
                              maximum).  On degree-ordered vertex ids the start of col holds the
                              largest hubs' lists.  0 = off                                   */
  int32_t reserved[1];     /* must be zero                                                    */
} n2v_tune;

/* Fill *t with the library defaults. */
void n2v_tune_default(n2v_tune* t);

/* ---- graph ----------------------------------------------------------------- */
typedef struct n2v_graph n2v_graph; /* opaque handle */

typedef struct n2v_graph_info {
  int64_t n, nnz;
  int32_t weighted;
  int32_t hub_count;      /* hubs that received a hashed neighbour set */
  int64_t max_degree;
  uint64_t max_wsum;      /* max over v of sum_x w(v,x) (= max degree when unweighted) */
  int64_t hub_min_degree; /* smallest degree among the hubs (0 if none) */
  int64_t hub_slots;      /* total slots of all hub hash sets */
  int64_t deg_hist[34];   /* [0]: degree 0; [i>=1]: degree in [2^(i-1), 2^i) */
  uint32_t w_min, w_max;  /* extreme edge weights (1, 1 when unweighted) */
  int32_t bitmap_hubs;    /* hubs that received a rank bitmap */
  int32_t reserved0;
  int64_t bitmap_min_degree; /* smallest degree among them (0 if none) */
} n2v_graph_info;

/* Bytes of device memory the caller must provide as `aux` to n2v_graph_load
 * for a graph of this size under tuning `t` (NULL = defaults).  Holds the
 * device status word, degree statistics, the per-edge static weight prefix of
 * weighted graphs (8 bytes per entry) and the hub neighbour caches (the GPU
 * counterparts of the FN-Cache neighbour cache, Section 3.4): hashed
 * neighbour sets (8 bytes per slot) and rank bitmaps (16 bytes per 64
 * vertices of the graph, per bitmap hub). */
int n2v_graph_aux_bytes(int64_t n, int64_t nnz, int weighted, const n2v_tune* t, size_t* bytes);

/* Validate a device-resident CSR graph and build its auxiliary structures in
 * `aux` (device memory of at least n2v_graph_aux_bytes bytes, 256-byte
 * aligned).  col must be 16-byte aligned (it is read by bulk copies) and
 * every degree must be below 2^30.  row_ptr, col, w and aux are BORROWED device pointers: the
 * caller keeps them alive until n2v_graph_free.  w may be NULL (unweighted).
 * Synchronises `stream` (this is set-up, not the hot path).  Returns
 * N2V_ERR_INVALID_GRAPH for a non-canonical CSR, N2V_ERR_NO_MEM when
 * aux_bytes is too small.  On success *out receives a new handle. */
int n2v_graph_load(const int64_t* row_ptr, const int32_t* col, const uint32_t* w, int64_t n, int64_t nnz,
                   void* aux, size_t aux_bytes, const n2v_tune* t, void* stream, n2v_graph** out);

/* Host copy of the statistics computed at load. */
int n2v_graph_info_get(const n2v_graph* g, n2v_graph_info* info);

/* Replace the tuning of a loaded graph.  Fields that size `aux` (hub_count,
 * hub_budget_mb, bitmap_hubs) must not grow beyond what aux was sized for
 * (N2V_ERR_NO_MEM); the hub caches are rebuilt on `stream` when a field that
 * shapes them changed.  Synchronises `stream`. */
int n2v_graph_retune(n2v_graph* g, const n2v_tune* t, void* stream);

/* Release the handle (and any CUDA graphs recorded on it).  Device buffers
 * stay the caller's. */
void n2v_graph_free(n2v_graph* g);

/* ---- walks ----------------------------------------------------------------- */

/* Bytes of device workspace n2v_walk needs for `walk_count` walks of length l
 * with `variant` (0 is a valid answer; ws may then be NULL). */
int n2v_walk_ws_bytes(const n2v_graph* g, int64_t walk_count, int32_t l, int variant, size_t* bytes);

/* Generate walks with ids [walk_begin, walk_begin + walk_count) of the job
 * "r walks from each of the n_starts vertices in `starts`" (Section 2.1: r
 * walks of length l per vertex).  Walk ids are round-major: id = round *
 * n_starts + i starts at starts[i], so one call, or any split of the id range
 * into several calls (chunking as in FN-Multi, Section 3.4; sharding over
 * devices), gives the same rows.
 *   starts   device int32 [n_starts], each in [0, n)
 *   walks    device int32 [walk_count][l], row-major; row i is walk id
 *            walk_begin + i
 *   ws       device workspace of n2v_walk_ws_bytes bytes (256-byte aligned)
 *   p, q     node2vec return / in-out parameters, finite and > 0, with
 *            65536/p and 65536/q rounding into [1, 2^24]
 *   seed     Philox key
 *   variant  N2V_PLAIN, N2V_BINNED or N2V_PERSISTENT, optionally | N2V_FLAG_CUDA_GRAPH
 * Asynchronous on `stream`.  Returns N2V_ERR_OVERFLOW when the weighted
 * totals could exceed 64 bits for these p, q.  A start vertex out of range
 * writes -1 rows and sets N2V_ERR_INVALID_ARG in the status word. */
int n2v_walk(const n2v_graph* g, const int32_t* starts, int64_t n_starts, int32_t r, int32_t l, double p,
             double q, uint64_t seed, int64_t walk_begin, int64_t walk_count, int32_t* walks, void* ws,
             size_t ws_bytes, int variant, void* stream);

/* Walks streamed to host memory, for outputs larger than device memory (the
 * output side of FN-Multi, Section 3.4: walkers run in rounds and each
 * round's walks are written out before the next).  The walk ids
 * [walk_begin, walk_begin + walk_count) of the job "r walks from each start"
 * run in chunks of ring_walks walks, each chunk one n2v_walk call on `stream`
 * into slot (chunk mod ring_slots) of a device ring; once a chunk is written
 * its rows are copied to host_walks by one cudaMemcpyAsync on copy_stream,
 * while the next chunk runs.  A chunk reuses a slot only after that slot's
 * previous copy finished (events, no host wait).  The rows are those of one
 * n2v_walk call over the whole range.
 *   host_walks  host int32 [walk_count][l]; pinned (cudaHostAlloc /
 *               cudaHostRegister) for the copies to overlap
 *   dev_ring    device int32 [ring_slots][ring_walks][l], caller-owned
 *   ring_slots  1 .. 8 (2 lets one chunk compute while the previous copies)
 *   ws          as for n2v_walk with walk_count = ring_walks
 *   variant     N2V_PLAIN, N2V_BINNED or N2V_PERSISTENT (no N2V_FLAG_CUDA_GRAPH)
 *   copy_stream a stream other than `stream` (NULL: the copies go on `stream`
 *               and do not overlap)
 * Asynchronous: when `stream` reaches the end of the call's work, every row
 * is in host_walks (the call makes `stream` wait for the last copies).
 * Creates and releases a few CUDA events (no device memory). */
int n2v_walk_stream(const n2v_graph* g, const int32_t* starts, int64_t n_starts, int32_t r, int32_t l, double p,
                    double q, uint64_t seed, int64_t walk_begin, int64_t walk_count, int32_t* host_walks,
                    int32_t* dev_ring, int64_t ring_walks, int32_t ring_slots, void* ws, size_t ws_bytes,
                    int variant, void* stream, void* copy_stream);

/* Allocation-free form of n2v_walk with variant N2V_PERSISTENT, for callers
 * that cannot allocate device memory (code running inside a memory pool or
 * arena owned by another runtime, plugins handed only a stream and their
 * input/output buffers, paths where an allocation could block or fail).
 * The paper has no counterpart: it only concerns memory management.
 *
 * Instead of a caller workspace it uses a scratch array inside the library
 * (4 MiB of device memory per GPU that loads the library, held until the
 * process exits).  Arguments and results are those of n2v_walk; the rows are
 * identical.  The first call on a device looks up that device's scratch
 * address (cudaGetSymbolAddress): make that first call before any stream
 * capture.  Every call on a device shares the one scratch array: calls that
 * overlap on the GPU (other streams, other threads, other graph handles)
 * race and give wrong rows; serialise them.  The scratch keeps the last
 * call's contents and each call clears what must start at zero.  The
 * device current at the call must be the one the graph was loaded on (its
 * scratch is the one used), else N2V_ERR_INVALID_ARG.  Returns
 * N2V_ERR_NO_MEM when the call would need more than 512 persistent launches
 * (walk_count / chunk_walkers), otherwise as n2v_walk.  Allocates nothing. */
int n2v_walk_noalloc(const n2v_graph* g, const int32_t* starts, int64_t n_starts, int32_t r, int32_t l, double p,
                     double q, uint64_t seed, int64_t walk_begin, int64_t walk_count, int32_t* walks, void* stream);

/* n2v_walk with FN-Approx (Section 3.4, Eq. 2-3): at a step from t to a
 * popular v (deg v >= popular_degree) where t is not popular (deg t <
 * popular_degree), the bounds LB, UB on the probability of moving to any
 * x != t are computed from deg v, deg t, the Q16 return parameters and the
 * graph's extreme weights; when UB - LB < eps the step samples by static
 * weights w(v, x) with the same draw.  The decision is made in IEEE double,
 * one rounding per operation in a fixed order, so every implementation of the
 * rule takes the same branch.  The bounds assume t is a neighbour of v
 * (undirected graphs).  The rows are approximate node2vec walks (not the exact
 * distribution); eps = 0 gives the exact rows of n2v_walk. */
int n2v_walk_approx(const n2v_graph* g, const int32_t* starts, int64_t n_starts, int32_t r, int32_t l, double p,
                    double q, uint64_t seed, int64_t walk_begin, int64_t walk_count, int32_t* walks, void* ws,
                    size_t ws_bytes, int variant, double eps, int64_t popular_degree, void* stream);

/* Q16 return parameters exactly as n2v_walk rounds them (host function). */
int n2v_alpha_q16(double p, double q, uint32_t* a_p, uint32_t* a_q);

/* Count, over walk rows [walk_begin, walk_begin + walk_count) that n2v_walk
 * wrote to `walks`, the real transitions (entries != -1) and the adjacency
 * bytes of the per-step model of Section 3.2 (N(v) read locally, N(t) as the
 * NEIG message): 16 + 4*deg(v)*(1 + weighted) + [k >= 1]*(16 + 4*deg(t)) + 4,
 * and of the lower model without the N(t) term: 16 + 4*deg(v)*(1 + weighted) + 4.
 * out3 is DEVICE uint64[3] and is overwritten: out3[0] = transitions,
 * out3[1] = model bytes, out3[2] = lower-model bytes.  Asynchronous on `stream`. */
int n2v_walk_traffic(const n2v_graph* g, const int32_t* starts, int64_t n_starts, int64_t walk_begin,
                     int64_t walk_count, int32_t l, const int32_t* walks, uint64_t* out3, void* stream);

/* Synchronise `stream`, return and clear the device status word of `g`
 * (N2V_OK, N2V_ERR_INVALID_ARG, N2V_ERR_TIMEOUT or, in the checked build,
 * N2V_ERR_INTERNAL), or N2V_ERR_CUDA when the stream reports a CUDA error. */
int n2v_stream_status(const n2v_graph* g, void* stream);

/* ---- autotuner -------------------------------------------------------------- */

/* Workspace bytes n2v_autotune needs for a sample of `sample` walks of length l. */
int n2v_autotune_ws_bytes(const n2v_graph* g, int64_t sample, int32_t l, size_t* bytes);

/* Pick the tuning of the persistent sampler for this graph and job shape:
 * a coordinate descent over stage_window, blocks_per_sm, stream_ratio,
 * merge_ratio, thread_max_deg, stage_buffers, smem_specials, block_min_deg
 * and, from none up to the sizes the graph was loaded with, bitmap_hubs and
 * hub_count (l2_persist_mb is left as given),
 * each candidate timed with CUDA events on walks [0, sample) of
 * the job "one walk from each of starts[0..sample)" (the caller should pass a
 * representative random sample of its start vertices).  A candidate is
 * timed as the faster of two runs (after one untimed run) and replaces the
 * current tuning only when it is at least 2% faster.  Every tuning gives
 * the same rows, so only time is compared.  `walks` (device int32
 * [sample][l]) and `ws` (n2v_autotune_ws_bytes) are scratch.  Synchronises
 * `stream`.  On success the best tuning is applied to g and returned in
 * *best (and its sample time in *best_ms). */
int n2v_autotune(n2v_graph* g, const int32_t* starts, int64_t n_starts, int32_t l, double p, double q, uint64_t seed,
                 int64_t sample, int32_t* walks, void* ws, size_t ws_bytes, void* stream, n2v_tune* best,
                 float* best_ms);

/* ---- serving: continuous batching of walk jobs ------------------------------- */
/* A job: one walk (r = 1) of length l from each of its n_starts start vertices
 * (repeats allowed), with its own p, q and seed.  Its rows are bit-identical
 * to n2v_walk(g, starts, n_starts, 1, l, p, q, seed, 0, n_starts, ...),
 * whatever other jobs it is mixed with.  There is no serving in the paper;
 * the job granularity plays the role of FN-Multi's rounds (Section 3.4). */
typedef struct n2v_job {
  const int32_t* starts;  /* HOST int32 [n_starts]; copied at submit */
  int64_t n_starts;
  int32_t l;
  int32_t reserved0;
  double p, q;
  uint64_t seed;
} n2v_job;

typedef struct n2v_serve_cfg {
  int64_t tick_walkers;      /* walkers per tick (one persistent launch)            */
  int32_t max_jobs_per_tick; /* jobs mixed into one tick                            */
  int32_t spill_specials;    /* per-warp spill slots (inside the arena)             */
  int64_t min_share;         /* smallest share of a tick given to one job           */
  int64_t reserved[4];
} n2v_serve_cfg;

typedef struct n2v_serve_stats_t {
  int64_t queued, active, arena_used, arena_bytes, ticks;
} n2v_serve_stats_t;

typedef struct n2v_server n2v_server; /* opaque */

void n2v_serve_cfg_default(n2v_serve_cfg* cfg);

/* A server over a loaded graph.  `arena` (device, caller-owned, 256-byte
 * aligned) holds the tick tables and, for every admitted job, its start
 * vertices and output rows: a job is admitted (in submission order) when its
 * bytes, 4*n_starts + 4*n_starts*l rounded up to 256, fit in the free part of
 * the arena -- admission by free HBM.  All device work goes on `stream`. */
int n2v_serve_create(const n2v_graph* g, void* arena, size_t arena_bytes, const n2v_serve_cfg* cfg, void* stream,
                     n2v_server** out);
/* Queue a job (host call, returns at once); *job_id identifies it. */
int n2v_serve_submit(n2v_server* s, const n2v_job* job, int64_t* job_id);
/* Non-blocking scheduler step: retire ticks the GPU finished, admit queued
 * jobs that fit, and, unless a tick is already queued, launch the next tick:
 * one persistent launch over up to tick_walkers walkers drawn from every
 * active job (equal shares).  *launched = 1 when a tick was launched. */
int n2v_serve_step(n2v_server* s, int* launched);
/* Up to max_ids finished job ids, oldest first. */
int n2v_serve_poll(n2v_server* s, int64_t* ids, int max_ids, int* n);
/* Device pointer to a finished job's rows, int32 [n_starts][l]. */
int n2v_serve_job_rows(n2v_server* s, int64_t job_id, int32_t** rows);
/* Give a finished job's arena space back (its rows become invalid). */
int n2v_serve_release(n2v_server* s, int64_t job_id);
int n2v_serve_stats(n2v_server* s, n2v_serve_stats_t* st);
/* Destroy the server (synchronise the stream first; the arena stays the caller's). */
void n2v_serve_destroy(n2v_server* s);

/* Failure-path self-test (failure detection without a GPU fault; the paper has no counterpart):
 * launch one warp that waits on an mbarrier nothing arrives on, with the
 * samplers' bounded wait and a limit of limit_cycles SM cycles (1 .. 2^34).
 * It gives up, records N2V_ERR_TIMEOUT in the status word of g and returns;
 * no fault, no trap.  n2v_stream_status then reports (and clears) it. */
int n2v_selftest_timeout(const n2v_graph* g, int64_t limit_cycles, void* stream);

/* Static text for a status code. */
const char* n2v_strerror(int code);

/* ---- stored transition tables (the baseline the paper avoids) ------------------
 * Section 3.2, Eq. 1: precomputing every transition distribution takes one
 * 8-byte value per (edge t->v, neighbour x of v) pair, 8 * sum_i d_i^2 bytes on
 * an undirected graph.  These calls build that table for one (p, q) -- the
 * cumulative weights C_j = sum_{i<=j} w(v,x_i) alpha(t,x_i) over N(v) for each
 * edge, in CSR edge order -- and walk with it: a step is one binary search of
 * r = floor(u * T / 2^64) in the stored C, so the rows equal n2v_walk's for
 * the same (p, q, seed) bit for bit.  It exists to measure the memory and time
 * the on-the-fly sampler saves.
 *
 * n2v_stored_bytes: size of the table buffer (header, per-edge offsets, scan
 *   scratch, 8 bytes per entry) and the entry count sum_e deg(col[e]).
 *   Synchronises `stream`.
 * n2v_stored_build: fill a caller-owned, 256-byte-aligned device buffer of at
 *   least n2v_stored_bytes bytes for (p, q).  N2V_ERR_NO_MEM if smaller,
 *   N2V_ERR_OVERFLOW as for n2v_walk.  Asynchronous after the size check.
 * n2v_stored_walk: walks of the job "r walks from each start" (same walk ids,
 *   draws and output layout as n2v_walk), with the (p, q) the table was built
 *   for.  N2V_ERR_INVALID_ARG if the table was not built for this graph handle.
 *   Reads the table header synchronously, then launches asynchronously; start
 *   vertices out of range are reported through n2v_stream_status. */
int n2v_stored_bytes(const n2v_graph* g, void* stream, size_t* bytes, int64_t* entries);
int n2v_stored_build(const n2v_graph* g, double p, double q, void* table, size_t table_bytes, void* stream);
int n2v_stored_walk(const n2v_graph* g, const void* table, const int32_t* starts, int64_t n_starts, int32_t r,
                    int32_t l, uint64_t seed, int64_t walk_begin, int64_t walk_count, int32_t* walks, void* stream);

/* Step statistics of the stats build (the library compiled with
 * -DN2V_STATS; the paper has no counterpart): out[0..n) receives, summed over
 * every sampler launch since the last reset, per kind of step the number of
 * steps, the SM clock cycles lane 0 of the warp spent in them and the lengths
 * of their shorter and longer lists (layout: lane-tier batches and cycles,
 * first steps and cycles, then four words per generator mode 0..4, then
 * segment re-enumerations, spilled steps, the warps' total cycles in the
 * persistent loop, and for the staged steps their chunks of keys, windows
 * landed and window searches).  Synchronises the device; reset != 0 zeroes the counters.
 * Other builds fill out with zeros and return N2V_ERR_INVALID_ARG.  n <= 32. */
int n2v_step_stats(uint64_t* out, int32_t n, int32_t reset);

/* Number of SMs and the persistent grid the handle would launch: blocks of
 * 128 threads, as many per SM as the tuning's resident warps ask for (20 by
 * default) and shared memory holds. */
int n2v_launch_shape(const n2v_graph* g, int32_t* sms, int32_t* blocks, int32_t* threads);

#ifdef __cplusplus
}
#endif
#endif /* N2V_H */
