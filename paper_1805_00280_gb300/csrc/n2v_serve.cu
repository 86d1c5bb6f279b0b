// Serving: continuous batching of walk jobs on a resident graph.
//
// Jobs (own starts, p, q, l, seed) are admitted when their start vertices and
// output rows fit in the caller's arena (device memory it owns); admitted jobs
// are mixed into "ticks": one persistent launch over walker slots drawn from
// every active job.  A job that arrives while others run joins at the next
// tick.  Walk ids are per job and the draw of every step depends only on
// (job seed, walk id, step), so each job's rows are those of a standalone
// n2v_walk call, whatever it is mixed with.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <deque>
#include <map>
#include <mutex>
#include <vector>

#include "n2v_step.cuh"

namespace n2v {

// One job's share of a tick, padded in the slot space to a multiple of 32 so
// that every warp batch belongs to one job.
struct DevSlice {
  const int32_t* starts;
  int32_t* walks;       // the job's [n_starts][l] rows
  int64_t n_starts;
  int64_t walk_begin;   // first walk id of this share
  int64_t count;
  int64_t slot_begin;   // prefix in the tick's slot space (multiple of 32)
  uint64_t seed;
  int32_t l;
  uint32_t a_p, a_q;
  uint32_t pad;
};

// 96 registers a thread: five resident 128-thread blocks per SM (the default
// grid).  KIND: the full or a lean instance (PersistKind).
template <int KIND>
__global__ void __launch_bounds__(kPersistThreads, 5)
    k_serve(GraphView g, const DevSlice* __restrict__ slices, int nslices, int64_t total_slots,
            unsigned long long* __restrict__ counter, LaunchCfg L, uint32_t* __restrict__ spill, uint32_t* status) {
  if (KIND == kPersistLeanUnw) fold_unweighted(g);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  WarpSmem sm = warp_smem(smem_raw, warp, L, spill ? spill + gw * (int64_t)L.spill_specials : nullptr);
  warp_smem_init(sm, lane);
  while (!sm.timed_out) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(counter, 32ull);
    base = __shfl_sync(kFull, base, 0);
    if ((int64_t)base >= total_slots) break;
    // the slice holding this batch: last slot_begin <= base
    int lo = 0, hi = nslices - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (slices[mid].slot_begin <= (int64_t)base) lo = mid;
      else hi = mid - 1;
    }
    const DevSlice S = slices[lo];
    const int64_t i = (int64_t)base - S.slot_begin + lane;
    const bool mine = i < S.count;
    const int64_t wid = S.walk_begin + i;
    int32_t* row = S.walks + wid * (int64_t)S.l;
    int64_t t = -1, v = -1;
    bool alive = false;
    if (mine) {
      const int64_t s0 = S.starts[wid % S.n_starts];
      if (s0 >= 0 && s0 < g.n) {
        v = s0;
        alive = true;
      } else {
        atomicOr(status, kStInvalidArg);
      }
    }
    int k = 0;
    for (; k < S.l; ++k) {
      if (sm.timed_out || !__any_sync(kFull, alive)) break;
      WalkJob J;  // the slice's parameters (serving is exact: no FN-Approx)
      J.seed = S.seed;
      J.a_p = S.a_p;
      J.a_q = S.a_q;
      J.approx = 0;
      const int32_t x = warp_binned_step<KIND == kPersistFull>(g, alive, t, v, k, (uint64_t)wid, J, L.thread_max_deg,
                                                               sm, L.stream_ratio, lane);
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
      for (int kk = k; kk < S.l; ++kk) row[kk] = -1;  // after the walk ended
  }
  if (sm.timed_out && lane == 0) atomicOr(status, kStTimeout);
}

// First-fit allocator over the caller's arena (offsets, 256-byte granules).
class ArenaAlloc {
 public:
  explicit ArenaAlloc(size_t bytes) { free_[0] = bytes; }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + 255) & ~(size_t)255;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        used_ += bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }

 private:
  std::map<size_t, size_t> free_;
  size_t used_ = 0;
};

enum JobState { kQueued = 0, kActive = 1, kDone = 2 };

struct Job {
  int64_t id;
  n2v_job spec;
  std::vector<int32_t> starts_copy;  // host copy until admitted
  uint32_t a_p, a_q;
  size_t off = 0, bytes = 0;
  int64_t launched = 0;  // walks handed to ticks
  int64_t finished = 0;  // walks whose tick completed
  int state = kQueued;
};

struct Tick {
  cudaEvent_t done;
  std::vector<std::pair<int64_t, int64_t>> shares;  // (job id, walks)
  bool busy = false;
};

}  // namespace n2v

struct n2v_server {
  const n2v_graph* g;
  char* arena;
  size_t arena_bytes;
  size_t table_bytes;  // slice tables + counters at the start of the arena
  n2v_serve_cfg cfg;
  cudaStream_t stream;
  n2v::ArenaAlloc* alloc;
  std::mutex mu;
  std::map<int64_t, n2v::Job> jobs;
  std::deque<int64_t> queue;          // admission order
  std::vector<int64_t> active;        // admitted, not finished
  std::vector<int64_t> completed;     // finished, not yet polled
  int64_t next_id = 1;
  n2v::Tick ticks[2];
  int cur = 0;
  std::vector<n2v::DevSlice> host_slices;
  int64_t ticks_launched = 0;
};

using namespace n2v;

static size_t server_table_bytes(const n2v_serve_cfg& c, int blocks_warps) {
  size_t b = 2 * (sizeof(DevSlice) * (size_t)c.max_jobs_per_tick + 256);  // two tick tables
  b += 256;                                                                 // two counters
  b += sizeof(uint32_t) * (size_t)blocks_warps * (size_t)c.spill_specials; // spill area
  return (b + 255) & ~(size_t)255;
}

extern "C" {

void n2v_serve_cfg_default(n2v_serve_cfg* c) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  c->tick_walkers = 1 << 20;
  c->max_jobs_per_tick = 1024;
  c->min_share = 4096;
  c->spill_specials = 1024;
}

int n2v_serve_create(const n2v_graph* g, void* arena, size_t arena_bytes, const n2v_serve_cfg* cfg, void* stream,
                     n2v_server** out) {
  if (!g || !arena || !out || ((uintptr_t)arena & 255)) return N2V_ERR_INVALID_ARG;
  *out = nullptr;
  n2v_serve_cfg c;
  n2v_serve_cfg_default(&c);
  if (cfg) c = *cfg;
  if (c.tick_walkers < 32 || c.max_jobs_per_tick < 1 || c.min_share < 32 || c.spill_specials < 0) return N2V_ERR_INVALID_ARG;
  LaunchCfg L = resolve_launch(g, N2V_PERSISTENT);
  const int warps = L.blocks * (L.block_threads / 32);
  const size_t tb = server_table_bytes(c, warps);
  if (tb + 4096 > arena_bytes) return N2V_ERR_NO_MEM;
  n2v_server* s = new n2v_server();
  s->g = g;
  s->arena = (char*)arena;
  s->arena_bytes = arena_bytes;
  s->table_bytes = tb;
  s->cfg = c;
  s->stream = (cudaStream_t)stream;
  s->alloc = new ArenaAlloc(arena_bytes - tb);
  for (auto& t : s->ticks) {
    if (cudaEventCreateWithFlags(&t.done, cudaEventDisableTiming) != cudaSuccess) {
      delete s->alloc;
      delete s;
      return N2V_ERR_CUDA;
    }
  }
  *out = s;
  return N2V_OK;
}

int n2v_serve_submit(n2v_server* s, const n2v_job* job, int64_t* job_id) {
  if (!s || !job || !job_id || !job->starts || job->n_starts < 1 || job->l < 1) return N2V_ERR_INVALID_ARG;
  Job j;
  if (n2v_alpha_q16(job->p, job->q, &j.a_p, &j.a_q) != N2V_OK) return N2V_ERR_INVALID_ARG;
  const uint64_t amax = std::max<uint64_t>(std::max<uint64_t>(j.a_p, j.a_q), kAlphaOne);
  if (s->g->info.max_wsum > UINT64_MAX / amax) return N2V_ERR_OVERFLOW;
  j.spec = *job;
  j.starts_copy.assign(job->starts, job->starts + job->n_starts);  // the caller's array may go away
  j.bytes = ((sizeof(int32_t) * (size_t)job->n_starts + 255) & ~(size_t)255) +
            sizeof(int32_t) * (size_t)job->n_starts * (size_t)job->l;
  if (j.bytes > s->arena_bytes - s->table_bytes) return N2V_ERR_NO_MEM;  // could never be admitted
  std::lock_guard<std::mutex> lock(s->mu);
  j.id = s->next_id++;
  *job_id = j.id;
  s->queue.push_back(j.id);
  s->jobs.emplace(j.id, std::move(j));
  return N2V_OK;
}

// Admit queued jobs in order while their bytes fit (FIFO: a job that does not
// fit blocks the ones behind it, so large jobs are not starved).
static int admit(n2v_server* s) {
  while (!s->queue.empty()) {
    Job& j = s->jobs.at(s->queue.front());
    size_t off;
    if (!s->alloc->alloc(j.bytes, &off)) break;
    j.off = off;
    j.state = kActive;
    int32_t* dst = (int32_t*)(s->arena + s->table_bytes + off);
    if (cudaMemcpyAsync(dst, j.starts_copy.data(), sizeof(int32_t) * j.starts_copy.size(), cudaMemcpyHostToDevice,
                        s->stream) != cudaSuccess)
      return N2V_ERR_CUDA;
    s->active.push_back(j.id);
    s->queue.pop_front();
  }
  return N2V_OK;
}

static int32_t* job_starts(n2v_server* s, const Job& j) { return (int32_t*)(s->arena + s->table_bytes + j.off); }
static int32_t* job_rows(n2v_server* s, const Job& j) {
  return (int32_t*)(s->arena + s->table_bytes + j.off + ((sizeof(int32_t) * (size_t)j.spec.n_starts + 255) & ~(size_t)255));
}

// Retire the shares of a finished tick.
static void retire(n2v_server* s, Tick& t) {
  for (auto& sh : t.shares) {
    Job& j = s->jobs.at(sh.first);
    j.finished += sh.second;
    if (j.finished == j.spec.n_starts) {
      j.state = kDone;
      s->completed.push_back(j.id);
      s->active.erase(std::find(s->active.begin(), s->active.end(), j.id));
    }
  }
  t.shares.clear();
  t.busy = false;
}

int n2v_serve_step(n2v_server* s, int* launched) {
  if (!s) return N2V_ERR_INVALID_ARG;
  if (launched) *launched = 0;
  std::lock_guard<std::mutex> lock(s->mu);
  // retire finished ticks
  for (auto& t : s->ticks) {
    if (!t.busy) continue;
    const cudaError_t q = cudaEventQuery(t.done);
    if (q == cudaSuccess) retire(s, t);
    else if (q != cudaErrorNotReady) return N2V_ERR_CUDA;
  }
  int rc = admit(s);
  if (rc != N2V_OK) return rc;
  // at most one tick queued behind the running one
  Tick& t = s->ticks[s->cur];
  if (t.busy) return N2V_OK;
  // shares: every active job with walks left gets up to an equal part of the tick
  std::vector<int64_t> todo;
  for (int64_t id : s->active) {
    const Job& j = s->jobs.at(id);
    if (j.launched < j.spec.n_starts) todo.push_back(id);
    if ((int)todo.size() >= s->cfg.max_jobs_per_tick) break;
  }
  if (todo.empty()) return N2V_OK;
  const int64_t fair = std::max<int64_t>(s->cfg.min_share, s->cfg.tick_walkers / (int64_t)todo.size());
  s->host_slices.clear();
  int64_t slots = 0, walkers = 0;
  for (int64_t id : todo) {
    Job& j = s->jobs.at(id);
    const int64_t take = std::min<int64_t>(fair, j.spec.n_starts - j.launched);
    if (take <= 0 || walkers >= s->cfg.tick_walkers) continue;
    DevSlice d;
    memset(&d, 0, sizeof(d));
    d.starts = job_starts(s, j);
    d.walks = job_rows(s, j);
    d.n_starts = j.spec.n_starts;
    d.walk_begin = j.launched;
    d.count = take;
    d.slot_begin = slots;
    d.seed = j.spec.seed;
    d.l = j.spec.l;
    d.a_p = j.a_p;
    d.a_q = j.a_q;
    s->host_slices.push_back(d);
    t.shares.push_back({id, take});
    j.launched += take;
    slots += (take + 31) / 32 * 32;
    walkers += take;
  }
  char* table = s->arena + (size_t)s->cur * (sizeof(DevSlice) * (size_t)s->cfg.max_jobs_per_tick + 256);
  unsigned long long* counter = (unsigned long long*)(s->arena + 2 * (sizeof(DevSlice) * (size_t)s->cfg.max_jobs_per_tick + 256) +
                                                      (size_t)s->cur * 128);
  uint32_t* spill = s->cfg.spill_specials > 0
                        ? (uint32_t*)(s->arena + 2 * (sizeof(DevSlice) * (size_t)s->cfg.max_jobs_per_tick + 256) + 256)
                        : nullptr;
  // the spill area is shared by the two tick slots: ticks run one after the other on one stream
  if (cudaMemcpyAsync(table, s->host_slices.data(), sizeof(DevSlice) * s->host_slices.size(), cudaMemcpyHostToDevice,
                      s->stream) != cudaSuccess ||
      cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s->stream) != cudaSuccess)
    return N2V_ERR_CUDA;
  LaunchCfg L = resolve_launch(s->g, N2V_PERSISTENT);
  L.spill_specials = s->cfg.spill_specials;
  const int smem = (L.block_threads / 32) * warp_smem_bytes(L);
  const int kind = persist_kind(L, s->g->view);
  auto kern = kind == kPersistLeanUnw ? k_serve<kPersistLeanUnw> : kind == kPersistLean ? k_serve<kPersistLean>
                                                                                         : k_serve<kPersistFull>;
  if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  kern<<<L.blocks, L.block_threads, smem, s->stream>>>(s->g->view, (const DevSlice*)table, (int)s->host_slices.size(),
                                                       slots, counter, L, spill, s->g->status);
  if (cudaGetLastError() != cudaSuccess || cudaEventRecord(t.done, s->stream) != cudaSuccess) return N2V_ERR_CUDA;
  t.busy = true;
  s->cur ^= 1;
  s->ticks_launched += 1;
  if (launched) *launched = 1;
  return N2V_OK;
}

int n2v_serve_poll(n2v_server* s, int64_t* ids, int max_ids, int* n) {
  if (!s || !n || (max_ids > 0 && !ids)) return N2V_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  const int k = (int)std::min<size_t>((size_t)std::max(max_ids, 0), s->completed.size());
  for (int i = 0; i < k; ++i) ids[i] = s->completed[i];
  s->completed.erase(s->completed.begin(), s->completed.begin() + k);
  *n = k;
  return N2V_OK;
}

int n2v_serve_job_rows(n2v_server* s, int64_t job_id, int32_t** rows) {
  if (!s || !rows) return N2V_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->jobs.find(job_id);
  if (it == s->jobs.end() || it->second.state != kDone) return N2V_ERR_INVALID_ARG;
  *rows = job_rows(s, it->second);
  return N2V_OK;
}

int n2v_serve_release(n2v_server* s, int64_t job_id) {
  if (!s) return N2V_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->jobs.find(job_id);
  if (it == s->jobs.end() || it->second.state != kDone) return N2V_ERR_INVALID_ARG;
  s->alloc->release(it->second.off, it->second.bytes);
  s->jobs.erase(it);
  return N2V_OK;
}

int n2v_serve_stats(n2v_server* s, n2v_serve_stats_t* st) {
  if (!s || !st) return N2V_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  st->queued = (int64_t)s->queue.size();
  st->active = (int64_t)s->active.size();
  st->arena_used = (int64_t)s->alloc->used();
  st->arena_bytes = (int64_t)(s->arena_bytes - s->table_bytes);
  st->ticks = s->ticks_launched;
  return N2V_OK;
}

void n2v_serve_destroy(n2v_server* s) {
  if (!s) return;
  for (auto& t : s->ticks) cudaEventDestroy(t.done);
  delete s->alloc;
  delete s;
}

}  // extern "C"
