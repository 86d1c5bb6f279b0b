// Autotuner of the persistent sampler: a coordinate descent over its
// tunables, each candidate timed with CUDA events on a sample of the job.
// The hub caches (hashed sets and rank bitmaps, the FN-Cache analogue of
// Section 3.4) are axes too, from none up to the sizes the graph was loaded
// with.
// Every tuning gives the same rows (the step is exact on every code path), so
// only speed is compared.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "n2v_internal.cuh"

namespace n2v {

struct Axis {
  int32_t n2v_tune::*field;
  std::vector<int32_t> values;
};

// resident warps per SM tried by the descent (blocks_per_sm follows from block_threads)
static const int kWarpTargets[] = {20, 16, 24};
// a candidate replaces the current tuning only when it is this much faster
// (run-to-run spread on one sample is about 1%)
static const float kMinGain = 0.02f;

static size_t ws_for(const n2v_graph* g, int64_t sample, int32_t l, int warps_per_sm, int spill) {
  const int64_t chunks = g->tune.chunk_walkers > 0 ? (sample + g->tune.chunk_walkers - 1) / g->tune.chunk_walkers : 1;
  size_t b = ((sizeof(unsigned long long) * (size_t)chunks) + 255) & ~(size_t)255;
  b += sizeof(uint32_t) * (size_t)g->sms * (size_t)warps_per_sm * (size_t)spill;
  (void)l;
  return b;
}

}  // namespace n2v

using namespace n2v;

extern "C" {

int n2v_autotune_ws_bytes(const n2v_graph* g, int64_t sample, int32_t l, size_t* bytes) {
  if (!g || !bytes || sample < 1 || l < 1) return N2V_ERR_INVALID_ARG;
  // the largest candidate grid: 24 resident warps per SM (or the caller's larger
  // choice, rounded up to whole 4-warp blocks of the persistent kernel)
  const int bw = g->tune.block_threads / 32;
  *bytes = ws_for(g, sample, l, std::max(24, (g->tune.blocks_per_sm * bw + 3) & ~3), g->tune.spill_specials);
  return N2V_OK;
}

int n2v_autotune(n2v_graph* g, const int32_t* starts, int64_t n_starts, int32_t l, double p, double q, uint64_t seed,
                 int64_t sample, int32_t* walks, void* ws, size_t ws_bytes, void* stream, n2v_tune* best,
                 float* best_ms) {
  if (!g || !starts || n_starts < 1 || l < 1 || sample < 1 || sample > n_starts || !walks || !ws) return N2V_ERR_INVALID_ARG;
  size_t need = 0;
  int rc = n2v_autotune_ws_bytes(g, sample, l, &need);
  if (rc != N2V_OK) return rc;
  if (ws_bytes < need) return N2V_ERR_NO_MEM;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return N2V_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return N2V_ERR_CUDA;
  }
  const n2v_tune start = g->tune;
  // the faster of two timed runs of the sample (after one untimed run) under tuning t
  auto measure = [&](const n2v_tune& t, float* ms) -> int {
    int r0 = n2v_graph_retune(g, &t, stream);
    if (r0 != N2V_OK) return r0;
    r0 = n2v_walk(g, starts, n_starts, 1, l, p, q, seed, 0, sample, walks, ws, ws_bytes, N2V_PERSISTENT, stream);
    if (r0 != N2V_OK) return r0;
    *ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {
      if (cudaEventRecord(e0, s) != cudaSuccess) return N2V_ERR_CUDA;
      r0 = n2v_walk(g, starts, n_starts, 1, l, p, q, seed, 0, sample, walks, ws, ws_bytes, N2V_PERSISTENT, stream);
      if (r0 != N2V_OK) return r0;
      float t_ms = 0.f;
      if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return N2V_ERR_CUDA;
      if (cudaEventElapsedTime(&t_ms, e0, e1) != cudaSuccess) return N2V_ERR_CUDA;
      *ms = rep == 0 ? t_ms : std::min(*ms, t_ms);
    }
    return n2v_stream_status(g, stream);
  };

  std::vector<Axis> axes;
  // the hub caches first (they change which generator most hub steps take), then the rest
  const n2v_tune& ld = g->tune_loaded;
  std::vector<Axis> cache_axes;
  if (ld.hub_count > 0) {
    Axis hb{&n2v_tune::hub_count, {ld.hub_count, 0}};
    if (ld.hub_count >= 64) hb.values.push_back(ld.hub_count / 8);
    cache_axes.push_back(hb);
  }
  if (ld.bitmap_hubs > 0) {
    Axis bm{&n2v_tune::bitmap_hubs, {ld.bitmap_hubs, 0}};
    if (ld.bitmap_hubs >= 8) bm.values.push_back(ld.bitmap_hubs / 4);
    cache_axes.push_back(bm);
  }
  for (const Axis& ax : cache_axes) axes.push_back(ax);
  axes.push_back({&n2v_tune::stage_window, {512, 1024, 256}});
  const size_t blocks_axis = axes.size();
  {
    const int bw = start.block_threads / 32;
    Axis blocks{&n2v_tune::blocks_per_sm, {}};
    for (int w : kWarpTargets)
      if (w % bw == 0) blocks.values.push_back(w / bw);
    if (blocks.values.empty()) blocks.values.push_back(std::max(1, 16 / bw));
    axes.push_back(blocks);
  }
  axes.push_back({&n2v_tune::stream_ratio, {15, 40, 100}});
  axes.push_back({&n2v_tune::merge_ratio, {0, 3, 10}});
  // (l2_persist_mb is not an axis: persisting windows of 32-96 MB over col measured within 0.3%)
  axes.push_back({&n2v_tune::thread_max_deg, {0, 16, 48}});
  axes.push_back({&n2v_tune::stage_buffers, {2, 4}});
  axes.push_back({&n2v_tune::smem_specials, {256, 128, 512}});
  // block batches with a block tier for the steps whose longer list is at least this long (0: off)
  axes.push_back({&n2v_tune::block_min_deg, {0, 1024, 16384}});
  // and the caches once more, now that the rest has moved (up to the sizes the graph was loaded with)
  for (const Axis& ax : cache_axes) axes.push_back(ax);

  n2v_tune cur = start;
  if (cur.blocks_per_sm <= 0) cur.blocks_per_sm = axes[blocks_axis].values[0];
  float cur_ms = 0.f;
  rc = measure(cur, &cur_ms);
  for (size_t a = 0; a < axes.size() && rc == N2V_OK; ++a) {
    for (int32_t val : axes[a].values) {
      if (cur.*(axes[a].field) == val) continue;
      n2v_tune cand = cur;
      cand.*(axes[a].field) = val;
      // four windows of 1024 per warp do not fit beside 20 or more resident warps: skip that corner
      if (cand.stage_buffers * (cand.stage_window + 8) * 4 * (cand.block_threads / 32) * cand.blocks_per_sm > 200 * 1024)
        continue;
      float ms = 0.f;
      rc = measure(cand, &ms);
      if (rc != N2V_OK) break;
      if (ms < cur_ms * (1.f - kMinGain)) {
        cur = cand;
        cur_ms = ms;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != N2V_OK) {
    n2v_graph_retune(g, &start, stream);
    return rc;
  }
  rc = n2v_graph_retune(g, &cur, stream);
  if (best) *best = cur;
  if (best_ms) *best_ms = cur_ms;
  return rc;
}

}  // extern "C"
