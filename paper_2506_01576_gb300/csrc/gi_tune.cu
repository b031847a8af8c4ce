// Autotuner of the lookup knobs: the parameter sweeps of Sections 7.2-7.4 and
// 8.2-8.4 (thread-block size, lookups per thread, limited concurrency, pinned
// levels, prefetch distance, lane-group size, lookup reordering) run on the
// caller's own index and probes, plus the process-wide table that hands the
// winners to other indexes of the same size class.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "gi_descent.h"
#include "gi_internal.cuh"

namespace {

using gi::tune::Move;
using gi::tune::one;
using gi::tune::two;
using gi::tune::descend;

int tfail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int tfail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  gi::set_last_error(buf);
  return code;
}

int tcuda(cudaError_t e, const char* what) {
  return tfail(e == cudaErrorMemoryAllocation ? GI_ERR_NOMEM : GI_ERR_CUDA, "%s: %s", what,
               cudaGetErrorString(e));
}

// ---------------------------------------------------------------- the table
// (key bytes, layout, k, floor(log2 n)) -> option values (-1: nothing recorded)
using TableKey = std::tuple<int, int, uint32_t, int>;
std::mutex g_mu;
std::map<TableKey, std::array<int64_t, 11>> g_table;
std::atomic<bool> g_table_used{false};
// (key bytes, floor(log2 n)) -> (layout, k) of the fastest layout gi_build_tuned found
std::map<std::pair<int, int>, std::pair<int, uint32_t>> g_layouts;

int size_class(uint64_t n) {
  int c = 0;
  while (n > 1) {
    n >>= 1;
    ++c;
  }
  return c;
}

// The knobs that apply to a layout, each with its candidate moves.
std::vector<std::vector<Move>> index_moves(const gi_info& info, int64_t hot_default) {
  std::vector<std::vector<Move>> g;
  const bool kary = info.layout == GI_EYTZINGER_KARY, ebs = info.layout == GI_EYTZINGER;
  if (kary) {
    std::vector<Move> v;
    for (int64_t x : {1, 2, 4, 8, 16, 32}) v.push_back(one(GI_OPT_GROUP, x));
    g.push_back(v);
  }
  if (info.layout != GI_SORTED) {
    std::vector<Move> v;
    for (int64_t x : {1, 2, 4}) v.push_back(one(GI_OPT_PER_THREAD, x));
    g.push_back(v);
  }
  {
    std::vector<Move> v;
    for (int64_t x : {64, 128, 256, 512}) v.push_back(one(GI_OPT_BLOCK, x));
    g.push_back(v);
  }
  {
    std::vector<Move> v;
    for (int64_t x : {0, 1, 2, 4, 8}) v.push_back(one(GI_OPT_BLOCKS_PER_SM, x));
    g.push_back(v);
  }
  if (info.layout != GI_SORTED) {
    std::vector<Move> v;
    const std::vector<int64_t> lv = ebs ? std::vector<int64_t>{0, 4, 6, 8, 10, 12, 13}
                                        : std::vector<int64_t>{0, 1, 2, 3, 4, 5};
    for (int64_t x : lv) {
      if (x > (int64_t)info.levels) continue;
      v.push_back(one(GI_OPT_SMEM_LEVELS, x));
      if (x > 0)
        for (int64_t b : {1, 2, 4}) v.push_back(two(GI_OPT_SMEM_LEVELS, x, GI_OPT_BLOCKS_PER_SM, b));
    }
    g.push_back(v);
  }
  if (ebs) {
    std::vector<Move> v;
    for (int64_t x : {0, 2, 3, 4}) v.push_back(one(GI_OPT_PREFETCH, x));
    g.push_back(v);
  }
  if (kary) {
    std::vector<Move> v;
    for (int64_t x : {(int64_t)0, hot_default - 2, hot_default - 1, hot_default + 1, hot_default + 2,
                      (int64_t)info.levels})
      if (x >= 0 && x <= (int64_t)info.levels) v.push_back(one(GI_OPT_HOT_LEVELS, x));
    g.push_back(v);
  }
  if (info.unique) {
    std::vector<Move> v;
    for (int64_t x : {0, 1}) v.push_back(one(GI_OPT_EARLY_EXIT, x));
    g.push_back(v);
  }
  {
    std::vector<Move> v;
    for (int64_t x : {0, 1}) v.push_back(one(GI_OPT_REORDER, x));
    g.push_back(v);
  }
  return g;
}

// ---------------------------------------------------------------- timing
// Makes the index's device current for the call (scratch and events live there).
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess || prev == dev) {
      prev = -1;
      return;
    }
    cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

struct Timer {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ~Timer() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};

// One untimed run, then the best of `reps` runs timed on `s`; < 0 if a run failed.
template <class Run>
double best_time(Run run, cudaStream_t s, Timer& t, uint32_t reps, int* rc) {
  *rc = run();
  if (*rc != GI_OK) return -1.0;
  float best = 1e30f;
  for (uint32_t r = 0; r < reps; ++r) {
    cudaEventRecord(t.e0, s);
    *rc = run();
    if (*rc != GI_OK) return -1.0;
    cudaEventRecord(t.e1, s);
    const cudaError_t e = cudaEventSynchronize(t.e1);
    if (e != cudaSuccess) {
      *rc = tcuda(e, "gi_tune: timing");
      return -1.0;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t.e0, t.e1);
    best = std::min(best, ms);
  }
  return best;
}

}  // namespace

namespace gi {

bool tune_table_lookup(int key_bytes, int layout, uint32_t k, uint64_t n, int64_t* opt) {
  if (!g_table_used.load(std::memory_order_acquire)) return false;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_table.find(TableKey{key_bytes, layout, layout == GI_EYTZINGER_KARY ? k : 0u, size_class(n)});
  if (it == g_table.end()) return false;
  for (int o = 0; o < 11; ++o) opt[o] = it->second[o];
  return true;
}

}  // namespace gi

extern "C" {

int gi_tune(gi_index* idx, const void* queries, uint64_t m, uint32_t reps, int flags,
            gi_tune_result* out) {
  gi::set_last_error("");
  if (!idx) return tfail(GI_ERR_INVALID, "gi_tune: NULL index");
  if (m == 0 || !queries) return tfail(GI_ERR_INVALID, "gi_tune: need m >= 1 probes");
  if (flags & ~(GI_TUNE_APPLY | GI_TUNE_RECORD)) return tfail(GI_ERR_INVALID, "gi_tune: unknown flags");
  cudaPointerAttributes pa{};
  if (cudaPointerGetAttributes(&pa, queries) != cudaSuccess || pa.type != cudaMemoryTypeDevice ||
      pa.device != gi::index_device(idx)) {
    cudaGetLastError();
    return tfail(GI_ERR_INVALID, "gi_tune: probes must be device memory of the index's device");
  }
  if (reps == 0) reps = 5;
  gi_info info{};
  int rc = gi_get_info(idx, &info);
  if (rc != GI_OK) return rc;
  const DeviceGuard dg(gi::index_device(idx));
  const cudaStream_t s = gi::index_stream(idx);
  // the settings on entry: raw (to restore) and resolved (the starting point)
  std::array<int64_t, 11> raw{}, cur{};
  raw.fill(-1);
  cur.fill(-1);
  for (int o = 1; o < 11; ++o) {
    raw[o] = gi::index_raw_option(idx, o);
    if (o == GI_OPT_RANGE_FILL) continue;  // not a point-lookup knob
    rc = gi_get_option(idx, o, &cur[o]);
    if (rc != GI_OK) return rc;
  }
  const std::array<int64_t, 11> start_pt = cur;
  auto restore = [&] {
    for (int o = 1; o < 11; ++o) gi_set_option(idx, o, raw[o]);
  };
  uint32_t* dout = nullptr;
  cudaError_t e = cudaMalloc((void**)&dout, m * sizeof(uint32_t));
  if (e != cudaSuccess) return tcuda(e, "gi_tune: scratch");
  Timer t;
  e = cudaEventCreate(&t.e0);
  if (e == cudaSuccess) e = cudaEventCreate(&t.e1);
  if (e != cudaSuccess) {
    cudaFree(dout);
    return tcuda(e, "gi_tune: events");
  }
  auto run = [&] { return gi_point_lookup(idx, queries, m, dout); };
  auto time = [&](int* r) { return best_time(run, s, t, reps, r); };
  auto set = [&](int o, int64_t v) { return gi_set_option(idx, o, v); };
  for (int o = 1; o < 11; ++o)
    if (cur[o] >= 0) set(o, cur[o]);
  const double start = time(&rc);
  double best = start;
  uint32_t trials = 1, passes = 0;
  if (rc == GI_OK)
    rc = descend(index_moves(info, cur[GI_OPT_HOT_LEVELS]), cur, set, time, start, &best, &trials,
                 &passes);
  if (rc == GI_OK) rc = gi_sync(idx);
  cudaFree(dout);
  if (rc != GI_OK) {
    restore();
    return rc;
  }
  if (flags & GI_TUNE_RECORD) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_table[TableKey{(int)info.key_bytes, info.layout,
                     info.layout == GI_EYTZINGER_KARY ? info.k : 0u, size_class(info.n)}] = cur;
    g_table_used.store(true, std::memory_order_release);
  }
  if (flags & GI_TUNE_APPLY) {
    for (int o = 1; o < 11; ++o)
      if (o != GI_OPT_RANGE_FILL) set(o, cur[o]);
  } else {
    restore();
  }
  if (out) {
    for (int o = 0; o < 11; ++o) out->options[o] = o == GI_OPT_RANGE_FILL ? -1 : cur[o];
    out->options[0] = -1;
    out->start_ms = start;
    out->best_ms = best;
    out->trials = trials;
    out->passes = passes;
    for (int o = 0; o < 11; ++o) out->start_options[o] = o == 0 ? -1 : start_pt[o];
  }
  return GI_OK;
}

int gi_tune_table_get(int layout, uint32_t k, uint64_t n, int64_t* options, int* found) {
  gi::set_last_error("");
  if (!options || !found) return tfail(GI_ERR_INVALID, "gi_tune_table_get: NULL argument");
  const int kb = (layout & 0xF00) == GI_KEY_U64 ? 8 : 4;
  for (int o = 0; o < 11; ++o) options[o] = -1;
  *found = gi::tune_table_lookup(kb, layout & 0xFF, k, n, options) ? 1 : 0;
  return GI_OK;
}

void gi_tune_table_clear(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_table.clear();
  g_layouts.clear();
  g_table_used.store(false, std::memory_order_release);
}

int gi_build_tuned(const void* keys, const uint32_t* rowids, uint64_t n, int key_flags,
                   const void* queries, uint64_t m, uint32_t reps, int flags, gi_index** out,
                   gi_tune_result* result) {
  gi::set_last_error("");
  if (!out) return tfail(GI_ERR_INVALID, "gi_build_tuned: out is NULL");
  *out = nullptr;
  if (key_flags & 0xFF) return tfail(GI_ERR_INVALID, "gi_build_tuned: pass the key width and build flags only");
  if (flags & ~(GI_TUNE_APPLY | GI_TUNE_RECORD)) return tfail(GI_ERR_INVALID, "gi_build_tuned: unknown flags");
  // the layouts of Sections 3 and 6 with compiled lane-group kernels: sorted, EBS,
  // k-ary with k - 1 a power of two
  static const int kLayouts[][2] = {{GI_SORTED, 0}, {GI_EYTZINGER, 2}, {GI_EYTZINGER_KARY, 3},
                                    {GI_EYTZINGER_KARY, 5}, {GI_EYTZINGER_KARY, 9},
                                    {GI_EYTZINGER_KARY, 17}};
  gi_index* best = nullptr;
  gi_tune_result best_r{};
  for (const auto& c : kLayouts) {
    gi_index* idx = nullptr;
    int rc = gi_build(keys, rowids, n, key_flags | c[0], (uint32_t)c[1], &idx);
    if (rc == GI_OK) {
      gi_tune_result r{};
      rc = gi_tune(idx, queries, m, reps, GI_TUNE_APPLY, &r);
      if (rc == GI_OK && (!best || r.best_ms < best_r.best_ms)) {
        gi_destroy(best);
        best = idx;
        best_r = r;
        idx = nullptr;
      }
    }
    gi_destroy(idx);
    if (rc != GI_OK) {
      gi_destroy(best);
      return rc;
    }
  }
  gi_info info{};
  gi_get_info(best, &info);
  if (flags & GI_TUNE_RECORD) {
    std::lock_guard<std::mutex> lk(g_mu);
    const int kb = (int)info.key_bytes, cls = size_class(n);
    g_table[TableKey{kb, info.layout, info.layout == GI_EYTZINGER_KARY ? info.k : 0u, cls}] = [&] {
      std::array<int64_t, 11> a{};
      for (int o = 0; o < 11; ++o) a[o] = o == GI_OPT_RANGE_FILL ? -1 : best_r.options[o];
      a[0] = -1;
      return a;
    }();
    g_layouts[{kb, cls}] = {info.layout, info.layout == GI_EYTZINGER_KARY ? info.k : 0u};
    g_table_used.store(true, std::memory_order_release);
  }
  if (!(flags & GI_TUNE_APPLY))
    for (int o = 1; o < 11; ++o) gi_set_option(best, o, -1);
  if (result) *result = best_r;
  *out = best;
  return GI_OK;
}

int gi_tune_table_layout(int key_flags, uint64_t n, int* layout, uint32_t* k, int* found) {
  gi::set_last_error("");
  if (!layout || !k || !found) return tfail(GI_ERR_INVALID, "gi_tune_table_layout: NULL argument");
  const int kb = (key_flags & 0xFF00) == GI_KEY_U64 ? 8 : 4;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_layouts.find({kb, size_class(n)});
  *found = it != g_layouts.end();
  *layout = *found ? it->second.first : -1;
  *k = *found ? it->second.second : 0u;
  return GI_OK;
}

int gi_batch_tune(gi_batch* b, const void* queries, const uint64_t* query_offsets, uint64_t m,
                  uint32_t reps, gi_tune_result* out) {
  gi::set_last_error("");
  if (!b) return tfail(GI_ERR_INVALID, "gi_batch_tune: NULL batch");
  if (reps == 0) reps = 5;
  const DeviceGuard dg(gi::batch_device(b));
  const cudaStream_t s = gi::batch_stream(b);
  std::array<int64_t, 11> cur{};
  cur.fill(-1);
  for (int o = GI_BATCH_OPT_CHUNK; o <= GI_BATCH_OPT_SMEM_BUDGET; ++o) cur[o] = gi::batch_option(b, o);
  const std::array<int64_t, 11> start_pt = cur;
  uint32_t* dout = nullptr;
  cudaError_t e = cudaMalloc((void**)&dout, (m ? m : 1) * sizeof(uint32_t));
  if (e != cudaSuccess) return tcuda(e, "gi_batch_tune: scratch");
  Timer t;
  e = cudaEventCreate(&t.e0);
  if (e == cudaSuccess) e = cudaEventCreate(&t.e1);
  if (e != cudaSuccess) {
    cudaFree(dout);
    return tcuda(e, "gi_batch_tune: events");
  }
  std::vector<std::vector<Move>> groups(3);
  for (int64_t x : {256, 512, 1024, 2048, 4096, 8192}) groups[0].push_back(one(GI_BATCH_OPT_CHUNK, x));
  for (int64_t x : {1, 2, 4, 8}) groups[1].push_back(one(GI_BATCH_OPT_BLOCKS_PER_SM, x));
  for (int64_t x : {0, 4096, 8192, 16384, 24576, 32768, 40960})
    groups[2].push_back(one(GI_BATCH_OPT_SMEM_BUDGET, x));
  auto run = [&] { return gi_batch_point_lookup(b, queries, query_offsets, m, dout); };
  auto time = [&](int* r) { return best_time(run, s, t, reps, r); };
  auto set = [&](int o, int64_t v) { return gi_batch_set_option(b, o, v); };
  int rc = GI_OK;
  const double start = time(&rc);
  double best = start;
  uint32_t trials = 1, passes = 0;
  if (rc == GI_OK) rc = descend(groups, cur, set, time, start, &best, &trials, &passes);
  if (rc == GI_OK) rc = gi_batch_sync(b);
  cudaFree(dout);
  if (rc != GI_OK) {
    for (int o = GI_BATCH_OPT_CHUNK; o <= GI_BATCH_OPT_SMEM_BUDGET; ++o) set(o, start_pt[o]);
    return rc;
  }
  if (out) {
    for (int o = 0; o < 11; ++o) {
      out->options[o] = cur[o];
      out->start_options[o] = start_pt[o];
    }
    out->options[0] = out->start_options[0] = -1;
    out->start_ms = start;
    out->best_ms = best;
    out->trials = trials;
    out->passes = passes;
  }
  return GI_OK;
}

}  // extern "C"
