// Serving form: a resident set of indexes answers a stream of point and range
// requests with continuous batching.
//
// Client threads submit requests (host buffers) at any time.  One server thread
// owns the device side:
//   admission   requests are admitted first-in first-out while a fixed device
//               arena has room for their inputs and results (the admission
//               budget); a request that can never fit is rejected at once.
//   batching    every admitted request, of any index and kind, joins the next
//               batch; one batch is a handful of launches shared by all of its
//               requests (lookups and range counts in one kernel, a per-request
//               scan, a range fill), with the copies in and out on the batch's
//               own stream.  Inputs and point results of large requests in
//               page-locked host memory are copied by the copy engine, one copy
//               per buffer, with no host work; small requests, and those in
//               pageable memory (whose copies the driver would stage
//               synchronously), are gathered on the host into one staging copy
//               per batch, and their point results come back in one copy that the
//               host scatters.  Range offsets and rows come back with one copy per
//               request.
//   overlap     up to `max_inflight` batches are on the GPU at once, each on its
//               own stream, so requests that arrive while others run are admitted
//               into the next batch as soon as arena space frees up.
//   ranges      take two passes: the count pass returns the offsets and the total;
//               the fill is admitted once arena room for the rows is free.
// Each request's submit and completion times are recorded for latency figures.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gi_internal.cuh"
#include "gi_point_impl.cuh"

namespace gi {
namespace sv {

struct ServeIndex {  // device descriptor of a resident index
  const void* keys;
  const uint32_t* rows;
  uint64_t n;
  uint32_t levels;
  uint32_t pad;
};

enum : uint32_t { kItemPoint = 0, kItemCount = 1, kItemFill = 2 };

struct ServeItem {  // one request's share of a batch (device copy of the table)
  const void* in;      // probes or lower bounds (the batch's staging or the arena)
  const void* in2;     // upper bounds
  void* out;           // point: results; count/fill: offsets (m+1)
  uint64_t* aux;       // count/fill: lower ranks
  uint32_t* rows;      // fill: rows
  uint64_t m;
  uint64_t work_start;  // first work item of this request in the batch
  uint32_t index;
  uint32_t kind;
};

constexpr uint32_t kChunk = 1024;  // probes or ranges per work item

__device__ __forceinline__ uint32_t find_item(const ServeItem* items, uint32_t count, uint64_t w) {
  uint32_t lo = 0, hi = count;  // items[lo].work_start <= w < items[hi].work_start
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (items[mid].work_start <= w) lo = mid; else hi = mid;
  }
  return lo;
}

// lower-bound slot (or ~0) of x in a k-ary index, one thread
template <class K, int KF>
__device__ __forceinline__ uint64_t eks_bound(const K* __restrict__ keys, uint64_t n, uint32_t levels,
                                              K x, bool upper) {
  constexpr int N = KF - 1;
  uint64_t s = 0, cand = ~0ull;
  for (uint32_t lv = 0; lv < levels; ++lv) {
    if (s >= n) break;
    K piv[N];
    if constexpr (pt::EksShape<K, KF, 1>::VEC) {
      pt::vec_load<K, N>(keys + s, piv);
    } else {
#pragma unroll
      for (int p = 0; p < N; ++p) piv[p] = __ldg(keys + s + p);
    }
    uint32_t c = 0;
#pragma unroll
    for (int p = 0; p < N; ++p) c += (upper ? piv[p] <= x : piv[p] < x) ? 1u : 0u;
    if (c < (uint32_t)N && s + c < n) cand = s + c;
    s = s * KF + (uint64_t)(c + 1) * N;
  }
  return cand;
}

template <class K>
__device__ __forceinline__ uint64_t sorted_bound(const K* __restrict__ keys, uint64_t n, K x, bool upper) {
  uint64_t lo = 0, len = n;
  while (len > 0) {
    const uint64_t half = len >> 1;
    const K v = __ldg(keys + lo + half);
    if (upper ? v <= x : v < x) {
      lo += half + 1;
      len -= half + 1;
    } else {
      len = half;
    }
  }
  return lo;
}

// KF == 0: sorted layout.  Point lookups and range counts of a whole batch.
template <class K, int KF>
__global__ void __launch_bounds__(256) k_serve_lookup(const ServeIndex* __restrict__ idx,
                                                      const ServeItem* __restrict__ items,
                                                      uint32_t nitems, uint64_t nwork,
                                                      unsigned char* __restrict__ arena) {
  __shared__ uint32_t s_item;
  for (uint64_t w = blockIdx.x; w < nwork; w += gridDim.x) {
    if (threadIdx.x == 0) s_item = find_item(items, nitems, w);
    __syncthreads();
    const ServeItem it = items[s_item];
    __syncthreads();
    if (it.kind == kItemFill) continue;
    const ServeIndex d = idx[it.index];
    const K* keys = (const K*)d.keys;
    const uint64_t i0 = (w - it.work_start) * kChunk;
    const uint64_t i1 = min(i0 + kChunk, it.m);
    const K* q = (const K*)it.in;
    if (it.kind == kItemPoint) {
      uint32_t* out = (uint32_t*)it.out;
      for (uint64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const K x = q[i];
        uint32_t res = GI_MISS;
        if constexpr (KF > 0) {
          const uint64_t c = eks_bound<K, KF>(keys, d.n, d.levels, x, false);
          if (c != ~0ull && __ldg(keys + c) == x) res = __ldg(d.rows + c);
        } else {
          const uint64_t c = sorted_bound<K>(keys, d.n, x, false);
          if (c < d.n && __ldg(keys + c) == x) res = __ldg(d.rows + c);
        }
        out[i] = res;
      }
    } else {  // range count: lower rank of L, upper rank of U
      const K* hi = (const K*)it.in2;
      uint64_t* cnt = (uint64_t*)it.out;
      uint64_t* lo_rank = it.aux;
      const Geom g = device_geom(d.n, KF > 1 ? (uint32_t)KF : 2u);
      for (uint64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const K L = q[i], U = hi[i];
        uint64_t rl = 0, ru = 0;
        if (L <= U) {
          if constexpr (KF > 0) {
            const uint64_t a = eks_bound<K, KF>(keys, d.n, d.levels, L, false);
            const uint64_t b = eks_bound<K, KF>(keys, d.n, d.levels, U, true);
            rl = a != ~0ull ? slot_to_rank<KF>(a, g) : d.n;
            ru = b != ~0ull ? slot_to_rank<KF>(b, g) : d.n;
          } else {
            rl = sorted_bound<K>(keys, d.n, L, false);
            ru = sorted_bound<K>(keys, d.n, U, true);
          }
        }
        cnt[i] = ru - rl;
        lo_rank[i] = rl;
      }
    }
  }
}

// exclusive scan of one count item's counts, in place, total at [m]; one CTA per item
__global__ void __launch_bounds__(1024) k_serve_scan(const ServeItem* __restrict__ items,
                                                     const uint32_t* __restrict__ count_items,
                                                     unsigned char* __restrict__ arena) {
  __shared__ uint64_t s_warp[32];
  const ServeItem it = items[count_items[blockIdx.x]];
  uint64_t* a = (uint64_t*)it.out;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  uint64_t carry = 0;
  for (uint64_t base = 0; base < it.m; base += blockDim.x) {
    const uint64_t j = base + threadIdx.x;
    const uint64_t v = j < it.m ? a[j] : 0;
    uint64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[wp] = x;
    __syncthreads();
    uint64_t pre = 0, tot = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      if (i < wp) pre += s_warp[i];
      tot += s_warp[i];
    }
    if (j < it.m) a[j] = carry + pre + x - v;
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) a[it.m] = carry;
}

// range fill: rows of rank r come from slot(r); a warp per 32 ranges, ranges of
// >= 32 rows done by the whole warp
template <int KF>
__global__ void __launch_bounds__(256) k_serve_fill(const ServeIndex* __restrict__ idx,
                                                    const ServeItem* __restrict__ items,
                                                    uint32_t nitems, uint64_t nwork,
                                                    unsigned char* __restrict__ arena) {
  __shared__ uint32_t s_item;
  __shared__ SlotMap sm;  // the item's 32-bit rank -> slot map
  const int lane = threadIdx.x & 31;
  for (uint64_t w = blockIdx.x; w < nwork; w += gridDim.x) {
    if (threadIdx.x == 0) s_item = find_item(items, nitems, w);
    __syncthreads();
    const ServeItem it = items[s_item];
    const ServeIndex d = idx[it.index];
    const Geom g = device_geom(d.n, KF > 1 ? (uint32_t)KF : 2u);
    const bool narrow = d.n < (1ull << 32);
    if (threadIdx.x == 0 && it.kind == kItemFill && KF > 0 && narrow) fill_slot_map(sm, g);
    __syncthreads();
    if (it.kind != kItemFill) continue;
    const uint64_t* offs = (const uint64_t*)it.out;
    const uint64_t* lo_rank = it.aux;
    uint32_t* out = it.rows;
    const uint64_t i0 = (w - it.work_start) * kChunk;
    const uint64_t i1 = min(i0 + kChunk, it.m);
    for (uint64_t wb = i0 + (threadIdx.x >> 5) * 32; wb < i1; wb += (blockDim.x >> 5) * 32) {
      const uint64_t i = wb + lane;
      uint64_t off = 0, cnt = 0, r0 = 0;
      if (i < i1) {
        off = offs[i];
        cnt = offs[i + 1] - off;
        r0 = lo_rank[i];
      }
      auto slot = [&](uint64_t r) -> uint64_t {
        if constexpr (KF > 0) return narrow ? slot_of_rank<KF>((uint32_t)r, sm) : rank_to_slot<KF>(r, g);
        else return r;
      };
      const bool big = cnt >= 32;
      uint32_t bm = __ballot_sync(0xffffffffu, big);
      while (bm) {
        const int b = __ffs(bm) - 1;
        bm &= bm - 1;
        const uint64_t bo = __shfl_sync(0xffffffffu, off, b);
        const uint64_t bc = __shfl_sync(0xffffffffu, cnt, b);
        const uint64_t br = __shfl_sync(0xffffffffu, r0, b);
        for (uint64_t j = lane; j < bc; j += 32) out[bo + j] = __ldg(d.rows + slot(br + j));
      }
      // short ranges: their rows dealt to the lanes (coalesced, 32 loads in flight);
      // a 5-step search over the lanes' running counts finds each row's range
      uint32_t c = big ? 0u : (uint32_t)cnt, x = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      const uint32_t rel = x - c;
      const uint32_t total = __shfl_sync(0xffffffffu, x, 31);
      for (uint32_t row0 = 0; row0 < total; row0 += 32) {  // warp-uniform for the shuffles
        const uint32_t row = row0 + lane;
        int src = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const uint32_t v = __shfl_sync(0xffffffffu, rel, src + step);
          if (v <= row) src += step;
        }
        const uint32_t k = row - __shfl_sync(0xffffffffu, rel, src);
        const uint64_t o = __shfl_sync(0xffffffffu, off, src) + k;
        const uint64_t r = __shfl_sync(0xffffffffu, r0, src) + k;
        if (row < total) out[o] = __ldg(d.rows + slot(r));
      }
    }
  }
}

}  // namespace sv
}  // namespace gi

// ================================================================= host side
namespace {

using Clock = std::chrono::steady_clock;

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now().time_since_epoch()).count();
}

// First-fit allocator over the arena (byte offsets), 256-byte granules.
class Arena {
 public:
  void init(uint64_t bytes) {
    total_ = bytes;
    free_.clear();
    free_[0] = bytes;
  }
  bool alloc(uint64_t bytes, uint64_t* off) {
    bytes = (bytes + 255) & ~255ull;
    if (bytes == 0) bytes = 256;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const uint64_t rest = it->second - bytes, at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        used_ += bytes;
        return true;
      }
    }
    return false;
  }
  void release(uint64_t off, uint64_t bytes) {
    bytes = (bytes + 255) & ~255ull;
    if (bytes == 0) bytes = 256;
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
  uint64_t total() const { return total_; }
  uint64_t used() const { return used_; }

 private:
  uint64_t total_ = 0, used_ = 0;
  std::map<uint64_t, uint64_t> free_;
};

struct Block {
  uint64_t off = 0, bytes = 0;
  bool live = false;
};

struct Req {
  gi_request r;
  uint64_t ticket = 0;
  int phase = 0;  // 0 queued, 1 point/count in flight, 2 counted, 3 fill in flight, 4 done
  int status = GI_OK;
  Block in, in2, out, aux, rows;
  // pinned: the inputs (all of them) / a point request's results are in
  // page-locked host memory, copied by the copy engine straight from / to them
  bool pinned_in = false, pinned_out = false;
  // staged: the inputs (and a point request's results) that are not pinned go
  // through the batch's staging buffers at these byte offsets, with one copy each
  // way per batch
  bool staged = false;
  uint64_t st_in = 0, st_out = 0;
  uint64_t total = 0;
  int64_t t_submit = 0, t_done = 0;
};

struct Batch {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  gi::sv::ServeItem* h_items = nullptr;  // pinned
  gi::sv::ServeItem* d_items = nullptr;
  uint32_t* h_count_items = nullptr;     // pinned
  uint32_t* d_count_items = nullptr;
  uint32_t capacity = 0;
  // staging: the requests' inputs gathered on the host into h_in (pinned) and
  // copied in once; point results copied out once into h_out and scattered on
  // the host (a copy call per request cost the server thread more than the GPU
  // spent on the lookups)
  unsigned char* h_in = nullptr;
  unsigned char* d_in = nullptr;
  unsigned char* h_out = nullptr;
  unsigned char* d_out = nullptr;
  uint64_t in_cap = 0, out_cap = 0, in_used = 0, out_used = 0;
  std::vector<std::shared_ptr<Req>> reqs;
  bool busy = false;
};

}  // namespace

struct gi_server {
  int device = 0;
  int key_bytes = 8;
  int layout = GI_EYTZINGER_KARY;
  uint32_t k = 0;
  uint32_t nidx = 0;
  gi::sv::ServeIndex* d_idx = nullptr;
  std::vector<gi::sv::ServeIndex> h_idx;
  unsigned char* arena = nullptr;
  Arena alloc;
  uint64_t max_batch = 1ull << 22;
  std::vector<Batch> batches;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_submit, cv_done;
  std::deque<std::shared_ptr<Req>> incoming;
  std::unordered_map<uint64_t, std::shared_ptr<Req>> by_ticket;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::atomic<uint64_t> n_batches{0}, n_requests{0}, n_probes{0};
  int fatal = GI_OK;
};

namespace {

int sfail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  gi::set_last_error(buf);
  return code;
}

uint64_t in_bytes(const gi_request& r, int kb) { return r.m * kb; }

// Whether a caller's host buffer is page-locked, cached per 64 KiB region of
// the address space so that a request costs no driver query once its regions
// have been seen (a query per buffer on the submitting threads measured 30% less
// server capacity: 171k against 245k requests/s).  A stale entry -- memory freed
// and allocated again as the other kind -- only picks the slower of two correct
// copy paths: every copy call takes any host memory.
constexpr int kPinCacheBits = 14;
constexpr uint64_t kStageAlways = 2048;  // probes or ranges: staged whatever the memory
std::atomic<uint64_t> g_pin_cache[1u << kPinCacheBits];  // (region << 2) | 1 pinned / 2 pageable

bool region_pinned(int device, uintptr_t addr) {
  const uint64_t region = (uint64_t)addr >> 16;
  const uint64_t slot = (region * 0x9E3779B97F4A7C15ull) >> (64 - kPinCacheBits);
  const uint64_t v = g_pin_cache[slot].load(std::memory_order_relaxed);
  if ((v & 3) && (v >> 2) == region) return (v & 3) == 1;
  int old = -1;
  cudaGetDevice(&old);
  if (old != device) cudaSetDevice(device);
  cudaPointerAttributes at{};
  bool pinned = false;
  if (cudaPointerGetAttributes(&at, (const void*)addr) == cudaSuccess)
    pinned = at.type == cudaMemoryTypeHost;
  else
    cudaGetLastError();
  if (old >= 0 && old != device) cudaSetDevice(old);
  g_pin_cache[slot].store((region << 2) | (pinned ? 1u : 2u), std::memory_order_relaxed);
  return pinned;
}

bool host_pinned(int device, const void* p, uint64_t bytes) {
  const uintptr_t a = (uintptr_t)p;
  return region_pinned(device, a) && region_pinned(device, a + (bytes - 1));
}

void free_block(gi_server* s, Block& b) {
  if (b.live) s->alloc.release(b.off, b.bytes);
  b.live = false;
}

bool take_block(gi_server* s, Block& b, uint64_t bytes) {
  if (!s->alloc.alloc(bytes, &b.off)) return false;
  b.bytes = bytes;
  b.live = true;
  return true;
}

// reserve arena room for a request's next phase; false if it does not fit now.
// in_free: its inputs need no arena room (staged); out_free: the same for a
// point request's results.
bool admit(gi_server* s, Req& q, bool in_free, bool out_free) {
  const int kb = s->key_bytes;
  const uint64_t m = q.r.m;
  if (q.phase == 0 && q.r.kind == GI_REQ_POINT) {
    if (!in_free && !take_block(s, q.in, m * kb)) return false;
    if (!out_free && !take_block(s, q.out, m * 4)) {
      free_block(s, q.in);
      return false;
    }
    return true;
  }
  if (q.phase == 0) {  // range count
    if (!in_free) {
      if (!take_block(s, q.in, m * kb)) return false;
      if (!take_block(s, q.in2, m * kb)) {
        free_block(s, q.in);
        return false;
      }
    }
    if (!take_block(s, q.out, (m + 1) * 8)) {
      free_block(s, q.in);
      free_block(s, q.in2);
      return false;
    }
    if (!take_block(s, q.aux, m * 8)) {
      free_block(s, q.in);
      free_block(s, q.in2);
      free_block(s, q.out);
      return false;
    }
    return true;
  }
  // fill: rows of the counted ranges
  return take_block(s, q.rows, std::max<uint64_t>(q.total, 1) * 4);
}

// staging bytes of a request's inputs / results (none where pinned; no results
// for ranges)
uint64_t stage_in_bytes(const Req& q, int kb) {
  return q.pinned_in ? 0 : q.r.m * kb * (q.r.kind == GI_REQ_RANGE ? 2u : 1u);
}
uint64_t stage_out_bytes(const Req& q) {
  return q.r.kind == GI_REQ_POINT && !q.pinned_out ? q.r.m * 4 : 0;
}
uint64_t up16(uint64_t x) { return (x + 15) & ~15ull; }

// bytes a request needs at its largest phase (for the can-never-fit check)
uint64_t peak_bytes(const gi_request& r, int kb) {
  auto g = [](uint64_t b) { return (std::max<uint64_t>(b, 1) + 255) & ~255ull; };
  if (r.kind == GI_REQ_POINT) return g(r.m * kb) + g(r.m * 4);
  return g(r.m * kb) * 2 + g((r.m + 1) * 8) + g(r.m * 8);
}

void launch_batch(gi_server* s, Batch& b) {
  using namespace gi::sv;
  const int kb = s->key_bytes;
  cudaStream_t st = b.stream;
  uint32_t n = 0, ncount = 0;
  uint64_t work = 0, fill_work = 0;
  // lookups and counts first, then fills (two work ranges in one table)
  unsigned char* const arena = s->arena;
  for (auto& q : b.reqs) {
    if (q->phase == 3) continue;
    ServeItem& it = b.h_items[n++];
    it.index = q->r.index;
    it.m = q->r.m;
    const uint64_t mb = q->r.m * kb;
    if (q->staged && !q->pinned_in) {  // gathered here, copied with the batch's one copy below
      memcpy(b.h_in + q->st_in, q->r.keys, mb);
      if (q->r.kind == GI_REQ_RANGE) memcpy(b.h_in + q->st_in + mb, q->r.hi, mb);
      it.in = b.d_in + q->st_in;
      it.in2 = b.d_in + q->st_in + mb;
    } else {
      cudaMemcpyAsync(arena + q->in.off, q->r.keys, mb, cudaMemcpyHostToDevice, st);
      if (q->r.kind == GI_REQ_RANGE)
        cudaMemcpyAsync(arena + q->in2.off, q->r.hi, mb, cudaMemcpyHostToDevice, st);
      it.in = arena + q->in.off;
      it.in2 = arena + q->in2.off;
    }
    const bool staged_out = q->staged && !q->pinned_out && q->r.kind == GI_REQ_POINT;
    it.out = staged_out ? (void*)(b.d_out + q->st_out) : (void*)(arena + q->out.off);
    it.aux = (uint64_t*)(arena + q->aux.off);
    it.rows = nullptr;
    it.kind = q->r.kind == GI_REQ_POINT ? kItemPoint : kItemCount;
    it.work_start = work;
    work += (q->r.m + kChunk - 1) / kChunk;
    if (it.kind == kItemCount) b.h_count_items[ncount++] = n - 1;
  }
  if (b.in_used) cudaMemcpyAsync(b.d_in, b.h_in, b.in_used, cudaMemcpyHostToDevice, st);
  const uint32_t nlook = n;
  for (auto& q : b.reqs) {
    if (q->phase != 3) continue;
    ServeItem& it = b.h_items[n++];
    it.index = q->r.index;
    it.m = q->r.m;
    it.out = arena + q->out.off;
    it.aux = (uint64_t*)(arena + q->aux.off);
    it.rows = (uint32_t*)(arena + q->rows.off);
    it.in = it.in2 = nullptr;
    it.kind = kItemFill;
    it.work_start = fill_work;
    fill_work += (q->r.m + kChunk - 1) / kChunk;
  }
  cudaMemcpyAsync(b.d_items, b.h_items, n * sizeof(ServeItem), cudaMemcpyHostToDevice, st);
  if (ncount)
    cudaMemcpyAsync(b.d_count_items, b.h_count_items, ncount * 4, cudaMemcpyHostToDevice, st);
  const unsigned cap = (unsigned)(gi::sm_count() * 8);
  auto grid = [&](uint64_t w) { return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(w, cap)); };
#define GI_SV(K, KF)                                                                              \
  do {                                                                                            \
    if (nlook) {                                                                                  \
      k_serve_lookup<K, KF><<<grid(work), 256, 0, st>>>(s->d_idx, b.d_items, nlook, work, s->arena); \
      gi::count_launch();                                                                         \
    }                                                                                             \
    if (ncount) {                                                                                 \
      k_serve_scan<<<ncount, 1024, 0, st>>>(b.d_items, b.d_count_items, s->arena);                \
      gi::count_launch();                                                                         \
    }                                                                                             \
    if (n > nlook) {                                                                              \
      k_serve_fill<KF><<<grid(fill_work), 256, 0, st>>>(s->d_idx, b.d_items + nlook, n - nlook,  \
                                                        fill_work, s->arena);                     \
      gi::count_launch();                                                                         \
    }                                                                                             \
  } while (0)
  if (kb == 8) {
    switch (s->k) {
      case 0: GI_SV(uint64_t, 0); break;
      case 3: GI_SV(uint64_t, 3); break;
      case 5: GI_SV(uint64_t, 5); break;
      case 9: GI_SV(uint64_t, 9); break;
      default: GI_SV(uint64_t, 17); break;
    }
  } else {
    switch (s->k) {
      case 0: GI_SV(uint32_t, 0); break;
      case 3: GI_SV(uint32_t, 3); break;
      case 5: GI_SV(uint32_t, 5); break;
      case 9: GI_SV(uint32_t, 9); break;
      default: GI_SV(uint32_t, 17); break;
    }
  }
#undef GI_SV
  // results back: staged point results in one copy (scattered by retire_batch),
  // the rest straight into the callers' host buffers
  if (b.out_used) cudaMemcpyAsync(b.h_out, b.d_out, b.out_used, cudaMemcpyDeviceToHost, st);
  for (auto& q : b.reqs) {
    if (q->phase == 3) {
      if (q->total)
        cudaMemcpyAsync(q->r.out_rowids, s->arena + q->rows.off, q->total * 4, cudaMemcpyDeviceToHost, st);
    } else if (q->r.kind == GI_REQ_POINT) {
      if (!q->staged || q->pinned_out)
        cudaMemcpyAsync(q->r.out_rowids, s->arena + q->out.off, q->r.m * 4, cudaMemcpyDeviceToHost, st);
    } else {
      cudaMemcpyAsync(q->r.out_offsets, s->arena + q->out.off, (q->r.m + 1) * 8, cudaMemcpyDeviceToHost, st);
    }
  }
  cudaEventRecord(b.done, st);
  b.busy = true;
  s->n_batches++;
}

// a finished batch: complete its requests or move counted ranges to the fill phase
void retire_batch(gi_server* s, Batch& b, std::deque<std::shared_ptr<Req>>& fills) {
  cudaError_t e = cudaEventQuery(b.done);
  if (e == cudaErrorNotReady) return;
  if (e != cudaSuccess) {
    s->fatal = GI_ERR_CUDA;
    cudaGetLastError();
  }
  const int64_t t = now_ns();
  std::vector<std::shared_ptr<Req>> done;
  for (auto& q : b.reqs) {
    if (q->r.kind == GI_REQ_POINT) {
      if (q->staged && !q->pinned_out) memcpy(q->r.out_rowids, b.h_out + q->st_out, q->r.m * 4);
      free_block(s, q->in);
      free_block(s, q->out);
      q->phase = 4;
      done.push_back(q);
    } else if (q->phase == 1) {  // counted
      free_block(s, q->in);
      free_block(s, q->in2);
      q->total = q->r.out_offsets[q->r.m];
      if (q->total > q->r.rows_capacity) {
        q->status = GI_ERR_CAPACITY;
        free_block(s, q->out);
        free_block(s, q->aux);
        q->phase = 4;
        done.push_back(q);
      } else {
        q->phase = 2;
        fills.push_back(q);
      }
    } else {  // filled
      free_block(s, q->out);
      free_block(s, q->aux);
      free_block(s, q->rows);
      q->phase = 4;
      done.push_back(q);
    }
  }
  if (s->fatal != GI_OK)
    for (auto& q : b.reqs) q->status = s->fatal;
  b.reqs.clear();
  b.busy = false;
  if (!done.empty()) {
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto& q : done) q->t_done = t;
  }
  s->cv_done.notify_all();
}

void server_loop(gi_server* s) {
  cudaSetDevice(s->device);
  std::deque<std::shared_ptr<Req>> queue, fills;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      const bool idle = queue.empty() && fills.empty() &&
                        std::none_of(s->batches.begin(), s->batches.end(), [](const Batch& b) { return b.busy; });
      if (idle && s->incoming.empty() && !s->stop)
        s->cv_submit.wait_for(lk, std::chrono::milliseconds(2));
      if (s->stop && s->incoming.empty() && idle) return;
      while (!s->incoming.empty()) {
        queue.push_back(s->incoming.front());
        s->incoming.pop_front();
      }
    }
    for (auto& b : s->batches)
      if (b.busy) retire_batch(s, b, fills);
    // a free batch slot takes every request whose memory can be reserved now:
    // counted ranges first (they hold memory already), then new requests in order
    Batch* slot = nullptr;
    for (auto& b : s->batches)
      if (!b.busy) {
        slot = &b;
        break;
      }
    // batches in flight: poll their events without sleeping (a sleep costs the
    // scheduler's timer slack, 50-100 us, on every request's latency)
    if (!slot) {
      std::this_thread::yield();
      continue;
    }
    uint64_t probes = 0;
    slot->in_used = slot->out_used = 0;
    while (!fills.empty() && slot->reqs.size() < slot->capacity && probes < s->max_batch) {
      auto& q = fills.front();
      if (!admit(s, *q, false, false)) break;
      q->phase = 3;
      probes += q->r.m;
      slot->reqs.push_back(q);
      fills.pop_front();
    }
    while (!queue.empty() && slot->reqs.size() < slot->capacity && probes < s->max_batch) {
      auto& q = queue.front();
      // inputs (and point results) that are not pinned go through the batch's
      // staging while it has room
      const uint64_t ib = stage_in_bytes(*q, s->key_bytes), ob = stage_out_bytes(*q);
      const uint64_t at_in = up16(slot->in_used), at_out = up16(slot->out_used);
      const bool staged = at_in + ib <= slot->in_cap && at_out + ob <= slot->out_cap;
      // first-in first-out: if it does not fit, later requests wait too
      if (!admit(s, *q, staged && !q->pinned_in, staged && !q->pinned_out)) break;
      q->staged = staged;
      if (staged) {
        q->st_in = at_in;
        slot->in_used = at_in + ib;
        if (ob) {
          q->st_out = at_out;
          slot->out_used = at_out + ob;
        }
      }
      q->phase = 1;
      probes += q->r.m;
      slot->reqs.push_back(q);
      queue.pop_front();
    }
    if (!slot->reqs.empty()) {
      s->n_probes += probes;
      launch_batch(s, *slot);
    } else {
      std::this_thread::yield();
    }
  }
}

}  // namespace

extern "C" {

int gi_server_create(gi_index* const* indexes, uint32_t count, uint64_t arena_bytes,
                     uint32_t max_inflight, gi_server** out) {
  gi::set_last_error("");
  if (!out) return sfail(GI_ERR_INVALID, "gi_server_create: out is NULL");
  *out = nullptr;
  if (!indexes || count == 0) return sfail(GI_ERR_INVALID, "gi_server_create: no indexes");
  if (arena_bytes < (1u << 20)) return sfail(GI_ERR_INVALID, "gi_server_create: arena below 1 MiB");
  if (max_inflight == 0 || max_inflight > 16) return sfail(GI_ERR_INVALID, "gi_server_create: 1..16 batches in flight");
  gi_server* s = new gi_server();
  cudaGetDevice(&s->device);
  for (uint32_t i = 0; i < count; ++i) {
    gi_info inf;
    if (!indexes[i] || gi_get_info(indexes[i], &inf) != GI_OK) {
      delete s;
      return sfail(GI_ERR_INVALID, "gi_server_create: index %u is not valid", i);
    }
    const int lay = inf.layout;
    const uint32_t k = lay == GI_SORTED ? 0 : inf.k;
    if (i == 0) {
      s->key_bytes = (int)inf.key_bytes;
      s->layout = lay;
      s->k = k;
      if (!(lay == GI_SORTED || (lay == GI_EYTZINGER_KARY && (k == 3 || k == 5 || k == 9 || k == 17)))) {
        delete s;
        return sfail(GI_ERR_INVALID, "gi_server_create: indexes must be GI_SORTED or GI_EYTZINGER_KARY with k in {3,5,9,17}");
      }
    } else if ((int)inf.key_bytes != s->key_bytes || lay != s->layout || k != s->k) {
      delete s;
      return sfail(GI_ERR_INVALID, "gi_server_create: all indexes need the same key width, layout and k");
    }
    gi::sv::ServeIndex d{};
    d.keys = inf.keys;
    d.rows = inf.rowids;
    d.n = inf.n;
    d.levels = lay == GI_SORTED ? 0 : inf.levels;
    s->h_idx.push_back(d);
  }
  s->nidx = count;
  auto fail_cuda = [&](cudaError_t e, const char* what) {
    cudaGetLastError();
    for (auto& b : s->batches) {
      if (b.stream) cudaStreamDestroy(b.stream);
      if (b.done) cudaEventDestroy(b.done);
      cudaFreeHost(b.h_items);
      cudaFree(b.d_items);
      cudaFreeHost(b.h_count_items);
      cudaFree(b.d_count_items);
      cudaFreeHost(b.h_in);
      cudaFree(b.d_in);
      cudaFreeHost(b.h_out);
      cudaFree(b.d_out);
    }
    cudaFree(s->d_idx);
    cudaFree(s->arena);
    delete s;
    return sfail(e == cudaErrorMemoryAllocation ? GI_ERR_NOMEM : GI_ERR_CUDA, "gi_server_create: %s: %s",
                 what, cudaGetErrorString(e));
  };
  cudaError_t e;
  if ((e = cudaMalloc((void**)&s->d_idx, count * sizeof(gi::sv::ServeIndex))) != cudaSuccess) return fail_cuda(e, "descriptors");
  if ((e = cudaMemcpy(s->d_idx, s->h_idx.data(), count * sizeof(gi::sv::ServeIndex), cudaMemcpyHostToDevice)) != cudaSuccess)
    return fail_cuda(e, "descriptors");
  if ((e = cudaMalloc((void**)&s->arena, arena_bytes)) != cudaSuccess) return fail_cuda(e, "arena");
  s->alloc.init(arena_bytes);
  s->batches.resize(max_inflight);
  for (auto& b : s->batches) {
    b.capacity = 4096;
    if ((e = cudaStreamCreateWithFlags(&b.stream, cudaStreamNonBlocking)) != cudaSuccess) return fail_cuda(e, "stream");
    if ((e = cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming)) != cudaSuccess) return fail_cuda(e, "event");
    if ((e = cudaMallocHost((void**)&b.h_items, b.capacity * sizeof(gi::sv::ServeItem))) != cudaSuccess) return fail_cuda(e, "tables");
    if ((e = cudaMalloc((void**)&b.d_items, b.capacity * sizeof(gi::sv::ServeItem))) != cudaSuccess) return fail_cuda(e, "tables");
    if ((e = cudaMallocHost((void**)&b.h_count_items, b.capacity * 4)) != cudaSuccess) return fail_cuda(e, "tables");
    if ((e = cudaMalloc((void**)&b.d_count_items, b.capacity * 4)) != cudaSuccess) return fail_cuda(e, "tables");
    // staging for a batch's worth of inputs (ranges: two bounds each) and point results
    b.in_cap = s->max_batch * 2ull * (uint64_t)s->key_bytes;
    b.out_cap = s->max_batch * 4ull;
    if ((e = cudaMallocHost((void**)&b.h_in, b.in_cap)) != cudaSuccess) return fail_cuda(e, "staging");
    if ((e = cudaMalloc((void**)&b.d_in, b.in_cap)) != cudaSuccess) return fail_cuda(e, "staging");
    if ((e = cudaMallocHost((void**)&b.h_out, b.out_cap)) != cudaSuccess) return fail_cuda(e, "staging");
    if ((e = cudaMalloc((void**)&b.d_out, b.out_cap)) != cudaSuccess) return fail_cuda(e, "staging");
  }
  s->worker = std::thread(server_loop, s);
  *out = s;
  return GI_OK;
}

int gi_server_submit(gi_server* s, const gi_request* r, uint64_t* ticket) {
  gi::set_last_error("");
  if (!s || !r || !ticket) return sfail(GI_ERR_INVALID, "gi_server_submit: NULL argument");
  if (r->index >= s->nidx) return sfail(GI_ERR_INVALID, "gi_server_submit: index %u out of range", r->index);
  if (r->kind != GI_REQ_POINT && r->kind != GI_REQ_RANGE) return sfail(GI_ERR_INVALID, "gi_server_submit: bad kind");
  if (r->m == 0) return sfail(GI_ERR_INVALID, "gi_server_submit: empty request");
  if (!r->keys || (r->kind == GI_REQ_RANGE && (!r->hi || !r->out_offsets)) ||
      (r->kind == GI_REQ_POINT && !r->out_rowids) ||
      (r->kind == GI_REQ_RANGE && r->rows_capacity && !r->out_rowids))
    return sfail(GI_ERR_INVALID, "gi_server_submit: missing buffer");
  if (peak_bytes(*r, s->key_bytes) > s->alloc.total())
    return sfail(GI_ERR_NOMEM, "gi_server_submit: the request needs more than the whole arena");
  auto q = std::make_shared<Req>();
  q->r = *r;
  q->t_submit = now_ns();
  // which buffers the copy engine takes directly (checked on this thread, off the
  // server's).  Small requests are staged even from page-locked memory: a copy
  // call costs the server thread more than gathering a few KB, and most requests
  // are small while most bytes are in the large ones.
  if (r->m > kStageAlways) {
    const uint64_t mb = r->m * s->key_bytes;
    q->pinned_in = host_pinned(s->device, r->keys, mb) &&
                   (r->kind != GI_REQ_RANGE || host_pinned(s->device, r->hi, mb));
    if (r->kind == GI_REQ_POINT) q->pinned_out = host_pinned(s->device, r->out_rowids, r->m * 4);
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    q->ticket = s->next_ticket++;
    s->by_ticket[q->ticket] = q;
    s->incoming.push_back(q);
  }
  s->n_requests++;
  s->cv_submit.notify_one();
  *ticket = q->ticket;
  return GI_OK;
}

int gi_server_wait(gi_server* s, uint64_t ticket, int64_t* submit_ns, int64_t* done_ns) {
  gi::set_last_error("");
  if (!s) return sfail(GI_ERR_INVALID, "gi_server_wait: NULL server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->by_ticket.find(ticket);
  if (it == s->by_ticket.end()) return sfail(GI_ERR_INVALID, "gi_server_wait: unknown ticket");
  auto q = it->second;
  s->cv_done.wait(lk, [&] { return q->t_done != 0; });
  s->by_ticket.erase(it);
  if (submit_ns) *submit_ns = q->t_submit;
  if (done_ns) *done_ns = q->t_done;
  if (q->status == GI_ERR_CAPACITY)
    return sfail(GI_ERR_CAPACITY, "range result of %llu rows exceeds rows_capacity", (unsigned long long)q->total);
  if (q->status != GI_OK) return sfail(q->status, "request failed on the device");
  return GI_OK;
}

int gi_server_stats(const gi_server* s, uint64_t* batches, uint64_t* requests, uint64_t* probes) {
  if (!s) return sfail(GI_ERR_INVALID, "gi_server_stats: NULL server");
  if (batches) *batches = s->n_batches.load();
  if (requests) *requests = s->n_requests.load();
  if (probes) *probes = s->n_probes.load();
  return GI_OK;
}

// ---------------------------------------------------------------- native load generator
namespace {

// sleep most of the way (the scheduler's timer slack is ~50-100 us), then yield
// until the time has come
void sleep_until_ns(int64_t t) {
  for (;;) {
    const int64_t d = t - now_ns();
    if (d <= 0) return;
    if (d > 300000) std::this_thread::sleep_for(std::chrono::nanoseconds(d - 200000));
    else std::this_thread::yield();
  }
}

int check_trace(const gi_request* reqs, const int64_t* arrival_ns, uint64_t count,
                const int64_t* latency_ns, const char* who) {
  if (count && (!reqs || !arrival_ns || !latency_ns))
    return sfail(GI_ERR_INVALID, "%s: NULL requests, arrivals or latencies", who);
  for (uint64_t i = 0; i < count; ++i)
    if (arrival_ns[i] < 0) return sfail(GI_ERR_INVALID, "%s: negative arrival time", who);
  return GI_OK;
}

}  // namespace

int gi_server_replay(gi_server* s, const gi_request* reqs, const int64_t* arrival_ns, uint64_t count,
                     uint32_t threads, int64_t* latency_ns, int* status, double* wall_s) {
  gi::set_last_error("");
  if (!s) return sfail(GI_ERR_INVALID, "gi_server_replay: NULL server");
  if (threads == 0 || threads > 64) return sfail(GI_ERR_INVALID, "gi_server_replay: 1..64 threads");
  int rc = check_trace(reqs, arrival_ns, count, latency_ns, "gi_server_replay");
  if (rc != GI_OK) return rc;
  std::vector<uint64_t> tickets(count, 0);
  std::unique_ptr<std::atomic<int>[]> state(new std::atomic<int>[count ? count : 1]);
  for (uint64_t i = 0; i < count; ++i) state[i].store(0, std::memory_order_relaxed);
  std::vector<int> sub_rc(count, GI_OK);
  const int64_t t0 = now_ns() + 2000000;  // every submitter is up before the first arrival
  std::vector<std::thread> pool;
  for (uint32_t t = 0; t < threads; ++t) {
    pool.emplace_back([&, t] {
      for (uint64_t i = t; i < count; i += threads) {
        sleep_until_ns(t0 + arrival_ns[i]);
        sub_rc[i] = gi_server_submit(s, &reqs[i], &tickets[i]);
        state[i].store(sub_rc[i] == GI_OK ? 1 : 2, std::memory_order_release);
      }
    });
  }
  // this thread collects the completions; latencies come from the server's own
  // completion times, so the order of collection does not matter
  int first_bad = GI_OK;
  for (uint64_t i = 0; i < count; ++i) {
    int st;
    while ((st = state[i].load(std::memory_order_acquire)) == 0) std::this_thread::yield();
    int r = sub_rc[i];
    int64_t sub = 0, done = 0;
    if (st == 1) r = gi_server_wait(s, tickets[i], &sub, &done);
    latency_ns[i] = st == 1 ? done - (t0 + arrival_ns[i]) : -1;
    if (status) status[i] = r;
    if (r != GI_OK && r != GI_ERR_CAPACITY && first_bad == GI_OK) first_bad = r;
  }
  for (auto& th : pool) th.join();
  if (wall_s) *wall_s = (double)(now_ns() - t0) * 1e-9;
  if (first_bad != GI_OK) return sfail(first_bad, "gi_server_replay: a request failed");
  return GI_OK;
}

int gi_replay_serial(gi_index* const* indexes, uint32_t nindexes, const gi_request* reqs,
                     const int64_t* arrival_ns, uint64_t count, int64_t* latency_ns, int* status,
                     double* wall_s) {
  gi::set_last_error("");
  if (!indexes || nindexes == 0) return sfail(GI_ERR_INVALID, "gi_replay_serial: no indexes");
  int rc = check_trace(reqs, arrival_ns, count, latency_ns, "gi_replay_serial");
  if (rc != GI_OK) return rc;
  for (uint64_t i = 0; i < count; ++i)
    if (reqs[i].index >= nindexes || !indexes[reqs[i].index] || reqs[i].m == 0)
      return sfail(GI_ERR_INVALID, "gi_replay_serial: request %llu names no index or is empty",
                   (unsigned long long)i);
  const int64_t t0 = now_ns() + 1000000;
  int first_bad = GI_OK;
  for (uint64_t i = 0; i < count; ++i) {
    const gi_request& q = reqs[i];
    sleep_until_ns(t0 + arrival_ns[i]);
    gi_index* ix = indexes[q.index];
    int r;
    if (q.kind == GI_REQ_POINT) {
      r = gi_point_lookup(ix, q.keys, q.m, q.out_rowids);
    } else {  // the two-call protocol: offsets, then the rows if they fit
      r = gi_range_lookup(ix, q.keys, q.hi, q.m, q.out_offsets, nullptr);
      if (r == GI_OK) {
        const uint64_t total = q.out_offsets[q.m];
        if (total > q.rows_capacity) r = GI_ERR_CAPACITY;
        else if (total) r = gi_range_lookup(ix, q.keys, q.hi, q.m, q.out_offsets, q.out_rowids);
      }
    }
    latency_ns[i] = now_ns() - (t0 + arrival_ns[i]);
    if (status) status[i] = r;
    if (r != GI_OK && r != GI_ERR_CAPACITY && first_bad == GI_OK) first_bad = r;
  }
  if (wall_s) *wall_s = (double)(now_ns() - t0) * 1e-9;
  if (first_bad != GI_OK) return sfail(first_bad, "gi_replay_serial: a request failed");
  return GI_OK;
}

void gi_server_destroy(gi_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_submit.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto& b : s->batches) {
    if (b.stream) cudaStreamSynchronize(b.stream);
    if (b.stream) cudaStreamDestroy(b.stream);
    if (b.done) cudaEventDestroy(b.done);
    cudaFreeHost(b.h_items);
    cudaFree(b.d_items);
    cudaFreeHost(b.h_count_items);
    cudaFree(b.d_count_items);
    cudaFreeHost(b.h_in);
    cudaFree(b.d_in);
    cudaFreeHost(b.h_out);
    cudaFree(b.d_out);
  }
  cudaFree(s->d_idx);
  cudaFree(s->arena);
  cudaGetLastError();
  delete s;
}

}  // extern "C"
