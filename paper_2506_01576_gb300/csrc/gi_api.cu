// The C ABI of include/gi.h: argument checks, the index object, device memory,
// host-memory staging, and the choice of kernel configuration.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include "gi_alloc.h"
#include "gi_internal.cuh"
#include "gi_ptr.h"

// ---------------------------------------------------------------- the index object
struct GiStaging {
  cudaStream_t st[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t ev = nullptr;
  cudaEvent_t cev[8] = {};  // one per range-fill chunk
  void* q[3] = {nullptr, nullptr, nullptr};
  uint32_t* out[3] = {nullptr, nullptr, nullptr};
  uint64_t chunk = 0;  // probes per chunk
};

struct gi_index {
  int device = 0;
  cudaStream_t stream = nullptr;
  uint64_t n = 0;
  int layout = 0;
  uint32_t k = 0;
  int key_bytes = 4;
  bool unique = true;
  void* keys = nullptr;        // EYTZINGER: slot t at keys[t+1]
  uint32_t* rows = nullptr;
  uint32_t* dflags = nullptr;  // device status word
  gi::Geom geom{};
  int64_t opt[11] = {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1};
  // range-lookup scratch and the state of the two-call protocol
  void* rscratch = nullptr;
  size_t rscratch_bytes = 0;
  const void* last_lo = nullptr;
  const void* last_hi = nullptr;
  uint64_t last_m = 0;
  const uint64_t* last_off = nullptr;
  bool counts_valid = false;
  GiStaging* stage = nullptr;
  uint32_t latched = 0;  // device status seen by the host
};

namespace {

thread_local std::string t_err;
thread_local cudaStream_t t_default_stream = nullptr;
std::atomic<uint64_t> g_launches{0};

int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  t_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  cudaGetLastError();  // clear a sticky-free error
  if (e == cudaErrorMemoryAllocation) return fail(GI_ERR_NOMEM, "%s: %s", what, cudaGetErrorString(e));
  return fail(GI_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define GI_CUDA(call, what)                     \
  do {                                          \
    cudaError_t e_ = (call);                    \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

// Makes the index's device current for the scope of a call, then restores.
struct DeviceScope {
  int prev = -1;
  explicit DeviceScope(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceScope() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

enum PtrKind { kDevice, kHost, kBad };

// How a call treats pointer p given the index's device `dev`: in place (device
// memory of `dev`, or managed memory), staged (host memory), or kBad (NULL, or
// device memory of another device, which a kernel on `dev` must not be given).
PtrKind pointer_kind(const void* p, int dev) {
  if (!p) return kBad;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  int type = -1, pdev = -1;
  if (e != cudaSuccess) {
    cudaGetLastError();
  } else {
    type = (int)a.type;
    pdev = a.device;
  }
  switch (gi::classify_pointer(type, pdev, dev)) {
    case gi::kPtrDevice: return kDevice;
    case gi::kPtrHost: return kHost;
    default: return kBad;
  }
}

// The device's view of page-locked (registered or cudaHostAlloc'ed) host memory,
// or NULL for pageable memory.
const void* mapped_host(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

using gi::key_alloc_bytes;  // key arrays: room for the empty slot and whole-node reads past n
using gi::key_used_bytes;
using gi::round256;
using gi::row_alloc_bytes;

// Page-locked host scratch of the calling thread for the build's small
// device-to-host reads (digit flags and counts): copies into pageable memory would
// block the host until the stream drains, before the next kernel is queued.  It
// lives as long as the thread (532 KB); it is not freed at thread exit, when the
// CUDA runtime may already be shutting down.
struct PinnedScratch {
  uint32_t* trivial = nullptr;        // [8]
  unsigned long long* hist = nullptr;  // [8][256]
  unsigned long long* h2 = nullptr;    // [256][256]
  unsigned long long* win = nullptr;   // [2 + 256]: the MSD window's record
  cudaEvent_t ev = nullptr;
  int device = -1;
  cudaError_t ensure() {
    int dev = 0;
    cudaGetDevice(&dev);
    if (trivial && dev == device) return cudaSuccess;
    if (trivial) {  // another device: new allocations in its context
      cudaFreeHost(trivial);
      cudaEventDestroy(ev);
      trivial = nullptr;
    }
    void* p = nullptr;
    const size_t bytes = 256 + sizeof(uint64_t) * (8 * 256 + 256 * 256 + 2 + 256);
    cudaError_t e = cudaMallocHost(&p, bytes);
    if (e != cudaSuccess) return e;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      cudaFreeHost(p);
      return e;
    }
    trivial = (uint32_t*)p;
    hist = (unsigned long long*)((char*)p + 256);
    h2 = hist + 8 * 256;
    win = h2 + 256 * 256;
    device = dev;
    return cudaSuccess;
  }
};
PinnedScratch& pinned_scratch() {
  static thread_local PinnedScratch t;
  return t;
}

// Device memory comes from the device's stream-ordered pool.  The pool's release
// threshold is raised once per device to 8 GiB (a setting of this process only):
// the sort buffers a build frees are reused by the next build instead of being
// unmapped and mapped again at every synchronisation, while freed memory beyond
// 8 GiB still goes back to the driver.
// Test hook (gi_debug_fail_alloc): the countdown of device allocations until one
// reports out-of-memory on the host side, or -1.
std::atomic<int64_t> g_fail_alloc{-1};

bool injected_alloc_failure() {
  int64_t v = g_fail_alloc.load();
  while (v >= 0)
    if (g_fail_alloc.compare_exchange_weak(v, v - 1)) return v == 0;
  return false;
}

cudaError_t dalloc(void** p, size_t bytes, cudaStream_t s) {
  if (injected_alloc_failure()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  static std::once_flag once[64];
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64) {
    std::call_once(once[dev], [dev] {
      cudaMemPool_t pool;
      if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = 8ull << 30;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
      }
      cudaGetLastError();
    });
  }
  return cudaMallocAsync(p, bytes, s);
}
void dfree(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

int read_flags(gi_index* idx) {
  uint32_t f = 0;
  cudaError_t e = cudaMemcpyAsync(&f, idx->dflags, sizeof f, cudaMemcpyDeviceToHost, idx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(idx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "reading device status");
  idx->latched |= f;
  return GI_OK;
}

int check_latched(gi_index* idx) {
  if (idx->latched & gi::kFlagTimeout)
    return fail(GI_ERR_TIMEOUT, "a bounded device-side wait gave up; results are not valid");
  return GI_OK;
}

gi::LookupCfg resolve_cfg(const gi_index* idx) {
  gi::LookupCfg c;
  c.layout = idx->layout;
  c.key_bytes = idx->key_bytes;
  // knobs left automatic take the autotuner's entry for this size class, if any
  int64_t o[11];
  for (int i = 0; i < 11; ++i) o[i] = idx->opt[i];
  int64_t tb[11];
  if (gi::tune_table_lookup(idx->key_bytes, idx->layout, idx->k, idx->n, tb)) {
    for (int i = 1; i < 11; ++i)
      if (o[i] < 0 && tb[i] >= 0 && i != GI_OPT_RANGE_FILL) o[i] = tb[i];
    if (o[GI_OPT_GROUP] >= 0 && idx->opt[GI_OPT_GROUP] < 0 &&
        (idx->layout != GI_EYTZINGER_KARY || !gi::eks_group_supported(idx->k, idx->key_bytes, (int)o[GI_OPT_GROUP])))
      o[GI_OPT_GROUP] = -1;
    if (o[GI_OPT_SMEM_LEVELS] > 0 && idx->opt[GI_OPT_SMEM_LEVELS] < 0) {
      const uint64_t slots = gi::smem_slots_for_levels(idx->layout, idx->geom, (int)o[GI_OPT_SMEM_LEVELS], idx->key_bytes);
      if (((slots * idx->key_bytes + 15) & ~15ull) > (uint64_t)gi::device_max_smem_optin() - 1024)
        o[GI_OPT_SMEM_LEVELS] = -1;  // the recorded depth does not fit this index
    }
  }
  c.group = o[GI_OPT_GROUP] >= 0 ? (int)o[GI_OPT_GROUP]
                                  : (idx->layout == GI_EYTZINGER_KARY
                                         ? gi::eks_default_group(idx->k, idx->key_bytes)
                                         : 1);
  int def_pt = 1;
  if (idx->layout == GI_EYTZINGER) def_pt = 4;
  c.per_thread = o[GI_OPT_PER_THREAD] >= 0 ? (int)o[GI_OPT_PER_THREAD] : def_pt;
  c.smem_levels = o[GI_OPT_SMEM_LEVELS] >= 0 ? (int)o[GI_OPT_SMEM_LEVELS] : 0;
  // k-ary lookups: 512 threads per block measured 3% faster than 256 at 2^26 u64
  // keys, k = 5 (interleaved A/B, 2^27 probes), and the autotuner picks 512 at
  // most sizes from 2^18 keys up
  c.block = o[GI_OPT_BLOCK] >= 0 ? (int)o[GI_OPT_BLOCK] : (idx->layout == GI_EYTZINGER_KARY ? 512 : 256);
  c.blocks_per_sm = o[GI_OPT_BLOCKS_PER_SM] >= 0 ? (int)o[GI_OPT_BLOCKS_PER_SM] : 0;
  c.prefetch = o[GI_OPT_PREFETCH] >= 0 ? (int)o[GI_OPT_PREFETCH] : 0;
  const int ee = o[GI_OPT_EARLY_EXIT] >= 0 ? (int)o[GI_OPT_EARLY_EXIT] : 1;
  c.early_exit = (ee && idx->unique) ? 1 : 0;
  if (c.layout == GI_SORTED) c.per_thread = 1;
  // the per-rank map measured faster except for 256-row ranges on 17-ary trees
  c.range_fill = o[GI_OPT_RANGE_FILL] >= 0 ? (int)o[GI_OPT_RANGE_FILL] : 0;
  c.reorder = o[GI_OPT_REORDER] >= 0 ? (int)o[GI_OPT_REORDER] : 0;
  int dev = idx->device, l2 = 0;
  cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
  if (o[GI_OPT_HOT_LEVELS] >= 0) {
    c.hot_levels = (int)o[GI_OPT_HOT_LEVELS];
  } else {
    // evict-last for the top levels that fit in 5/8 of L2.  Measured at 2^26 u64
    // keys, k = 5, 2^27 probes, with the deep levels kept out of L1 (below):
    // levels 0..9 (78 MB of the 135 MB L2) evict-last, 5.22 ms; 0..8 (16 MB),
    // 5.79 ms; 0..7, 5.88 ms.  (While every level was also allocated in L1,
    // 0..8 and 0..9 measured within 3% of each other.)
    c.hot_levels = gi::levels_within(idx->geom, idx->key_bytes, (uint64_t)l2 * 5 / 8);
  }
  // top levels read through L1: those within 128 KB of keys (the L1 of an SM
  // holds them while no shared memory is used).  Measured at 2^26 u64 keys, k = 5:
  // levels 0..5 (125 KB) through L1 and the rest not allocated there, 5.78 ms;
  // every level allocated, 5.97 ms; 0..3, 5.88 ms; 0..7, 6.00 ms.  An index whose
  // keys and rowIDs fit in 192 KB keeps everything in L1 (rowIDs included).
  const uint64_t index_bytes = idx->n * (uint64_t)(idx->key_bytes + 4);
  c.l1_levels = index_bytes <= (192u << 10) ? (int)idx->geom.levels
                                            : gi::levels_within(idx->geom, idx->key_bytes, 128u << 10);
  return c;
}

cudaError_t launch_point(const gi_index* idx, const gi::LookupCfg& c, const void* q, uint64_t m,
                         uint32_t* out, cudaStream_t s) {
  if (idx->key_bytes == 4)
    return gi::point_lookup_u32(idx->keys, idx->rows, idx->geom, c, q, m, out, idx->dflags, s);
  return gi::point_lookup_u64(idx->keys, idx->rows, idx->geom, c, q, m, out, idx->dflags, s);
}

void free_staging(gi_index* idx) {
  GiStaging* st = idx->stage;
  if (!st) return;
  cudaStreamSynchronize(idx->stream);
  for (int i = 0; i < 3; ++i) {
    if (st->st[i]) cudaStreamSynchronize(st->st[i]);
    if (st->q[i]) cudaFreeAsync(st->q[i], st->st[i]);
    if (st->out[i]) cudaFreeAsync(st->out[i], st->st[i]);
    if (st->st[i]) {
      cudaStreamSynchronize(st->st[i]);
      cudaStreamDestroy(st->st[i]);
    }
  }
  if (st->ev) cudaEventDestroy(st->ev);
  for (cudaEvent_t e : st->cev)
    if (e) cudaEventDestroy(e);
  delete st;
  idx->stage = nullptr;
}

int ensure_staging(gi_index* idx, uint64_t chunk) {
  if (idx->stage && idx->stage->chunk >= chunk) return GI_OK;
  free_staging(idx);
  GiStaging* st = new GiStaging();
  st->chunk = chunk;
  idx->stage = st;
  // on any failure the partial staging is freed, so a later call starts over
  // instead of finding buffers that were never allocated
  auto give_up = [&](cudaError_t e, const char* what) {
    free_staging(idx);
    return cuda_fail(e, what);
  };
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&st->st[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = dalloc(&st->q[i], chunk * idx->key_bytes, st->st[i]);
    if (e == cudaSuccess) e = dalloc((void**)&st->out[i], chunk * 4, st->st[i]);
  }
  if (e != cudaSuccess) return give_up(e, "staging buffer");
  e = cudaEventCreateWithFlags(&st->ev, cudaEventDisableTiming);
  for (cudaEvent_t& ev : st->cev)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e != cudaSuccess) return give_up(e, "staging event");
  return GI_OK;
}

int ensure_range_scratch(gi_index* idx, uint64_t m) {
  const size_t need = gi::range_scratch_bytes(m);
  if (idx->rscratch_bytes >= need) return GI_OK;
  dfree(idx->rscratch, idx->stream);
  idx->rscratch = nullptr;
  idx->rscratch_bytes = 0;
  idx->counts_valid = false;
  GI_CUDA(dalloc(&idx->rscratch, need, idx->stream), "range scratch");
  idx->rscratch_bytes = need;
  return GI_OK;
}

}  // namespace

namespace gi {

void count_launch(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

cudaStream_t index_stream(const gi_index* idx) { return idx->stream; }

int index_device(const gi_index* idx) { return idx->device; }

int64_t index_raw_option(const gi_index* idx, int option) { return idx->opt[option]; }

void set_last_error(const char* msg) { t_err = msg; }

int sm_count() {
  static int cached[64];
  static std::once_flag once[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  std::call_once(once[dev], [&] {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = v > 0 ? v : 1;
  });
  return cached[dev];
}

int device_max_smem_optin() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v;
}

Geom make_geom(uint64_t n, uint32_t k) {
  Geom g{};
  g.n = n;
  g.k = k;
  g.log2k = ((k & (k - 1)) == 0) ? ilog2_const(k) : 0;
  if (n == 0) return g;
  uint32_t m = 0;
  uint64_t p = 1;
  while (p <= n / k) {
    p *= k;
    ++m;
  }
  g.m = m;
  g.top = p - 1;
  g.b = n - g.top;
  g.levels = m + 1;
  return g;
}

size_t range_scratch_bytes(uint64_t m) {
  const uint64_t nb = (m + 2047) / 2048;
  return round256(sizeof(uint64_t) * (m ? m : 1)) + round256(sizeof(uint64_t) * (nb + 1));
}

bool eks_group_supported(uint32_t k, int key_bytes, int group) {
#define GI_X(KF, G) \
  if (k == KF && group == G) return true;
  if (key_bytes == 8) {
    GI_EKS_PAIRS_U64(GI_X)
  } else {
    GI_EKS_PAIRS_U32(GI_X)
  }
#undef GI_X
  return false;
}

int eks_default_group(uint32_t k, int key_bytes) {
  // One thread per lookup reading its whole node measured fastest wherever that
  // kernel is compiled: with vector loads up to 128-byte nodes (2^26 u64 keys,
  // k = 17: 10.9 ms for 2^27 lookups against 12.6 ms with 4 lanes of 32 bytes;
  // k = 9: 6.7 ms against 10.3 with 2 lanes), and with one load per key for nodes
  // that are not whole 16-byte vectors (k = 16, u64, 120-byte nodes: 8.2 G
  // lookups/s against 4.2 with 16 lanes at 2^26 keys, 48.9 against 9.3 at 2^10).
  // Fan-outs without a one-lane kernel split the node over lanes in 32-byte
  // pieces, one sector per lane, else 16-byte pieces.
  const int node_bytes = (int)(k - 1) * key_bytes;
  if (eks_group_supported(k, key_bytes, 1)) return 1;
  if (node_bytes % 32 == 0 && eks_group_supported(k, key_bytes, node_bytes / 32)) return node_bytes / 32;
  if (node_bytes % 16 == 0 && eks_group_supported(k, key_bytes, node_bytes / 16)) return node_bytes / 16;
  for (int g = 32; g >= 1; g >>= 1)
    if (eks_group_supported(k, key_bytes, g)) return g;
  return 1;  // generic kernel
}

int levels_within(const Geom& g, int key_bytes, uint64_t budget) {
  if (g.n == 0 || g.k < 2) return 0;
  uint64_t cum = 0, width = g.k - 1;
  int l = 0;
  while (l < (int)g.levels) {
    const uint64_t keys = l + 1 < (int)g.levels ? width : g.b;
    cum += keys * key_bytes;
    if (cum > budget) break;
    ++l;
    if (width > (~0ull) / g.k) break;
    width *= g.k;
  }
  return l;
}

uint64_t smem_slots_for_levels(int layout, const Geom& g, int levels, int key_bytes) {
  (void)key_bytes;
  if (levels <= 0 || g.n == 0 || layout == GI_SORTED) return 0;
  if (layout == GI_EYTZINGER) {
    const uint64_t s = levels >= 40 ? (1ull << 40) : (1ull << levels);  // slots 0 .. 2^d - 1
    return std::min<uint64_t>(s, g.n + 1);
  }
  uint64_t top = 1;
  for (int i = 0; i < levels && top <= g.n; ++i) top *= g.k;
  top -= 1;  // k^d - 1 slots: d whole levels
  const uint64_t node = g.k - 1;
  const uint64_t whole = (g.n + node - 1) / node * node;  // round n up to whole nodes
  return std::min<uint64_t>(top, whole);
}

}  // namespace gi

// ================================================================= C ABI
extern "C" {

const char* gi_last_error(void) { return t_err.c_str(); }

uint64_t gi_launch_count(void) { return g_launches.load(); }

void gi_debug_fail_alloc(int64_t after) { g_fail_alloc.store(after < 0 ? -1 : after); }

int gi_set_stream(gi_index* idx, void* stream) {
  t_err.clear();
  if (!idx) {
    t_default_stream = (cudaStream_t)stream;
    return GI_OK;
  }
  idx->stream = (cudaStream_t)stream;
  return GI_OK;
}

static void destroy_impl(gi_index* idx) {
  if (!idx) return;
  DeviceScope ds(idx->device);
  cudaStreamSynchronize(idx->stream);
  free_staging(idx);
  dfree(idx->keys, idx->stream);
  dfree(idx->rows, idx->stream);
  dfree(idx->dflags, idx->stream);
  dfree(idx->rscratch, idx->stream);
  cudaStreamSynchronize(idx->stream);
  cudaGetLastError();
  delete idx;
}

void gi_destroy(gi_index* idx) { destroy_impl(idx); }

int gi_build(const void* keys, const uint32_t* rowids, uint64_t n, int layout, uint32_t k,
             gi_index** out) {
  t_err.clear();
  if (!out) return fail(GI_ERR_INVALID, "gi_build: out is NULL");
  *out = nullptr;
  const int lay = layout & 0xFF;
  const int kw = layout & 0xFF00;
  const int flags = layout & ~0xFFFF;
  if (kw != GI_KEY_U32 && kw != GI_KEY_U64) return fail(GI_ERR_INVALID, "gi_build: bad key width bits 0x%x", kw);
  if (flags & ~(GI_BUILD_LSD | GI_BUILD_HYBRID))
    return fail(GI_ERR_INVALID, "gi_build: unknown build flags 0x%x", flags);
  if ((flags & GI_BUILD_LSD) && (flags & GI_BUILD_HYBRID))
    return fail(GI_ERR_INVALID, "gi_build: GI_BUILD_LSD and GI_BUILD_HYBRID together");
  if (lay != GI_SORTED && lay != GI_EYTZINGER && lay != GI_EYTZINGER_KARY)
    return fail(GI_ERR_INVALID, "gi_build: unknown layout %d", lay);
  if (lay == GI_EYTZINGER_KARY && (k < 2 || k > 33))
    return fail(GI_ERR_INVALID, "gi_build: k must be in [2, 33], got %u", k);
  if (n > 0 && (!keys || !rowids)) return fail(GI_ERR_INVALID, "gi_build: NULL keys or rowids");
  if (n >= (1ull << 40)) return fail(GI_ERR_INVALID, "gi_build: n too large");
  const int kb = kw == GI_KEY_U64 ? 8 : 4;

  gi_index* idx = new gi_index();
  idx->stream = t_default_stream;
  cudaGetDevice(&idx->device);
  idx->n = n;
  idx->layout = lay;
  idx->k = lay == GI_SORTED ? 0 : (lay == GI_EYTZINGER ? 2 : k);
  idx->key_bytes = kb;
  idx->geom = gi::make_geom(n, lay == GI_SORTED ? 2 : idx->k);
  cudaStream_t s = idx->stream;

  auto bail = [&](int rc) {
    destroy_impl(idx);
    return rc;
  };
  int rc = GI_OK;
#define GI_TRY(call, what)                      \
  do {                                          \
    cudaError_t e_ = (call);                    \
    if (e_ != cudaSuccess) return bail(cuda_fail(e_, what)); \
  } while (0)

  GI_TRY(dalloc((void**)&idx->dflags, 256, s), "status word");
  GI_TRY(cudaMemsetAsync(idx->dflags, 0, 256, s), "status word");
  const size_t kbytes = key_alloc_bytes(n, kb), rbytes = row_alloc_bytes(n);
  if (n == 0) {
    GI_TRY(dalloc(&idx->keys, kbytes, s), "index keys");
    GI_TRY(dalloc((void**)&idx->rows, rbytes, s), "index rows");
    GI_TRY(cudaMemsetAsync(idx->keys, 0xFF, kbytes, s), "index keys");
    GI_TRY(cudaStreamSynchronize(s), "gi_build");
    *out = idx;
    return GI_OK;
  }
  const PtrKind kk = pointer_kind(keys, idx->device), rk = pointer_kind(rowids, idx->device);
  if (kk == kBad || rk == kBad)
    return bail(fail(GI_ERR_INVALID, "gi_build: keys or rowids are device memory of another device"));
  void* bk[2] = {nullptr, nullptr};
  uint32_t* bv[2] = {nullptr, nullptr};
  void* scratch = nullptr;
  auto free_tmp = [&]() {
    for (int i = 0; i < 2; ++i) {
      if (bk[i] != idx->keys) dfree(bk[i], s);
      if (bv[i] != idx->rows) dfree(bv[i], s);
    }
    dfree(scratch, s);
  };
  auto bail_tmp = [&](int code) {
    free_tmp();
    return bail(code);
  };
#define GI_TRY2(call, what)                     \
  do {                                          \
    cudaError_t e_ = (call);                    \
    if (e_ != cudaSuccess) return bail_tmp(cuda_fail(e_, what)); \
  } while (0)
  for (int i = 0; i < 2; ++i) {
    GI_TRY2(dalloc(&bk[i], kbytes, s), "sort buffer");
    GI_TRY2(dalloc((void**)&bv[i], rbytes, s), "sort buffer");
  }
  // Host inputs.  Page-locked memory is read by the kernels over the bus: the
  // histogram pass copies the keys into bk[0] as it counts them, and the first
  // sort pass reads the rowIDs where they are (each crosses the bus once, and
  // the copies overlap the histogram and the first pass).  Pageable memory is
  // copied first.
  const void* src_k = keys;
  const uint32_t* src_v = rowids;
  const void* keys_bus = nullptr;  // page-locked host keys, device view
  bool staged = false;
  if (kk == kHost) {
    keys_bus = mapped_host(keys);
    if (!keys_bus)
      GI_TRY2(cudaMemcpyAsync(bk[0], keys, n * kb, cudaMemcpyHostToDevice, s), "copying keys");
    src_k = bk[0];
    staged = true;
  }
  if (rk == kHost) {
    const void* rows_bus = mapped_host(rowids);
    if (rows_bus) {
      src_v = (const uint32_t*)rows_bus;
    } else {
      GI_TRY2(cudaMemcpyAsync(bv[0], rowids, n * 4, cudaMemcpyHostToDevice, s), "copying rowids");
      src_v = bv[0];
      staged = true;
    }
  }
  const size_t sbytes = gi::sort_scratch_bytes(n, kb);
  GI_TRY2(dalloc(&scratch, sbytes, s), "sort scratch");
  // histogram and digit offsets; their copy to the host is waited for only after
  // the first MSD pass is queued behind them (speculatively on the top byte, where
  // the hybrid sort starts for keys that use it), so the GPU does not idle while
  // the host plans
  PinnedScratch& pin = pinned_scratch();
  GI_TRY2(pin.ensure(), "page-locked scratch");
  // Where the hybrid sort will likely follow (u64 keys from 2^18 pairs up, u32
  // keys from 2^23, or forced), the histogram pass also finds the bits in which keys differ and a
  // second read counts the 8-bit window just below the highest of them; the first
  // MSD scatter on that window is queued at once, before the host has seen any
  // counts.  Up to 256 x 256 x 7/8 of the bucket capacity pairs: beyond, buckets
  // of uniform keys would be too large for a CTA and the LSD sort would redo it.
  const uint64_t spec_max = 256ull * 256ull * gi::local_sort_capacity() / 8 * 7;
  const bool hybrid_ok = !(flags & GI_BUILD_LSD) && n < (1ull << 32) &&
                         ((n >= gi::hybrid_min_pairs(kb) && n <= spec_max) || (flags & GI_BUILD_HYBRID));
  GI_TRY2(gi::sort_prepare(keys_bus ? keys_bus : src_k, keys_bus ? bk[0] : nullptr, n, kb, scratch,
                           s, pin.trivial, hybrid_ok ? pin.win : nullptr,
                           (flags & GI_BUILD_HYBRID) ? 2u : gi::hybrid_min_digits(kb)),
          "histogram");
  cudaEvent_t hist_ready = pin.ev;
  GI_TRY2(cudaEventRecord(hist_ready, s), "histogram");
  // Ping-pong between the two buffers; the first pass writes the buffer that does
  // not hold a staged copy of the input.
  const void* ck = src_k;
  const uint32_t* cv = src_v;
  int cur = -1;  // -1: the data is still the (caller's or staged) input
  int next_dst = staged ? 1 : 0;
  bool speculate = hybrid_ok;
  if (speculate)  // skipped on the device if every key has the same window value
    GI_TRY2(gi::sort_window_pass(ck, cv, bk[next_dst], bv[next_dst], n, kb, scratch, idx->dflags, s),
            "radix pass");
  GI_TRY2(cudaEventSynchronize(hist_ready), "histogram");
  uint32_t trivial = 0;  // digits with one value only: zero bytes of the OR of key ^ keys[0]
  for (int p = 0; p < kb; ++p)
    if (hybrid_ok ? ((pin.win[0] >> (8 * p)) & 0xFF) == 0 : pin.trivial[p] != 0) trivial |= 1u << p;
  if (speculate && (pin.win[1] >> 32)) speculate = false;  // that pass wrote nothing
  bool sorted_done = false, pass1_pending_reset = false;
  if (speculate) {  // the MSD pass ran: a stable permutation into bk[next_dst]
    ck = bk[next_dst];
    cv = bv[next_dst];
    cur = next_dst;
    pass1_pending_reset = true;
  }
  if (!(flags & GI_BUILD_LSD)) {  // hybrid MSD + shared-memory bucket sort where it applies
    int res = -1, verify = -1;
    bool used = false;
    const uint32_t nontrivial = ~trivial & ((1u << kb) - 1);
    GI_TRY2(gi::hybrid_sort(speculate ? src_k : ck, speculate ? src_v : cv, bk, bv,
                            speculate ? cur : next_dst, n, kb, nontrivial,
                            hybrid_ok ? pin.win : nullptr, scratch, idx->geom, lay == GI_SORTED,
                            lay == GI_EYTZINGER ? 1u : 0u, (flags & GI_BUILD_HYBRID) != 0,
                            speculate, pin.h2, idx->dflags, s, &res, &used, &verify),
            "hybrid sort");
    if (used && verify >= 0) {
      // the bucket lists were made on the device: a bucket too large for one CTA
      // (skewed keys) was left out and counted; then sort from the scattered data
      GI_TRY2(cudaStreamSynchronize(s), "hybrid sort");
      if (*(volatile uint32_t*)pin.h2 != 0) {
        used = false;
        res = verify;
        GI_TRY2(gi::sort_reset_counters(scratch, kb, s), "radix pass");
      }
    }
    if (res >= 0) {
      ck = bk[res];
      cv = bv[res];
      pass1_pending_reset = pass1_pending_reset && res == cur;  // else reset inside
      cur = res;
      sorted_done = used;  // bk[res] holds the finished layout, duplicates flagged
    }
  }
  if (cur >= 0) next_dst = 1 - cur;
  if (!sorted_done && pass1_pending_reset)  // the LSD passes reuse the MSD pass's ticket
    GI_TRY2(gi::sort_reset_counters(scratch, kb, s), "radix pass");
  if (!sorted_done && hybrid_ok && (trivial != (1u << kb) - 1))  // digit counts skipped so far
    GI_TRY2(gi::sort_counts(ck, n, kb, scratch, s), "histogram");
  for (int p = 0; p < kb && !sorted_done; ++p) {
    if (trivial & (1u << p)) continue;  // every key has the same digit here
    const int dst = next_dst;
    // the pass that reads the input rowIDs checks them for the reserved value
    GI_TRY2(gi::sort_pass(ck, cv, bk[dst], bv[dst], n, kb, p, scratch, idx->dflags, cur < 0, s),
            "radix pass");
    ck = bk[dst];
    cv = bv[dst];
    cur = dst;
    next_dst = 1 - dst;
  }
  if (cur < 0) GI_TRY2(gi::check_rowids(cv, n, idx->dflags, s), "rowID check");  // no pass ran
  if (sorted_done) {
    idx->keys = bk[cur];
    idx->rows = bv[cur];
  } else if (lay == GI_SORTED) {
    if (cur < 0) {  // no pass ran (all keys equal): the input order is the sorted order
      cur = next_dst;
      GI_TRY2(cudaMemcpyAsync(bk[cur], ck, n * kb, cudaMemcpyDefault, s), "copy");
      GI_TRY2(cudaMemcpyAsync(bv[cur], cv, n * 4, cudaMemcpyDefault, s), "copy");
    }
    idx->keys = bk[cur];
    idx->rows = bv[cur];
    GI_TRY2(gi::check_sorted_dups(idx->keys, n, kb, idx->dflags, s), "duplicate check");
  } else {
    const int dst = cur >= 0 ? 1 - cur : next_dst;
    GI_TRY2(gi::layout_gather(ck, cv, bk[dst], bv[dst], idx->geom, kb,
                              lay == GI_EYTZINGER ? 1u : 0u, idx->dflags, s),
            "layout permutation");
    idx->keys = bk[dst];
    idx->rows = bv[dst];
  }
  {
    // slots past the last key hold the maximum key: whole-node reads need no bounds checks
    const size_t used = key_used_bytes(n, kb, lay == GI_EYTZINGER);
    GI_TRY2(cudaMemsetAsync((char*)idx->keys + used, 0xFF, kbytes - used, s), "key padding");
  }
  free_tmp();
  rc = read_flags(idx);
  if (rc != GI_OK) return bail(rc);
  if (idx->latched & gi::kFlagReservedRowid)
    return bail(fail(GI_ERR_INVALID, "gi_build: a rowID equals the reserved value GI_MISS"));
  if (idx->latched & gi::kFlagTimeout)
    return bail(fail(GI_ERR_TIMEOUT, "gi_build: a bounded device-side wait gave up"));
  idx->unique = !(idx->latched & gi::kFlagDuplicate);
  idx->latched = 0;
  GI_TRY(cudaMemsetAsync(idx->dflags, 0, 256, s), "status word");
  *out = idx;
  return GI_OK;
#undef GI_TRY
#undef GI_TRY2
}

int gi_point_lookup(const gi_index* cidx, const void* queries, uint64_t m, uint32_t* out_rowids) {
  t_err.clear();
  gi_index* idx = const_cast<gi_index*>(cidx);
  if (!idx) return fail(GI_ERR_INVALID, "gi_point_lookup: NULL index");
  if (m == 0) return GI_OK;
  if (!queries || !out_rowids) return fail(GI_ERR_INVALID, "gi_point_lookup: NULL pointer");
  DeviceScope ds(idx->device);
  const gi::LookupCfg c = resolve_cfg(idx);
  const PtrKind qk = pointer_kind(queries, idx->device), ok = pointer_kind(out_rowids, idx->device);
  if (qk == kBad || ok == kBad)
    return fail(GI_ERR_INVALID, "gi_point_lookup: a buffer is device memory of another device");
  if (qk == kDevice && ok == kDevice) {
    GI_CUDA(launch_point(idx, c, queries, m, out_rowids, idx->stream), "point lookup");
    return GI_OK;
  }
  // host memory: pipelined chunks on three internal streams
  const uint64_t chunk = std::min<uint64_t>(m, 1ull << 22);
  int rc = ensure_staging(idx, chunk);
  if (rc != GI_OK) return rc;
  GiStaging* st = idx->stage;
  GI_CUDA(cudaEventRecord(st->ev, idx->stream), "staging event");
  for (int i = 0; i < 3; ++i) GI_CUDA(cudaStreamWaitEvent(st->st[i], st->ev, 0), "staging wait");
  const int kb = idx->key_bytes;
  uint64_t ci = 0;
  for (uint64_t off = 0; off < m; off += chunk, ++ci) {
    const uint64_t len = std::min<uint64_t>(chunk, m - off);
    const int b = (int)(ci % 3);
    cudaStream_t s = st->st[b];
    const void* qd = (const char*)queries + off * kb;
    if (qk == kHost) {
      GI_CUDA(cudaMemcpyAsync(st->q[b], qd, len * kb, cudaMemcpyHostToDevice, s), "copying probes");
      qd = st->q[b];
    }
    uint32_t* od = ok == kHost ? st->out[b] : out_rowids + off;
    GI_CUDA(launch_point(idx, c, qd, len, od, s), "point lookup");
    if (ok == kHost)
      GI_CUDA(cudaMemcpyAsync(out_rowids + off, od, len * 4, cudaMemcpyDeviceToHost, s), "copying results");
  }
  for (int i = 0; i < 3; ++i) GI_CUDA(cudaStreamSynchronize(st->st[i]), "point lookup");
  rc = read_flags(idx);
  if (rc != GI_OK) return rc;
  return check_latched(idx);
}

int gi_range_lookup(const gi_index* cidx, const void* lo, const void* hi, uint64_t m,
                    uint64_t* out_offsets, uint32_t* out_rowids) {
  t_err.clear();
  gi_index* idx = const_cast<gi_index*>(cidx);
  if (!idx) return fail(GI_ERR_INVALID, "gi_range_lookup: NULL index");
  if (!out_offsets) return fail(GI_ERR_INVALID, "gi_range_lookup: NULL out_offsets");
  if (m > 0 && (!lo || !hi)) return fail(GI_ERR_INVALID, "gi_range_lookup: NULL bounds");
  DeviceScope ds(idx->device);
  const gi::LookupCfg c = resolve_cfg(idx);
  const int kb = idx->key_bytes;
  cudaStream_t s = idx->stream;
  const int dv = idx->device;
  const PtrKind lk = m ? pointer_kind(lo, dv) : kDevice, hk = m ? pointer_kind(hi, dv) : kDevice;
  const PtrKind ofk = pointer_kind(out_offsets, dv);
  const PtrKind rk = out_rowids ? pointer_kind(out_rowids, dv) : kDevice;
  if (lk == kBad || hk == kBad || ofk == kBad || rk == kBad)
    return fail(GI_ERR_INVALID, "gi_range_lookup: a buffer is device memory of another device");
  auto run = [&](const void* dlo, const void* dhi, uint64_t* doff, uint32_t* drows,
                 bool ready) -> cudaError_t {
    if (kb == 4)
      return gi::range_lookup_u32(idx->keys, idx->rows, idx->geom, c, dlo, dhi, m, doff, drows,
                                  idx->rscratch, ready, s);
    return gi::range_lookup_u64(idx->keys, idx->rows, idx->geom, c, dlo, dhi, m, doff, drows,
                                idx->rscratch, ready, s);
  };
  int rc = ensure_range_scratch(idx, m);
  if (rc != GI_OK) return rc;
  if (lk == kDevice && hk == kDevice && ofk == kDevice && rk == kDevice) {
    const bool ready = out_rowids && idx->counts_valid && idx->last_lo == lo &&
                       idx->last_hi == hi && idx->last_m == m && idx->last_off == out_offsets;
    GI_CUDA(run(lo, hi, out_offsets, out_rowids, ready), "range lookup");
    idx->counts_valid = out_rowids == nullptr;
    idx->last_lo = lo;
    idx->last_hi = hi;
    idx->last_m = m;
    idx->last_off = out_offsets;
    return GI_OK;
  }
  // host memory somewhere: stage everything through temporary device buffers
  idx->counts_valid = false;
  void *dlo = nullptr, *dhi = nullptr;
  uint64_t* doff = nullptr;
  uint32_t* drows = nullptr;
  auto cleanup = [&]() {
    if (idx->stage)  // copies of a pipelined fill may still read the staged rows
      for (int i = 0; i < 3; ++i) cudaStreamSynchronize(idx->stage->st[i]);
    if (lk == kHost) dfree(dlo, s);
    if (hk == kHost) dfree(dhi, s);
    if (ofk == kHost) dfree(doff, s);
    if (out_rowids && rk == kHost) dfree(drows, s);
    cudaStreamSynchronize(s);
  };
  auto stage_fail = [&](cudaError_t e, const char* what) {
    cleanup();
    return cuda_fail(e, what);
  };
#define GI_TRY3(call, what)                          \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return stage_fail(e_, what); \
  } while (0)
  const size_t bb = (m ? m : 1) * kb;
  if (lk == kHost) {
    GI_TRY3(dalloc(&dlo, bb, s), "staging");
    GI_TRY3(cudaMemcpyAsync(dlo, lo, m * kb, cudaMemcpyHostToDevice, s), "copying bounds");
  } else {
    dlo = const_cast<void*>(lo);
  }
  if (hk == kHost) {
    GI_TRY3(dalloc(&dhi, bb, s), "staging");
    GI_TRY3(cudaMemcpyAsync(dhi, hi, m * kb, cudaMemcpyHostToDevice, s), "copying bounds");
  } else {
    dhi = const_cast<void*>(hi);
  }
  if (ofk == kHost) {
    GI_TRY3(dalloc((void**)&doff, (m + 1) * 8, s), "staging");
  } else {
    doff = out_offsets;
  }
  GI_TRY3(run(dlo, dhi, doff, nullptr, false), "range lookup");
  if (out_rowids) {
    uint64_t total = 0;
    GI_TRY3(cudaMemcpyAsync(&total, doff + m, 8, cudaMemcpyDeviceToHost, s), "reading total");
    GI_TRY3(cudaStreamSynchronize(s), "range lookup");
    if (rk == kHost) {
      GI_TRY3(dalloc((void**)&drows, (total ? total : 1) * 4, s), "staging");
    } else {
      drows = out_rowids;
    }
    constexpr int kChunks = 8;  // fill chunk c while chunk c-1's rows go to the host
    if (rk == kHost && total >= (1ull << 22) && m >= (uint64_t)kChunks) {
      rc = ensure_staging(idx, std::min<uint64_t>(m, 1ull << 22));
      if (rc != GI_OK) {
        cleanup();
        return rc;
      }
      GiStaging* st = idx->stage;
      uint64_t first[kChunks + 1], row0[kChunks + 1];
      for (int i = 0; i <= kChunks; ++i) first[i] = m * i / kChunks;
      for (int i = 0; i < kChunks; ++i)  // each chunk's first row
        GI_TRY3(cudaMemcpyAsync(&row0[i], doff + first[i], 8, cudaMemcpyDeviceToHost, s), "reading offsets");
      GI_TRY3(cudaStreamSynchronize(s), "range lookup");
      row0[kChunks] = total;
      const uint64_t* lo_rank = (const uint64_t*)idx->rscratch;
      for (int i = 0; i < kChunks; ++i) {
        GI_TRY3(gi::range_fill_rows(idx->rows, idx->geom, c, doff + first[i], lo_rank + first[i],
                                    first[i + 1] - first[i], drows, s), "range fill");
        GI_TRY3(cudaEventRecord(st->cev[i], s), "staging event");
        cudaStream_t cs = st->st[i % 3];
        GI_TRY3(cudaStreamWaitEvent(cs, st->cev[i], 0), "staging wait");
        if (row0[i + 1] > row0[i])
          GI_TRY3(cudaMemcpyAsync(out_rowids + row0[i], drows + row0[i], (row0[i + 1] - row0[i]) * 4,
                                  cudaMemcpyDeviceToHost, cs), "copying rows");
      }
      for (int i = 0; i < 3; ++i) GI_TRY3(cudaStreamSynchronize(st->st[i]), "copying rows");
    } else {
      GI_TRY3(run(dlo, dhi, doff, drows, true), "range fill");
      if (rk == kHost && total)
        GI_TRY3(cudaMemcpyAsync(out_rowids, drows, total * 4, cudaMemcpyDeviceToHost, s), "copying rows");
    }
  }
  if (ofk == kHost)
    GI_TRY3(cudaMemcpyAsync(out_offsets, doff, (m + 1) * 8, cudaMemcpyDeviceToHost, s), "copying offsets");
  cleanup();
  GI_CUDA(cudaGetLastError(), "range lookup");
  rc = read_flags(idx);
  if (rc != GI_OK) return rc;
  return check_latched(idx);
#undef GI_TRY3
}

int gi_sync(gi_index* idx) {
  t_err.clear();
  if (!idx) return fail(GI_ERR_INVALID, "gi_sync: NULL index");
  DeviceScope ds(idx->device);
  int rc = read_flags(idx);
  if (rc != GI_OK) return rc;
  return check_latched(idx);
}

uint64_t gi_footprint_bytes(const gi_index* idx) {
  if (!idx) return 0;
  return idx->n * (uint64_t)(idx->key_bytes + 4) + (idx->layout == GI_EYTZINGER ? idx->key_bytes : 0);
}

int gi_get_info(const gi_index* idx, gi_info* out) {
  t_err.clear();
  if (!idx || !out) return fail(GI_ERR_INVALID, "gi_get_info: NULL argument");
  memset(out, 0, sizeof *out);
  out->n = idx->n;
  out->layout = idx->layout;
  out->k = idx->k;
  out->key_bytes = idx->key_bytes;
  out->unique = idx->unique ? 1 : 0;
  if (idx->layout == GI_SORTED) {
    uint32_t l = 0;
    while (l < 64 && (1ull << l) <= idx->n) ++l;
    out->levels = l;
  } else {
    out->levels = idx->geom.levels;
  }
  out->keys = idx->keys;
  out->rowids = idx->rows;
  out->footprint_bytes = gi_footprint_bytes(idx);
  return GI_OK;
}

int gi_copy_layout(const gi_index* cidx, void* keys_out, uint32_t* rowids_out) {
  t_err.clear();
  gi_index* idx = const_cast<gi_index*>(cidx);
  if (!idx) return fail(GI_ERR_INVALID, "gi_copy_layout: NULL index");
  DeviceScope ds(idx->device);
  const char* src = (const char*)idx->keys + (idx->layout == GI_EYTZINGER ? idx->key_bytes : 0);
  if (keys_out && idx->n)
    GI_CUDA(cudaMemcpyAsync(keys_out, src, idx->n * idx->key_bytes, cudaMemcpyDefault, idx->stream),
            "copying keys");
  if (rowids_out && idx->n)
    GI_CUDA(cudaMemcpyAsync(rowids_out, idx->rows, idx->n * 4, cudaMemcpyDefault, idx->stream),
            "copying rowids");
  GI_CUDA(cudaStreamSynchronize(idx->stream), "gi_copy_layout");
  return GI_OK;
}

int gi_set_option(gi_index* idx, int option, int64_t v) {
  t_err.clear();
  if (!idx) return fail(GI_ERR_INVALID, "gi_set_option: NULL index");
  if (option < 1 || option > 10) return fail(GI_ERR_INVALID, "gi_set_option: unknown option %d", option);
  if (v == -1) {
    idx->opt[option] = -1;
    return GI_OK;
  }
  switch (option) {
    case GI_OPT_GROUP:
      if (idx->layout != GI_EYTZINGER_KARY || !gi::eks_group_supported(idx->k, idx->key_bytes, (int)v))
        return fail(GI_ERR_INVALID, "gi_set_option: group %lld not available for this index", (long long)v);
      break;
    case GI_OPT_PER_THREAD:
      if (v != 1 && v != 2 && v != 4) return fail(GI_ERR_INVALID, "gi_set_option: per-thread must be 1, 2 or 4");
      break;
    case GI_OPT_SMEM_LEVELS: {
      if (v < 0 || v > 40) return fail(GI_ERR_INVALID, "gi_set_option: smem levels out of range");
      DeviceScope ds(idx->device);
      const uint64_t slots = gi::smem_slots_for_levels(idx->layout, idx->geom, (int)v, idx->key_bytes);
      const uint64_t bytes = (slots * idx->key_bytes + 15) & ~15ull;
      if (bytes > (uint64_t)gi::device_max_smem_optin() - 1024)
        return fail(GI_ERR_INVALID, "gi_set_option: %lld levels need %llu bytes of shared memory",
                    (long long)v, (unsigned long long)bytes);
      break;
    }
    case GI_OPT_BLOCK:
      if (v != 64 && v != 128 && v != 256 && v != 512)
        return fail(GI_ERR_INVALID, "gi_set_option: block must be 64, 128, 256 or 512");
      break;
    case GI_OPT_BLOCKS_PER_SM:
      if (v < 0 || v > 32) return fail(GI_ERR_INVALID, "gi_set_option: blocks per SM out of range");
      break;
    case GI_OPT_PREFETCH:
      if (v != 0 && v != 2 && v != 3 && v != 4) return fail(GI_ERR_INVALID, "gi_set_option: prefetch must be 0, 2, 3 or 4");
      break;
    case GI_OPT_EARLY_EXIT:
      if (v != 0 && v != 1) return fail(GI_ERR_INVALID, "gi_set_option: early exit must be 0 or 1");
      break;
    case GI_OPT_HOT_LEVELS:
      if (v < 0 || v > 64) return fail(GI_ERR_INVALID, "gi_set_option: hot levels out of range");
      break;
    case GI_OPT_RANGE_FILL:
      if (v != 0 && v != 1) return fail(GI_ERR_INVALID, "gi_set_option: range fill must be 0 or 1");
      break;
    case GI_OPT_REORDER:
      if (v != 0 && v != 1) return fail(GI_ERR_INVALID, "gi_set_option: reorder must be 0 or 1");
      break;
  }
  idx->opt[option] = v;
  return GI_OK;
}

int gi_get_option(const gi_index* idx, int option, int64_t* v) {
  t_err.clear();
  if (!idx || !v) return fail(GI_ERR_INVALID, "gi_get_option: NULL argument");
  if (option < 1 || option > 10) return fail(GI_ERR_INVALID, "gi_get_option: unknown option %d", option);
  const gi::LookupCfg c = resolve_cfg(idx);
  switch (option) {
    case GI_OPT_GROUP: *v = c.group; break;
    case GI_OPT_PER_THREAD: *v = c.per_thread; break;
    case GI_OPT_SMEM_LEVELS: *v = c.smem_levels; break;
    case GI_OPT_BLOCK: *v = c.block; break;
    case GI_OPT_BLOCKS_PER_SM: *v = c.blocks_per_sm; break;
    case GI_OPT_PREFETCH: *v = c.prefetch; break;
    case GI_OPT_EARLY_EXIT: *v = c.early_exit; break;
    case GI_OPT_HOT_LEVELS: *v = c.hot_levels; break;
    case GI_OPT_RANGE_FILL: *v = c.range_fill; break;
    case GI_OPT_REORDER: *v = c.reorder; break;
  }
  return GI_OK;
}

int gi_probe_random_sectors(const void* buf, uint64_t bytes, uint32_t chunk_bytes, uint64_t loads,
                            uint64_t seed, uint64_t* sink, void* stream) {
  t_err.clear();
  if (!buf || !sink) return fail(GI_ERR_INVALID, "gi_probe_random_sectors: NULL pointer");
  if (chunk_bytes != 16 && chunk_bytes != 32 && chunk_bytes != 64 && chunk_bytes != 128 &&
      chunk_bytes != 256)
    return fail(GI_ERR_INVALID, "gi_probe_random_sectors: chunk must be 16..256 bytes, a power of two");
  if (((uintptr_t)buf & 255) || bytes < chunk_bytes)
    return fail(GI_ERR_INVALID, "gi_probe_random_sectors: buffer must be 256-byte aligned and hold a chunk");
  int dev = 0;
  cudaGetDevice(&dev);
  if (pointer_kind(buf, dev) != kDevice || pointer_kind(sink, dev) != kDevice)
    return fail(GI_ERR_INVALID, "gi_probe_random_sectors: buffers must be device memory of the current device");
  GI_CUDA(gi::probe_random_sectors(buf, bytes, chunk_bytes, loads, seed, sink, (cudaStream_t)stream),
          "probe");
  return GI_OK;
}

int gi_coalescing_probe(const uint32_t* buf, uint64_t entries, uint32_t threads, uint32_t group,
                        uint32_t steps, uint64_t seed, uint64_t* sink, void* stream) {
  t_err.clear();
  if (!buf || !sink) return fail(GI_ERR_INVALID, "gi_coalescing_probe: NULL pointer");
  if (group == 0 || group > threads || group > entries || threads == 0)
    return fail(GI_ERR_INVALID, "gi_coalescing_probe: need 0 < group <= threads, group <= entries");
  int dev = 0;
  cudaGetDevice(&dev);
  if (pointer_kind(buf, dev) != kDevice || pointer_kind(sink, dev) != kDevice)
    return fail(GI_ERR_INVALID, "gi_coalescing_probe: buffers must be device memory of the current device");
  GI_CUDA(gi::coalescing_probe(buf, entries, threads, group, steps, seed, sink, (cudaStream_t)stream),
          "probe");
  return GI_OK;
}

}  // extern "C"

// ================================================================= allocation-free range lookups
// For callers that cannot allocate device memory (see gi_range_lookup_noalloc in
// gi.h).  The scratch of the range lookup lives in this file-scope device array;
// host code only ever passes the device address looked up below, never the
// array's name (which in host code is a host-side stand-in, not device memory).
static __device__ __align__(256) unsigned char g_noalloc_scratch[GI_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
struct NoAllocAddr {
  void* ptr = nullptr;
  unsigned long long ctx = 0;  // id of the context the address belongs to
};
NoAllocAddr g_noalloc_addr[kNoAllocMaxDevices];

// Id of the calling thread's current CUDA context, unique for the life of the
// process (a context made after cudaDeviceReset gets a new one); 0 if unknown.
// Taken through the driver entry points the runtime hands out, so the library
// needs no link against the driver library.
unsigned long long current_context_id() {
  using GetCurrent = int (*)(void**);
  using GetId = int (*)(void*, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = (GetCurrent)f;
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (GetId)f;
    cudaGetLastError();
  });
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

// Device address of the scratch array on `dev` (which must be current).  It is
// looked up once per device and context: after a context change (for example a
// cudaDeviceReset in the caller's process) the module, and with it the array, is
// loaded anew at another address, which is looked up again.  The lookup may load
// the module, which a stream capture in progress must not see: it is refused
// while `s` is capturing.
int noalloc_scratch(int dev, cudaStream_t s, void** out) {
  if (dev < 0 || dev >= kNoAllocMaxDevices)
    return fail(GI_ERR_INVALID, "gi_range_lookup_noalloc: device %d out of range", dev);
  const unsigned long long ctx = current_context_id();
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  NoAllocAddr& a = g_noalloc_addr[dev];
  if (!a.ptr || ctx == 0 || a.ctx != ctx) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
      cudaGetLastError();
      return fail(GI_ERR_INVALID,
                  "gi_range_lookup_noalloc: the first call on a device (or after a context "
                  "change) looks up the scratch address and must not run during stream "
                  "capture; make one call before capturing");
    }
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e != cudaSuccess ? e : cudaErrorUnknown,
                                                 "gi_range_lookup_noalloc: scratch address");
    a.ptr = p;
    a.ctx = ctx;
  }
  *out = a.ptr;
  return GI_OK;
}
}  // namespace

extern "C" int gi_range_lookup_noalloc(const gi_index* idx, const void* lo, const void* hi,
                                       uint64_t m, uint64_t* out_offsets, uint32_t* out_rowids) {
  t_err.clear();
  if (!idx) return fail(GI_ERR_INVALID, "gi_range_lookup_noalloc: NULL index");
  if (!out_offsets) return fail(GI_ERR_INVALID, "gi_range_lookup_noalloc: NULL out_offsets");
  if (m > GI_NOALLOC_MAX_RANGES)
    return fail(GI_ERR_INVALID, "gi_range_lookup_noalloc: %llu ranges exceed the maximum of %u",
                (unsigned long long)m, (unsigned)GI_NOALLOC_MAX_RANGES);
  if (m > 0 && (!lo || !hi)) return fail(GI_ERR_INVALID, "gi_range_lookup_noalloc: NULL bounds");
  if (gi::range_scratch_bytes(m) > GI_NOALLOC_SCRATCH_BYTES)
    return fail(GI_ERR_INVALID, "gi_range_lookup_noalloc: scratch too small for %llu ranges",
                (unsigned long long)m);
  DeviceScope ds(idx->device);
  const int dv = idx->device;
  if ((m && (pointer_kind(lo, dv) != kDevice || pointer_kind(hi, dv) != kDevice)) ||
      pointer_kind(out_offsets, dv) != kDevice ||
      (out_rowids && pointer_kind(out_rowids, dv) != kDevice))
    return fail(GI_ERR_INVALID,
                "gi_range_lookup_noalloc: every buffer must be device memory of the index's device");
  void* scratch = nullptr;
  int rc = noalloc_scratch(idx->device, idx->stream, &scratch);
  if (rc != GI_OK) return rc;
  // this call writes out_offsets and its own lower ranks, not the index's: a later
  // gi_range_lookup must not take the two-call shortcut on counts from before
  const_cast<gi_index*>(idx)->counts_valid = false;
  const gi::LookupCfg c = resolve_cfg(idx);
  // counts_ready = false: another call may have overwritten the shared scratch
  cudaError_t e = idx->key_bytes == 4
      ? gi::range_lookup_u32(idx->keys, idx->rows, idx->geom, c, lo, hi, m, out_offsets,
                             out_rowids, scratch, false, idx->stream)
      : gi::range_lookup_u64(idx->keys, idx->rows, idx->geom, c, lo, hi, m, out_offsets,
                             out_rowids, scratch, false, idx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "gi_range_lookup_noalloc");
  return GI_OK;
}

