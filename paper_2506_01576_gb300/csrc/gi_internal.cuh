// Internal declarations shared by the CUDA translation units of libgi.
//
// Index geometry and the two closed-form maps between a slot of the
// (k-ary) Eytzinger array and the rank (sorted position) of the key it holds:
//   slot -> rank : p'(t) of Section 6.1 (k = 2: Section 4), read with the bottom
//                  level at t >= k^m - 1 and the level of slot t as
//                  floor(log_k(t + 1));
//   rank -> slot : its inverse, derived from the same level structure.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gi.h"

namespace gi {

// ---------------------------------------------------------------- device status bits
enum : uint32_t {
  kFlagReservedRowid = 1u << 0,  // an input rowID equals GI_MISS
  kFlagDuplicate = 1u << 1,      // two equal keys were found (index not unique)
  kFlagTimeout = 1u << 2,        // a bounded spin gave up
};

// Spin limit for every device-side wait (each iteration sleeps ~100 ns or more).
constexpr uint32_t kSpinLimit = 1u << 22;

// ---------------------------------------------------------------- geometry
struct Geom {
  uint64_t n;          // keys
  uint64_t top;        // k^m - 1: keys in the full levels 0..m-1
  uint64_t b;          // n - top: keys in the (partial) bottom level m, 1 <= b
  uint32_t k;          // fan-out (2 = Eytzinger)
  uint32_t m;          // floor(log_k n)
  uint32_t levels;     // m + 1 for n >= 1, 0 for n == 0
  uint32_t log2k;      // log2(k) if k is a power of two, else 0
};

Geom make_geom(uint64_t n, uint32_t k);  // host

__host__ __device__ constexpr uint32_t ilog2_const(uint32_t v) {
  return v <= 1 ? 0 : 1 + ilog2_const(v >> 1);
}

// k^e (e small; the caller guarantees no overflow)
template <int KF>
__host__ __device__ __forceinline__ uint64_t kpow(uint32_t e, const Geom& g) {
  const uint32_t k = KF ? KF : g.k;
  if ((k & (k - 1)) == 0) return 1ull << (e * (KF ? ilog2_const(KF) : g.log2k));
  uint64_t p = 1;
  for (uint32_t i = 0; i < e; ++i) p *= k;
  return p;
}

// floor(log_k(x)) for 1 <= x
template <int KF>
__host__ __device__ __forceinline__ uint32_t floor_log_k(uint64_t x, const Geom& g) {
  const uint32_t k = KF ? KF : g.k;
  if ((k & (k - 1)) == 0) {
    const uint32_t s = KF ? ilog2_const(KF) : g.log2k;
#ifdef __CUDA_ARCH__
    const uint32_t lg = 63 - __clzll((long long)x);
#else
    const uint32_t lg = 63 - __builtin_clzll(x);
#endif
    return lg / s;
  }
  uint32_t l = 0;
  uint64_t p = k;
  while (p <= x) {
    ++l;
    if (p > x / k) break;
    p *= k;
  }
  return l;
}

// Slot t (0-based) -> rank of the key it holds (Section 6.1, Section 4 for k = 2).
template <int KF>
__host__ __device__ __forceinline__ uint64_t slot_to_rank(uint64_t t, const Geom& g) {
  const uint64_t k = KF ? (uint64_t)KF : (uint64_t)g.k;
  const uint64_t km1 = k - 1;
  if (t >= g.top) {  // bottom level: node-major, one rank skipped after each node
    const uint64_t i = t - g.top;
    return i + i / km1;
  }
  const uint32_t l = floor_log_k<KF>(t + 1, g);
  const uint64_t i = t - (kpow<KF>(l, g) - 1);
  const uint64_t p = kpow<KF>(g.m - l - 1, g) * (1 + i + i / km1) - 1;  // rank in the perfect tree
  const uint64_t corr = km1 * (p + 1);                                   // bottom keys to its left
  return p + (g.b < corr ? g.b : corr);
}

// Rank r -> slot holding it (inverse of slot_to_rank).
template <int KF>
__host__ __device__ __forceinline__ uint64_t rank_to_slot(uint64_t r, const Geom& g) {
  const uint64_t k = KF ? (uint64_t)KF : (uint64_t)g.k;
  const uint64_t km1 = k - 1;
  const uint64_t c = r / k, o = r - c * k;
  if (o < km1 && c * km1 + o < g.b) return g.top + c * km1 + o;  // bottom-level key
  const uint64_t below = c * km1 + o;
  const uint64_t q = r - (g.b < below ? g.b : below);  // rank among the upper-level keys
  uint64_t x = q + 1;
  uint32_t z = 0;
  while (x % k == 0) {
    x /= k;
    ++z;
  }
  const uint32_t l = g.m - 1 - z;
  const uint64_t xd = x / k;
  return (kpow<KF>(l, g) - 1) + xd * km1 + (x - xd * k) - 1;
}

// The rank -> slot map of the k-ary layout (rank_to_slot) in 32-bit arithmetic,
// valid because n < 2^32 (rowIDs are 32-bit), with the first slot of every level
// (k^l - 1) from a table instead of a power loop.  A rank with remainder o < k-1
// mod k is a bottom-level key while the bottom level lasts; every other rank is
// an upper-level key of the perfect tree, whose level is m-1 minus the number of
// factors k in its 1-based rank among the upper-level keys.
struct SlotMap {
  uint32_t top, b, m, k;
  uint32_t first[32];  // first slot of level l, l <= m
};

template <int KF>
__host__ __device__ __forceinline__ uint32_t slot_of_rank(uint32_t r, const SlotMap& sm) {
  const uint32_t k = KF ? (uint32_t)KF : sm.k, km1 = k - 1;
  const uint32_t c = r / k, o = r - c * k;
  const uint32_t below = c * km1 + o;  // bottom-level keys of smaller rank, if unbounded
  if (o < km1 && below < sm.b) return sm.top + below;
  uint32_t x = r - (below < sm.b ? below : sm.b) + 1;
  uint32_t l = sm.m - 1;
  while (x % k == 0) {
    x /= k;
    --l;
  }
  const uint32_t xd = x / k;
  return sm.first[l] + xd * km1 + (x - xd * k) - 1;
}

// The same map for a fan-out chosen per index (batches whose indexes each have
// their own k): sm.k == 0 marks the sorted layout (slot = rank); the compiled
// fan-outs take their constant-divisor forms.  sm.k is uniform over a bucket, so
// the switch does not diverge.
__host__ __device__ __forceinline__ uint32_t slot_of_rank_any(uint32_t r, const SlotMap& sm) {
  switch (sm.k) {
    case 0: return r;
    case 2: return slot_of_rank<2>(r, sm);
    case 3: return slot_of_rank<3>(r, sm);
    case 5: return slot_of_rank<5>(r, sm);
    case 9: return slot_of_rank<9>(r, sm);
    case 17: return slot_of_rank<17>(r, sm);
    default: return slot_of_rank<0>(r, sm);
  }
}

// The 32-bit map of a geometry with n < 2^32 (host or device; on the device
// fill_slot_map can write straight into shared memory).
__host__ __device__ inline void fill_slot_map(SlotMap& sm, const Geom& g) {
  sm.top = (uint32_t)g.top;
  sm.b = (uint32_t)g.b;
  sm.m = g.m;
  sm.k = g.k;
  uint64_t p = 1;
  for (uint32_t l = 0; l < 32 && l <= g.m; ++l, p *= g.k) sm.first[l] = (uint32_t)(p - 1);
}
inline SlotMap make_slot_map(const Geom& g) {
  SlotMap sm{};
  fill_slot_map(sm, g);
  return sm;
}

// Geometry computed on the device (the host version is make_geom); k >= 2.
__device__ __forceinline__ Geom device_geom(uint64_t n, uint32_t k) {
  Geom g;
  g.n = n;
  g.k = k;
  g.log2k = ((k & (k - 1)) == 0) ? (31 - __clz(k)) : 0;
  g.m = 0;
  g.top = 0;
  g.b = n;
  g.levels = n ? 1 : 0;
  if (n) {
    uint64_t p = 1;
    uint32_t m = 0;
    while (p <= n / k) {
      p *= k;
      ++m;
    }
    g.m = m;
    g.top = p - 1;
    g.b = n - g.top;
    g.levels = m + 1;
  }
  return g;
}

// ---------------------------------------------------------------- launch bookkeeping
void count_launch(uint64_t n = 1);
// accessors for the autotuner (gi_tune.cu)
cudaStream_t index_stream(const gi_index* idx);
int index_device(const gi_index* idx);
int batch_device(const gi_batch* b);
int64_t index_raw_option(const gi_index* idx, int option);  // -1: automatic
cudaStream_t batch_stream(const gi_batch* b);
int64_t batch_option(const gi_batch* b, int option);
// the autotuner's recorded options for (key bytes, layout, k, floor(log2 n)); false if none
bool tune_table_lookup(int key_bytes, int layout, uint32_t k, uint64_t n, int64_t* opt);
void set_last_error(const char* msg);  // the thread's gi_last_error() text
int sm_count();
int device_max_smem_optin();

// ---------------------------------------------------------------- kernel entry points (host side)
// Radix sort + layout (gi_sort.cu).  Returns cudaError_t.
struct SortBuffers {
  void* keys[2];
  uint32_t* vals[2];
  void* scratch;          // histogram + status + counters
  size_t scratch_bytes;
};
size_t sort_scratch_bytes(uint64_t n, int key_bytes);
// Histogram all digits and scan them on the device, then copy the per-digit
// "one value only" flags to host_trivial[key_bytes] (page-locked; valid once the
// stream gets there: no synchronisation inside).  copy_to != NULL: `keys` is
// page-locked host memory, copied to copy_to by the same pass.
// host_win != NULL (the hybrid sort may follow): instead no digit counts (see
// sort_counts), but the counts of the 8-bit window just below the highest bit in
// which two keys differ, into host_win[2..257], with host_win[0] = the OR of
// key ^ keys[0] (its zero bytes are the trivial digits) and host_win[1] = window
// shift | (1 if one value only) << 32 (page-locked, 258 words); min_bytes: with
// fewer differing key bytes the window is marked trivial (the hybrid sort does not
// apply, and the window pass skips).
cudaError_t sort_prepare(const void* keys, void* copy_to, uint64_t n, int key_bytes,
                         void* scratch, cudaStream_t s, uint32_t* host_trivial,
                         unsigned long long* host_win, uint32_t min_bytes);
// The digit counts and offsets the LSD passes use, after a sort_prepare with
// host_win (`keys`: any permutation of the input, on the device).
cudaError_t sort_counts(const void* keys, uint64_t n, int key_bytes, void* scratch, cudaStream_t s);
// The stable MSD scatter on that window (after sort_prepare with host_win; its
// shift and offsets are read on the device, so it can be queued before the host
// has seen them), reading the input rowIDs (checked for the reserved value).
// Skipped on the device if every key has the same window value.
cudaError_t sort_window_pass(const void* src_k, const uint32_t* src_v, void* dst_k, uint32_t* dst_v,
                             uint64_t n, int key_bytes, void* scratch, uint32_t* dflags,
                             cudaStream_t s);
// Tile tickets back to zero (before LSD passes that follow an MSD pass).
cudaError_t sort_reset_counters(void* scratch, int key_bytes, cudaStream_t s);
// check_rows: this pass reads the caller's rowIDs; flag any equal to GI_MISS.
cudaError_t sort_pass(const void* src_k, const uint32_t* src_v, void* dst_k, uint32_t* dst_v,
                      uint64_t n, int key_bytes, int pass, void* scratch, uint32_t* dflags,
                      bool check_rows, cudaStream_t s);
cudaError_t check_rowids(const uint32_t* rows, uint64_t n, uint32_t* dflags, cudaStream_t s);
cudaError_t layout_gather(const void* sk, const uint32_t* sv, void* dk, uint32_t* dv,
                          const Geom& g, int key_bytes, uint32_t key_off, uint32_t* dflags,
                          cudaStream_t s);
cudaError_t check_sorted_dups(const void* sk, uint64_t n, int key_bytes, uint32_t* dflags,
                              cudaStream_t s);

// Batched build of many independent indexes (gi_sort.cu).  Inputs are the
// concatenation of all indexes' pairs; seg_start[s] .. seg_start[s+1] is index s.
struct BatchTile {
  uint64_t start;   // first element (global position in the concatenated input)
  uint32_t seg;     // index the tile belongs to
  uint32_t count;   // elements in the tile
  uint32_t local;   // tile number within its index
  uint32_t pad;
};
constexpr uint32_t kBatchChunk = 65536;  // elements per histogram work item
uint32_t batch_sort_tile(int key_bytes);  // elements per radix tile
size_t batch_sort_scratch_bytes(uint64_t ntiles, uint32_t nseg, int key_bytes);

// How one index of a batch is sorted; written on the device from its digit
// histograms, so the whole build stays free of host round trips.
enum : uint32_t {
  kPlanEmpty = 0,  // no keys
  kPlanWhole = 1,  // at most local_sort_capacity() pairs: one CTA sorts the index
  kPlanMsd = 2,    // one stable scatter on its top 8 significant bits, then buckets
  kPlanLsd = 3,    // a bucket would be too large: the segmented LSD passes
};
struct BatchPlan {
  uint32_t mode;
  uint32_t s1;        // shift of the MSD window (kPlanMsd)
  uint32_t ts;        // shift of the bucket sort's top window
  uint32_t lsd_mask;  // bytes that differ between the index's keys
};
// Device tables of the hybrid batch build (allocated with the batch).
struct BatchHybrid {
  BatchPlan* plan;              // [nseg]
  SlotMap* slot_maps;           // [nseg] (k-ary layouts)
  unsigned long long* hist_w;   // [nseg][256] counts of the MSD window
  unsigned long long* offs_w;   // [nseg][256] their absolute starts
  uint32_t* counter;            // tile tickets of the MSD pass
  void* out_k;                  // the batch's padded key / rowID arrays
  uint32_t* out_v;
  const uint64_t* seg_base;     // slot 0 of every index in out_k / out_v
  const uint32_t* tile0;        // [nseg + 1] first radix tile of every index
  uint32_t* prefix_msd;         // [nseg + 1] tiles of the kPlanMsd indexes before index s
  uint32_t* prefix_lsd;         // [nseg + 1] same for kPlanLsd
  uint32_t* list_msd;           // [ntiles] tiles of the kPlanMsd indexes, in order
  uint32_t* list_lsd;           // [ntiles] tiles of the kPlanLsd indexes, in order
  uint32_t* buckets;            // [3][nseg * 257] bucket ids per bucket-sort size class
  uint32_t* bucket_count;       // [3]
  unsigned long long* xor_or;   // [nseg] OR over the index of key ^ (its first key)
  uint32_t k;                   // fan-out; 0 = sorted layout; kBatchMixed: kidx
  const uint32_t* kidx;         // [nseg] fan-out of every index (0 = sorted), if mixed
};
// BatchHybrid::k of a batch whose indexes each have their own fan-out
constexpr uint32_t kBatchMixed = 0xFFFFFFFFu;
// the fan-outs a batch lays its indexes out with: 0 (sorted), 2, 3, 5, 9, 17
inline bool batch_fanout_ok(uint32_t k) { return k == 0 || k == 2 || k == 3 || k == 5 || k == 9 || k == 17; }
size_t batch_hybrid_bytes(uint32_t nseg, uint64_t ntiles);  // device bytes of the tables
// hist/offsets/status/counters live in `scratch` (batch_sort_scratch_bytes); no host
// sync.  hy != NULL: indexes are sorted per their plan (whole / MSD + buckets, written
// straight into hy->out_k / out_v), and only kPlanLsd indexes take the LSD passes
// (their result then needs batch_gather with the same plan).
cudaError_t batch_sort(const void* keys, const uint32_t* vals, void* tmp_k[2], uint32_t* tmp_v[2],
                       uint64_t n, int key_bytes, const uint64_t* seg_start, uint32_t nseg,
                       const BatchTile* tiles, uint64_t ntiles, const BatchTile* chunks,
                       uint64_t nchunks, void* scratch, uint32_t* dflags, cudaStream_t s,
                       int* result_buf, const BatchHybrid* hy);
// The bucket sort of a batch: every index of plan kPlanWhole, and every MSD bucket
// of the kPlanMsd indexes (in src_k / src_v after the MSD pass).
cudaError_t batch_local_sort(const void* keys, const uint32_t* vals, const void* src_k,
                             const uint32_t* src_v, const uint64_t* seg_start, uint32_t nseg,
                             int key_bytes, const BatchHybrid& hy, uint32_t* dflags,
                             cudaStream_t s);
// Raises the bucket-sort kernels' shared-memory limit (once, before any capture).
cudaError_t batch_local_sort_setup(int key_bytes, uint32_t k);
// hy != NULL: only the tiles of the kPlanLsd indexes (of nseg)
// permute every index into k-ary order (k = 0: sorted; kBatchMixed: hy->kidx) at
// out + seg_base[s]
cudaError_t batch_gather(const void* sk, const uint32_t* sv, void* ok, uint32_t* ov,
                         const BatchTile* tiles, uint64_t ntiles, const uint64_t* seg_start,
                         const uint64_t* seg_base, uint32_t k, int key_bytes, uint32_t* dflags,
                         cudaStream_t s, const BatchHybrid* hy, uint32_t nseg);


// Hybrid sort: stable MSD scatter(s) on one or two 8-bit windows just below the
// highest bit in which two keys differ (by default only where it measured
// faster; force = GI_BUILD_HYBRID: wherever it can run), then every bucket
// sorted in shared memory and written straight into the final layout
// (gi_local_sort.cu): slot = rank for the sorted layout, else the k-ary (k = g.k;
// Eytzinger for k = 2, keys shifted by key_off) slot of the rank.
// host_win: sort_prepare's window record (NULL: not applicable).  pass1_done: the
// caller already ran sort_window_pass into bk[first_dst].  host_h2: page-locked
// room for one count.
// *used = true: bk[*result] / bv[*result] hold the finished layout and the
// duplicate flag is set -- unless *verify_src >= 0 and, once the stream is done,
// the count in host_h2 is not zero: then buckets too large for a CTA were left
// out, and bk[*verify_src] holds the data after both MSD scatters, for a full
// LSD sort (the caller resets the pass counters).  *used = false and
// *result = -1: not applicable, nothing launched.  *used = false and
// *result >= 0: bk[*result] holds the data after stable MSD scatter(s) (not
// applicable after a caller's pass 1), for a full LSD sort.
cudaError_t hybrid_sort(const void* src_k, const uint32_t* src_v, void* bk[2], uint32_t* bv[2],
                        int first_dst, uint64_t n, int key_bytes, uint32_t nontrivial,
                        const unsigned long long* host_win, void* scratch, const Geom& g,
                        bool sorted_layout, uint32_t key_off, bool force, bool pass1_done,
                        unsigned long long* host_h2, uint32_t* dflags, cudaStream_t s,
                        int* result, bool* used, int* verify_src);
// The size classes of the single-index bucket sort: the largest bucket each
// takes (the launch table in gi_local_sort.cu checks itself against this list).
constexpr int kLocalClasses = 5;
__host__ __device__ constexpr uint32_t local_class_max(int i) {
  return i == 0 ? 1536u : i == 1 ? 2560u : i == 2 ? 3072u : i == 3 ? 4096u : 5120u;
}
// the class (0..kLocalClasses-1) of a bucket of `count` pairs; kLocalClasses if
// it is too large for any
__host__ __device__ inline int local_sort_class(uint64_t count) {
  int c = 0;
#pragma unroll
  for (int i = 0; i < kLocalClasses; ++i) c += count > local_class_max(i) ? 1 : 0;
  return c;
}
// Shared-memory sort of buckets of at most local_sort_capacity() pairs whose keys
// agree on every bit outside the bytes of lsd_mask and above top_shift + 8: one
// stable split on the 8 bits at top_shift, then count ranking (or, with a large
// sub-bucket, one ballot pass per byte of lsd_mask; single: the split alone
// sorts), written into the layout (see above).
uint32_t local_sort_capacity();
// cls >= 0 runs that size class's kernel (buckets of at most local_class_max(cls)
// pairs), else the class of max_count; nseg_dev != NULL: the number of buckets
// is read on the device (a list written there), nseg is its upper bound.
cudaError_t local_sort(const void* sk, const uint32_t* sv, void* dk, uint32_t* dv,
                       const BatchTile* segs, uint64_t nseg, const uint32_t* nseg_dev,
                       uint64_t max_count, int cls, uint32_t top_shift, uint32_t lsd_mask,
                       bool single, int key_bytes, const Geom& g, bool sorted_layout,
                       uint32_t key_off, uint32_t* dflags, cudaStream_t s);

// Point lookups (gi_point.cu).
struct LookupCfg {
  int layout;         // GI_SORTED / GI_EYTZINGER / GI_EYTZINGER_KARY
  int key_bytes;
  int group;          // lanes per lookup (EKS)
  int per_thread;     // lookups interleaved per thread / group
  int smem_levels;    // top levels staged in shared memory
  int block;          // threads per block
  int blocks_per_sm;  // 0: one thread (group) per work item
  int prefetch;       // EBS prefetch distance
  int early_exit;     // stop on an equal pivot (unique keys only)
  int hot_levels;     // k-ary: top levels kept in L2 (evict_last); the rest streamed
  int l1_levels;      // k-ary: top levels read through L1; deeper ones not allocated there
  int range_fill;     // 0: rows by rank -> slot; 1: rows by per-level runs
  int reorder;        // point lookups: sort each CTA's probe tile first (Section 7.4)
};
// top levels whose keys fit in `budget` bytes
int levels_within(const Geom& g, int key_bytes, uint64_t budget);
cudaError_t point_lookup_u32(const void* keys, const uint32_t* rows, const Geom& g,
                             const LookupCfg& c, const void* q, uint64_t m, uint32_t* out,
                             uint32_t* dflags, cudaStream_t s);
cudaError_t point_lookup_u64(const void* keys, const uint32_t* rows, const Geom& g,
                             const LookupCfg& c, const void* q, uint64_t m, uint32_t* out,
                             uint32_t* dflags, cudaStream_t s);
// (k, lanes per lookup) pairs the k-ary lookup kernel is compiled for, per key
// width.  Lanes hold 8/16/32-byte vectors of a node where it splits evenly;
// otherwise one key per lane (or the whole node in one lane, G = 1).
#define GI_EKS_PAIRS_U64(X)                         \
  X(3, 1) X(3, 2)                                   \
  X(4, 1) X(4, 4)                                   \
  X(5, 1) X(5, 2) X(5, 4)                           \
  X(8, 1) X(8, 8)                                   \
  X(9, 1) X(9, 2) X(9, 4) X(9, 8)                   \
  X(16, 1) X(16, 16)                                \
  X(17, 1) X(17, 4) X(17, 8) X(17, 16)              \
  X(32, 32)                                         \
  X(33, 8) X(33, 16) X(33, 32)
#define GI_EKS_PAIRS_U32(X)                         \
  X(3, 1) X(3, 2)                                   \
  X(4, 1) X(4, 4)                                   \
  X(5, 1) X(5, 2) X(5, 4)                           \
  X(8, 1) X(8, 8)                                   \
  X(9, 1) X(9, 2) X(9, 4) X(9, 8)                   \
  X(16, 1) X(16, 16)                                \
  X(17, 1) X(17, 2) X(17, 4) X(17, 8) X(17, 16)     \
  X(32, 32)                                         \
  X(33, 4) X(33, 8) X(33, 16) X(33, 32)
// Where the hybrid sort (MSD windows + shared-memory bucket sort) replaces the
// LSD passes by default.  Measured on GB300, whole builds of unique keys, layouts
// identical, with the bucket lists made on the device: u64 keys 2^18 0.10 vs
// 0.17 ms (LSD), 2^19 0.18 vs 0.20, 2^20 0.20 vs 0.25, 2^21 0.24 vs 0.37; u32 keys
// 2^23 0.40 vs 0.41, 2^24 0.67 vs 0.73, 2^26 2.09 vs 2.53 (smaller sizes were not
// measured).  Keys that differ in fewer bytes than hybrid_min_digits save too few
// LSD passes to pay for the two MSD passes.
inline uint64_t hybrid_min_pairs(int key_bytes) { return key_bytes == 8 ? (1ull << 18) : (1ull << 23); }
inline uint32_t hybrid_min_digits(int key_bytes) { return key_bytes == 8 ? 5u : 4u; }
bool eks_group_supported(uint32_t k, int key_bytes, int group);
int eks_default_group(uint32_t k, int key_bytes);
// slots staged in shared memory for `levels` top levels (0 = none)
uint64_t smem_slots_for_levels(int layout, const Geom& g, int levels, int key_bytes);

// Range lookups (gi_lookup_u32/u64.cu).  scratch: range_scratch_bytes(m) bytes.
// counts_ready: `offsets` already holds the scanned offsets of these ranges and
// scratch their lower ranks (the first call of the two-call protocol).
size_t range_scratch_bytes(uint64_t m);
cudaError_t range_lookup_u32(const void* keys, const uint32_t* rows, const Geom& g,
                             const LookupCfg& c, const void* lo, const void* hi, uint64_t m,
                             uint64_t* offsets, uint32_t* out_rows, void* scratch,
                             bool counts_ready, cudaStream_t s);
cudaError_t range_lookup_u64(const void* keys, const uint32_t* rows, const Geom& g,
                             const LookupCfg& c, const void* lo, const void* hi, uint64_t m,
                             uint64_t* offsets, uint32_t* out_rows, void* scratch,
                             bool counts_ready, cudaStream_t s);
// The fill alone (any key width): ranges [0, m) of `offsets` / `lo_rank` (the
// scratch's first m words after the count pass); offsets are absolute, so
// offsets + a, lo_rank + a, m = b - a fill ranges [a, b).
cudaError_t range_fill_rows(const uint32_t* rows, const Geom& g, const LookupCfg& c,
                            const uint64_t* offsets, const uint64_t* lo_rank, uint64_t m,
                            uint32_t* out_rows, cudaStream_t s);

// Probes (gi_probe.cu).
cudaError_t probe_random_sectors(const void* buf, uint64_t bytes, uint32_t chunk_bytes,
                                 uint64_t loads, uint64_t seed, uint64_t* sink,
                                 cudaStream_t s);
cudaError_t coalescing_probe(const uint32_t* buf, uint64_t entries, uint32_t threads,
                             uint32_t group, uint32_t steps, uint64_t seed, uint64_t* sink,
                             cudaStream_t s);

}  // namespace gi
