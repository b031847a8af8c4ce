// Bucket sort in shared memory, the last step of the hybrid build sort.
//
// After the stable MSD scatters on the top digits (gi_sort.cu) the pairs lie in
// buckets: runs whose keys agree on every digit outside `local_mask`.  One CTA
// takes one bucket at a time:
//
//   1. it loads the bucket into shared memory (padding keys ~0 sort last);
//   2. it splits the bucket on its top local digit into 256 sub-buckets: for
//      64-bit keys whose lower bits and a 13-bit load position fit in 64 bits
//      (the single-index build of u64 keys), by shared-memory atomics, in any
//      order, each key carried as (lower bits << 13 | load position), whose
//      order is the (key, input position) order, while the rowIDs stay where
//      they were loaded (2^26 u64 keys: 2.41 ms per build against 2.58 with the
//      stable ballot scatter; 2^28: 10.1 against 10.6); otherwise stably with
//      the warp-ballot ranking of the radix passes;
//   3. count ranking: every key's final place inside its sub-bucket is the number
//      of keys there that are smaller, or equal and earlier (earlier = first in
//      the input: every scatter so far was stable, or the position is part of
//      the compared value).  Sub-buckets hold a few
//      keys on average, so this costs a few compares per key instead of one
//      ballot pass per remaining digit.  A bucket with a sub-bucket larger than
//      `limit` instead runs the ballot pass for every local digit (LSD order);
//   4. it writes the bucket in sorted order straight into the final layout:
//      rank r = bucket start + position goes to slot rank_to_slot(r) of the
//      k-ary (or Eytzinger) order -- the inverse of the closed-form slot -> rank
//      map of Section 4 / Section 6.1 -- or to slot r for the sorted layout, so
//      no separate permutation pass reads the sorted array again.  Equal
//      neighbours in sorted order raise the duplicate flag (a bucket holds every
//      copy of its keys, so no pair of equal keys straddles two buckets).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "gi_internal.cuh"

namespace gi {

namespace {

constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
// CTA widths: 256 threads (thread d owns digit d in the scans) or 512 (the second
// half only ranks and moves keys) for the largest buckets.
constexpr uint32_t kCapacity = 5120;  // pairs per bucket: 512 threads x 10

template <int T>
struct LocalSmem {
  template <class K>
  static size_t bytes(int items) {
    const size_t tile = (size_t)T * items;
    return tile * sizeof(K) + tile * 4 +              // keys, rowIDs
           sizeof(uint32_t) * kRadix * (T / 32) +     // per-warp digit counts
           sizeof(uint32_t) * (2 * kRadix + T / 32) +  // sub-bucket starts / ends, warp totals
           sizeof(uint16_t) * tile;                   // sorted position -> current position
  }
};

// One stable scatter of the keys in shared memory on the digit at `shift`.
// Warp w holds the contiguous run [w * 32 * items, (w + 1) * 32 * items), so the
// order inside a warp (item-major, then lane) and across warps is the input order.
// On return s_start[d] is the first position of digit d.
template <class K, int ITEMS, int T>
__device__ __forceinline__ void digit_pass(K* s_k, uint32_t* s_v, uint32_t (*h)[kRadix],
                                           uint32_t* s_start, uint32_t* s_wt, uint32_t items,
                                           uint32_t shift) {
  constexpr int W = T / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const uint32_t wofs = (uint32_t)warp * 32 * items + lane;
  K key[ITEMS];
  uint32_t val[ITEMS], rnk[ITEMS];
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    if (i < (int)items) {
      key[i] = s_k[wofs + i * 32];
      val[i] = s_v[wofs + i * 32];
    }
  }
  for (int i = lane; i < kRadix; i += 32) h[warp][i] = 0;
  __syncwarp();
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    if (i < (int)items) {
      const uint32_t d = (uint32_t)(key[i] >> shift) & 0xFF;
      uint32_t peers = 0xffffffffu;  // lanes holding the same digit
#pragma unroll
      for (int b = 0; b < kRadixBits; ++b) {
        const uint32_t bit = (d >> b) & 1u;
        peers &= ~(__ballot_sync(0xffffffffu, bit) ^ (0u - bit));
      }
      const uint32_t base = h[warp][d];
      __syncwarp();
      if (lane == 31 - __clz(peers)) h[warp][d] = base + __popc(peers);
      __syncwarp();
      rnk[i] = base + __popc(peers & lt_mask);
    }
  }
  __syncthreads();
  // threads d < 256: digit d's count over warps, then a scan over digits
  const uint32_t d = tid;
  uint32_t cnt = 0, x = 0;
  if (tid < kRadix) {
#pragma unroll
    for (int w = 0; w < W; ++w) {
      const uint32_t c = h[w][d];
      h[w][d] = cnt;
      cnt += c;
    }
    x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_wt[warp] = x;
  }
  __syncthreads();
  if (tid < kRadix) {
    uint32_t wpre = 0;
#pragma unroll
    for (int w = 0; w < kRadix / 32; ++w) wpre += (w < warp) ? s_wt[w] : 0u;
    s_start[d] = wpre + x - cnt;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    if (i < (int)items) {
      const uint32_t dd = (uint32_t)(key[i] >> shift) & 0xFF;
      const uint32_t pos = s_start[dd] + h[warp][dd] + rnk[i];
      s_k[pos] = key[i];
      s_v[pos] = val[i];
    }
  }
  __syncthreads();
}

// Shared-memory views of one CTA's bucket (dynamic shared memory, LocalSmem::bytes).
template <class K, int ITEMS, int T>
struct BucketSmem {
  static constexpr int TILE = T * ITEMS;
  K* s_k;
  uint32_t* s_v;
  uint32_t (*h)[kRadix];  // [warps][256]
  uint32_t* s_start;
  uint32_t* s_end;
  uint32_t* s_wt;
  uint16_t* s_src;  // sorted position -> position in s_k / s_v
  __device__ explicit BucketSmem(unsigned char* raw) {
    s_k = (K*)raw;
    s_v = (uint32_t*)(s_k + TILE);
    h = (uint32_t (*)[kRadix])(s_v + TILE);
    s_start = (uint32_t*)(h + T / 32);
    s_end = s_start + kRadix;
    s_wt = s_end + kRadix;
    s_src = (uint16_t*)(s_wt + T / 32);
  }
};

// Where a sorted bucket's pairs are: direct = s_k / s_v in sorted order, else
// sorted position j is at s_src[j]; packed = s_k holds (key & low mask) << 13 |
// position instead of the key, which is hi | (s_k[p] >> 13).
template <class K>
struct BucketOrder {
  bool direct;
  bool packed;
  K hi;
  bool orig;  // packed, and the rowIDs stayed in load order: rowID of s_k[p] is s_v[s_k[p] & 8191]
  __device__ __forceinline__ K key(K stored) const { return packed ? (K)(hi | (stored >> 13)) : stored; }
  __device__ __forceinline__ uint32_t val(const uint32_t* s_v, K stored, uint32_t p) const {
    return orig ? s_v[(uint32_t)stored & 8191u] : s_v[p];
  }
};

// Sorts the `count` pairs at src + start (count <= T * ITEMS) in shared memory.
// top_shift: the window (8 bits at that shift) that splits the bucket into
// sub-buckets for count ranking; every key of the bucket agrees on the bits at
// and above top_shift + 8; lsd_mask: the bytes that may differ inside the bucket,
// sorted one ballot pass each (LSD order) when a sub-bucket is larger than
// `limit`; single: the top window alone orders the bucket.  Block-uniform.
template <class K, int ITEMS, int T>
__device__ __forceinline__ BucketOrder<K> sort_bucket(const BucketSmem<K, ITEMS, T>& m,
                                            const K* __restrict__ src_k,
                                            const uint32_t* __restrict__ src_v, uint64_t start,
                                            uint32_t count, uint32_t top_shift, uint32_t lsd_mask,
                                            bool single, uint32_t limit, bool check_rows,
                                            uint32_t* __restrict__ flags) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t items = (count + T - 1) / T;  // <= ITEMS
  const uint32_t used = items * T;
  bool bad = false;  // an input rowID equal to the reserved miss value
  for (uint32_t j = tid; j < used; j += T) {
    const bool in = j < count;
    m.s_k[j] = in ? src_k[start + j] : ~K(0);  // padding sorts last, stably
    const uint32_t v = in ? src_v[start + j] : 0u;
    bad |= check_rows && in && v == GI_MISS;
    m.s_v[j] = v;
  }
  if (check_rows && __any_sync(0xffffffffu, bad) && lane == 0) atomicOr(flags, kFlagReservedRowid);
  __syncthreads();
  // the top window first; if a sub-bucket is too big for count ranking, every
  // byte of lsd_mask again in LSD order (one pass loop keeps one copy of the
  // pass's code and its registers)
  bool first = lsd_mask != 0, direct = single || lsd_mask == 0;
  uint32_t todo = first ? 1u : 0u;
  while (todo) {
    const uint32_t shift = first ? top_shift : 8u * (uint32_t)(__ffs(todo) - 1);
    todo &= todo - 1;
    digit_pass<K, ITEMS, T>(m.s_k, m.s_v, m.h, m.s_start, m.s_wt, items, shift);
    if (first) {
      first = false;
      if (!single) {
        // sub-bucket d covers [s_start[d], s_end[d]) of real keys (padding sits
        // after count: it has the largest window value and came last)
        bool big = false;
        if (tid < kRadix) {
          const uint32_t st = m.s_start[tid];
          const uint32_t en = tid < kRadix - 1 ? m.s_start[tid + 1] : used;
          const uint32_t en_real = en < count ? en : count;
          m.s_end[tid] = en_real;
          big = (en_real > st ? en_real - st : 0u) > limit;
        }
        if (__syncthreads_or(big)) {
          todo = lsd_mask;
          direct = true;
        }
      }
    }
  }
  BucketOrder<K> ord{direct, false, K(0), false};
  if (!direct) {
    const uint32_t wofs = (uint32_t)warp * 32 * items + lane;
    // 64-bit keys: inside a sub-bucket only the bits below top_shift + 8 differ.
    // When they and the 13-bit position fit in 64 bits, every key is replaced in
    // place by (those bits << 13 | position): distinct values whose order is the
    // (key, position) order, so one 64-bit compare ranks a pair.
    const uint32_t low = top_shift + 8;
    if (sizeof(K) == 8 && low + 13 <= 64) {
      const uint64_t lmask = (1ull << low) - 1;
      const K hi = (K)((uint64_t)m.s_k[0] & ~lmask);  // position 0 holds a real key (count >= 1)
      __syncthreads();
      for (uint32_t j = tid; j < count; j += T) m.s_k[j] = (K)((((uint64_t)m.s_k[j] & lmask) << 13) | j);
      __syncthreads();
#pragma unroll 1
      for (uint32_t i = 0; i < items; ++i) {
        const uint32_t p = wofs + i * 32;
        if (p < count) {
          const K c = m.s_k[p];
          const uint32_t d = (uint32_t)(c >> (top_shift + 13)) & 0xFF;
          const uint32_t b = m.s_start[d], e = m.s_end[d];
          uint32_t r = 0, j = b;
          for (; j + 1 < e; j += 2) r += (m.s_k[j] < c ? 1u : 0u) + (m.s_k[j + 1] < c ? 1u : 0u);
          if (j < e) r += m.s_k[j] < c ? 1u : 0u;
          m.s_src[b + r] = (uint16_t)p;
        }
      }
      ord.packed = true;
      ord.hi = hi;
    } else {
#pragma unroll 1
      for (uint32_t i = 0; i < items; ++i) {
        const uint32_t p = wofs + i * 32;
        if (p < count) {
          const K x = m.s_k[p];
          const uint32_t d = (uint32_t)(x >> top_shift) & 0xFF;
          const uint32_t b = m.s_start[d], e = m.s_end[d];
          uint32_t r = 0;
          for (uint32_t j = b; j < e; ++j) {
            const K y = m.s_k[j];
            r += (y < x || (y == x && j < p)) ? 1u : 0u;
          }
          m.s_src[b + r] = (uint16_t)p;
        }
      }
    }
    __syncthreads();
  }
  return ord;
}

// The same sort for 64-bit keys whose low bits (below top_shift + 8) and a 13-bit
// position fit in 64 bits, without the ballot pass: every key becomes the composite
// (low bits << 13 | its load position) in a register, the top window is counted
// with shared-memory atomics and the composites are scattered to their window's
// sub-bucket in any order (the split need not be stable: the load position inside
// the composite breaks ties between equal keys, so count ranking restores input
// order); the rowIDs never move (the composite names their slot).  Returns false,
// with nothing sorted, if a sub-bucket is larger than `limit` (the caller then
// takes sort_bucket).
template <class K, int ITEMS, int T>
__device__ __forceinline__ bool sort_bucket_split(const BucketSmem<K, ITEMS, T>& m,
                                                  const K* __restrict__ src_k,
                                                  const uint32_t* __restrict__ src_v, uint64_t start,
                                                  uint32_t count, uint32_t top_shift, uint32_t limit,
                                                  BucketOrder<K>& ord) {
  static_assert(sizeof(K) == 8, "64-bit keys");
  static_assert(ITEMS * T <= 8192, "a position takes 13 bits");
  static_assert(ITEMS <= 16, "the 16-bit order fits in the histogram words");
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t low = top_shift + 8;
  const uint64_t lmask = (1ull << low) - 1;
  uint32_t* cnt = m.s_end;  // counters first; ends after the scan
  if (tid < kRadix) cnt[tid] = 0;
  __syncthreads();
  // composites stay in registers; each pair's place in its sub-bucket waits in s_src
  uint64_t comp[ITEMS];
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const uint32_t j = tid + i * T;
    if (j < count) {
      const uint64_t key = (uint64_t)src_k[start + j];
      m.s_v[j] = src_v[start + j];
      comp[i] = ((key & lmask) << 13) | j;
      if (j == 0) ((K*)m.s_wt)[0] = (K)(key & ~lmask);  // the bits every key shares
      m.s_src[j] = (uint16_t)atomicAdd(&cnt[(uint32_t)(key >> top_shift) & 0xFF], 1u);
    }
  }
  __syncthreads();
  // exclusive scan of the 256 counts (thread d owns digit d)
  bool big = false;
  uint32_t c = 0, x = 0;
  if (tid < kRadix) {
    c = cnt[tid];
    big = c > limit;
    x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
  }
  __shared__ uint32_t s_wsum[kRadix / 32];
  if (tid < kRadix && lane == 31) s_wsum[warp] = x;
  if (__syncthreads_or(big)) return false;
  if (tid < kRadix) {
    uint32_t pre = 0;
#pragma unroll
    for (int w = 0; w < kRadix / 32; ++w) pre += w < warp ? s_wsum[w] : 0u;
    m.s_start[tid] = pre + x - c;
    cnt[tid] = pre + x;  // now the sub-bucket's end
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const uint32_t j = tid + i * T;
    if (j < count) {
      const uint32_t d = (uint32_t)(comp[i] >> (top_shift + 13)) & 0xFF;
      m.s_k[m.s_start[d] + m.s_src[j]] = (K)comp[i];
    }
  }
  __syncthreads();
  // count ranking inside each sub-bucket: one 64-bit compare per pair
#pragma unroll 1
  for (uint32_t p = tid; p < count; p += T) {
    const K cp = m.s_k[p];
    const uint32_t d = (uint32_t)(cp >> (top_shift + 13)) & 0xFF;
    const uint32_t b = m.s_start[d], e = m.s_end[d];
    uint32_t r = 0, j = b;
    for (; j + 1 < e; j += 2) r += (m.s_k[j] < cp ? 1u : 0u) + (m.s_k[j + 1] < cp ? 1u : 0u);
    if (j < e) r += m.s_k[j] < cp ? 1u : 0u;
    m.s_src[b + r] = (uint16_t)p;
  }
  ord.direct = false;
  ord.packed = true;
  ord.orig = true;
  ord.hi = ((const K*)m.s_wt)[0];
  __syncthreads();
  return true;
}

// KF: 1 = sorted layout (slot = rank); >= 2 = k-ary Eytzinger with that fan-out
// (2 = Eytzinger); 0 = k-ary with the fan-out read at run time.
template <class K, int ITEMS, int T, int MINB, int KF>
__global__ void __launch_bounds__(T, MINB) k_local_sort(
    const K* __restrict__ src_k, const uint32_t* __restrict__ src_v, K* __restrict__ dst_k,
    uint32_t* __restrict__ dst_v, const BatchTile* __restrict__ segs, uint64_t nseg,
    const uint32_t* __restrict__ nseg_dev, uint32_t top_shift, uint32_t lsd_mask, uint32_t single,
    uint32_t limit, SlotMap sm, uint32_t key_off, uint32_t* __restrict__ flags) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (nseg_dev) nseg = *nseg_dev;  // the list was written on the device
  const BucketSmem<K, ITEMS, T> m(smem_raw);
  __shared__ SlotMap s_map;  // the slot map from shared memory: 12% faster than from the
                             // kernel parameters in the layout write (measured)
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid < (int)(sizeof(SlotMap) / 4)) ((uint32_t*)&s_map)[tid] = ((const uint32_t*)&sm)[tid];
  // the atomic split where its composites fit (64-bit keys, low bits + 13 <= 64)
  const bool split = sizeof(K) == 8 && !single && lsd_mask != 0 && top_shift + 8 + 13 <= 64;
  bool dup = false;
  for (uint64_t sg = blockIdx.x; sg < nseg; sg += gridDim.x) {
    const BatchTile seg = segs[sg];
    BucketOrder<K> ord{false, false, K(0), false};
    bool done = false;
    if constexpr (sizeof(K) == 8) {
      if (split)
        done = sort_bucket_split<K, ITEMS, T>(m, src_k, src_v, seg.start, seg.count, top_shift,
                                              limit, ord);
    }
    if (!done)
      ord = sort_bucket<K, ITEMS, T>(m, src_k, src_v, seg.start, seg.count, top_shift, lsd_mask,
                                     single != 0, limit, false, flags);
    // sorted position j -> rank seg.start + j -> its slot in the layout
    for (uint32_t j = tid; j < seg.count; j += T) {
      const uint32_t p = ord.direct ? j : m.s_src[j];
      const K stored = m.s_k[p];
      const K key = ord.key(stored);
      if (j > 0) dup |= ord.key(m.s_k[ord.direct ? j - 1 : m.s_src[j - 1]]) == key;
      const uint32_t r = (uint32_t)(seg.start + j);
      uint32_t t = r;
      if constexpr (KF != 1) t = slot_of_rank<KF>(r, s_map);
      dst_k[t + key_off] = key;
      dst_v[t] = ord.val(m.s_v, stored, p);
    }
    __syncthreads();
  }
  if (key_off && blockIdx.x == 0 && tid == 0) dst_k[0] = K(0);  // Eytzinger's empty slot
  if (__any_sync(0xffffffffu, dup) && lane == 0) atomicOr(flags, kFlagDuplicate);
}

// The batch's buckets: bucket id < nseg * 256 is window value (id & 255) of index
// id >> 8 (indexes of plan kPlanMsd, sorted pairs in src after the MSD pass);
// id >= nseg * 256 is the whole index id - nseg * 256 (plan kPlanWhole, pairs still
// in the input).  A launch takes the ids of one size class, (lo_count, hi_count]
// pairs, from `list` (written by k_batch_bucket_lists).  Each bucket writes its
// index's layout at out + seg_base[i].
template <class K, int ITEMS, int T, int MINB, int KF>
__global__ void __launch_bounds__(T, MINB) k_batch_local_sort(
    const K* __restrict__ keys, const uint32_t* __restrict__ vals, const K* __restrict__ src_k,
    const uint32_t* __restrict__ src_v, const uint64_t* __restrict__ seg_start, uint32_t nseg,
    const BatchPlan* __restrict__ plan, const SlotMap* __restrict__ maps,
    const unsigned long long* __restrict__ hist_w, const unsigned long long* __restrict__ offs_w,
    K* __restrict__ out_k, uint32_t* __restrict__ out_v, const uint64_t* __restrict__ seg_base,
    uint32_t lo_count, uint32_t hi_count, const uint32_t* __restrict__ list,
    const uint32_t* __restrict__ list_count, uint32_t* __restrict__ flags) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const BucketSmem<K, ITEMS, T> m(smem_raw);
  __shared__ SlotMap s_map;
  const int tid = threadIdx.x, lane = tid & 31;
  bool dup = false;
  const uint32_t total = *list_count;
  for (uint32_t li = blockIdx.x; li < total; li += gridDim.x) {
    const uint64_t id = list[li];
    const bool msd = id < (uint64_t)nseg * kRadix;
    const uint32_t i = msd ? (uint32_t)(id >> 8) : (uint32_t)(id - (uint64_t)nseg * kRadix);
    const BatchPlan pl = plan[i];
    if (pl.mode != (msd ? kPlanMsd : kPlanWhole)) continue;
    const uint64_t s0 = seg_start[i];
    const uint64_t start = msd ? offs_w[id] : s0;
    const uint32_t count = (uint32_t)(msd ? hist_w[id] : seg_start[i + 1] - s0);
    if (count <= lo_count || count > hi_count) continue;  // another launch's size class
    if constexpr (KF != 1) {  // (KF == -1: the map's k is the index's own fan-out)
      if (tid < (int)(sizeof(SlotMap) / 4)) ((uint32_t*)&s_map)[tid] = ((const uint32_t*)&maps[i])[tid];
    }
    const uint32_t limit = 8u * (uint32_t)__popc(pl.lsd_mask) + 8u;
    // a whole index is read straight from the input: its rowIDs are checked here
    const BucketOrder<K> ord = sort_bucket<K, ITEMS, T>(m, msd ? src_k : keys, msd ? src_v : vals,
                                                        start, count, pl.ts, pl.lsd_mask, false,
                                                        limit, !msd, flags);
    const uint64_t base = seg_base[i];
    const uint32_t r0 = (uint32_t)(start - s0);
    for (uint32_t j = tid; j < count; j += T) {
      const uint32_t p = ord.direct ? j : m.s_src[j];
      const K key = ord.key(m.s_k[p]);
      if (j > 0) dup |= ord.key(m.s_k[ord.direct ? j - 1 : m.s_src[j - 1]]) == key;
      const uint32_t r = r0 + j;
      uint32_t t = r;
      if constexpr (KF == -1) t = slot_of_rank_any(r, s_map);
      else if constexpr (KF != 1) t = slot_of_rank<KF>(r, s_map);
      out_k[base + t] = key;
      out_v[base + t] = m.s_v[p];
    }
    __syncthreads();
  }
  if (__any_sync(0xffffffffu, dup) && lane == 0) atomicOr(flags, kFlagDuplicate);
}

// One CTA per index: its buckets' ids into the list of their size class (one
// atomic per class per CTA).
__global__ void __launch_bounds__(256) k_batch_bucket_lists(
    const BatchPlan* __restrict__ plan, const unsigned long long* __restrict__ hist_w,
    const uint64_t* __restrict__ seg_start, uint32_t nseg, uint32_t b0, uint32_t b1, uint32_t b2,
    uint32_t* __restrict__ lists, uint32_t* __restrict__ counts) {
  __shared__ uint32_t s_cnt[3], s_base[3];
  const uint32_t i = blockIdx.x;
  const int d = threadIdx.x;
  const uint32_t mode = plan[i].mode;
  if (mode != kPlanMsd && mode != kPlanWhole) return;
  if (d < 3) s_cnt[d] = 0;
  __syncthreads();
  uint64_t c = 0, id = 0;
  if (mode == kPlanMsd) {
    id = (uint64_t)i * kRadix + d;
    c = hist_w[id];
  } else if (d == 0) {
    id = (uint64_t)nseg * kRadix + i;
    c = seg_start[i + 1] - seg_start[i];
  }
  const int cls = c == 0 ? -1 : c <= b0 ? 0 : c <= b1 ? 1 : c <= b2 ? 2 : -1;
  uint32_t pos = 0;
  if (cls >= 0) pos = atomicAdd(&s_cnt[cls], 1u);
  __syncthreads();
  if (d < 3 && s_cnt[d]) s_base[d] = atomicAdd(&counts[d], s_cnt[d]);
  __syncthreads();
  if (cls >= 0) lists[(uint64_t)cls * nseg * (kRadix + 1) + s_base[cls] + pos] = (uint32_t)id;
}

// Size classes of the bucket sort: up to 3072 pairs (256 threads x 12, 3 CTAs per
// SM), up to 4096 (256 x 16, 2 per SM), up to 5120 (512 x 10, 2 per SM).
#define GI_LOCAL_CLASSES(X) X(12, 256, 3, 0u, 3072u) X(16, 256, 2, 3072u, 4096u) X(10, 512, 2, 4096u, 5120u)

// Size classes of the single-index bucket sort (one launch per class, each bucket
// in the narrowest class that holds it): smaller buckets in narrower classes
// leave room for more CTAs per SM.  Up to 1536 pairs: 256 threads x 6, 6 CTAs
// per SM (40 registers, 32 KB of shared memory each; 3.4% faster whole builds at
// 2^26 u64 keys than 5 CTAs with 48 registers, despite 72 bytes of spills);
// 2560: x 10, 4 per SM
// (2.6% faster than the 3072 class on 2048-pair buckets); 4096: 512 threads x 8,
// 2 per SM (twice the threads of the batch's 256 x 16 class); then as the batch.
#define GI_LOCAL_CLASSES_SINGLE(X) \
  X(6, 256, 6, 0u, 1536u) X(10, 256, 4, 1536u, 2560u) X(12, 256, 3, 2560u, 3072u) \
  X(8, 512, 2, 3072u, 4096u) X(10, 512, 2, 4096u, 5120u)

// cls >= 0: that class's kernel; else the class of the largest bucket (max_count).
// nseg_dev: the bucket count on the device (nseg is then its upper bound).
template <class K, int KF>
cudaError_t launch(const K* sk, const uint32_t* sv, K* dk, uint32_t* dv, const BatchTile* segs,
                   uint64_t nseg, const uint32_t* nseg_dev, uint64_t max_count, int cls,
                   uint32_t top_shift, uint32_t mask, uint32_t single, uint32_t limit,
                   const SlotMap& sm, uint32_t key_off, uint32_t* dflags, cudaStream_t s) {
  bool done = false;
  int ci = 0;
#define GI_LS(IT, T, MB, LO, HI)                                                               \
  if (!done && (cls >= 0 ? ci == cls : max_count <= HI)) {                                     \
    auto kern = k_local_sort<K, IT, T, MB, KF>;                                                \
    const size_t smem = LocalSmem<T>::template bytes<K>(IT);                                   \
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                                         (int)smem);                                           \
    if (e != cudaSuccess) return e;                                                            \
    const unsigned grid = (unsigned)std::min<uint64_t>(nseg, (uint64_t)sm_count() * MB * 4);   \
    kern<<<grid, T, smem, s>>>(sk, sv, dk, dv, segs, nseg, nseg_dev, top_shift, mask, single,   \
                               limit, sm, key_off, dflags);                                    \
    done = true;                                                                               \
  }                                                                                            \
  ++ci;
  GI_LOCAL_CLASSES_SINGLE(GI_LS)
#undef GI_LS
  if (!done) return cudaErrorInvalidValue;
  count_launch();
  return cudaGetLastError();
}

template <class K>
cudaError_t launch_kf(const void* sk, const uint32_t* sv, void* dk, uint32_t* dv,
                      const BatchTile* segs, uint64_t nseg, const uint32_t* nseg_dev,
                      uint64_t max_count, int cls, uint32_t top_shift, uint32_t mask,
                      uint32_t single, uint32_t limit, const Geom& g, bool sorted,
                      uint32_t key_off, uint32_t* dflags, cudaStream_t s) {
  const K* a = (const K*)sk;
  K* b = (K*)dk;
  const SlotMap sm = make_slot_map(g);
#define GI_L(KF, OFF)                                                                          \
  launch<K, KF>(a, sv, b, dv, segs, nseg, nseg_dev, max_count, cls, top_shift, mask, single, limit, \
                sm, OFF, dflags, s)
  if (sorted) return GI_L(1, 0);
  switch (g.k) {
    case 2: return GI_L(2, key_off);
    case 3: return GI_L(3, key_off);
    case 5: return GI_L(5, key_off);
    case 9: return GI_L(9, key_off);
    case 17: return GI_L(17, key_off);
    default: return GI_L(0, key_off);
  }
#undef GI_L
}

// setup: only raise the kernels' dynamic shared-memory limit (done when the batch
// is created, so that builds launch kernels only and can be captured in a graph)
template <class K, int KF>
cudaError_t launch_batch(const void* keys, const uint32_t* vals, const void* src_k,
                         const uint32_t* src_v, const uint64_t* seg_start, uint32_t nseg,
                         const BatchHybrid& hy, uint32_t* dflags, cudaStream_t s, bool setup) {
#define GI_BLS(IT, T, MB, LO, HI)                                                              \
  {                                                                                            \
    auto kern = k_batch_local_sort<K, IT, T, MB, KF>;                                          \
    const size_t smem = LocalSmem<T>::template bytes<K>(IT);                                   \
    if (setup) {                                                                               \
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                                           (int)smem);                                         \
      if (e != cudaSuccess) return e;                                                          \
    } else {                                                                                   \
      const unsigned grid = (unsigned)sm_count() * MB * 4;                                     \
      kern<<<grid, T, smem, s>>>((const K*)keys, vals, (const K*)src_k, src_v, seg_start, nseg, \
                                 hy.plan, hy.slot_maps, hy.hist_w, hy.offs_w, (K*)hy.out_k,    \
                                 hy.out_v, hy.seg_base, LO, HI,                                \
                                 hy.buckets + (uint64_t)cls * nseg * (kRadix + 1),             \
                                 hy.bucket_count + cls, dflags);                               \
      count_launch();                                                                          \
    }                                                                                          \
    ++cls;                                                                                     \
  }
  int cls = 0;
  GI_LOCAL_CLASSES(GI_BLS)
#undef GI_BLS
  return cudaGetLastError();
}

// ids of the classes (the bounds of GI_LOCAL_CLASSES)
cudaError_t launch_bucket_lists(const uint64_t* seg_start, uint32_t nseg, const BatchHybrid& hy,
                                cudaStream_t s) {
  k_batch_bucket_lists<<<nseg, 256, 0, s>>>(hy.plan, hy.hist_w, seg_start, nseg, 3072u, 4096u,
                                            5120u, hy.buckets, hy.bucket_count);
  count_launch();
  return cudaGetLastError();
}

template <class K>
cudaError_t launch_batch_kf(const void* keys, const uint32_t* vals, const void* src_k,
                            const uint32_t* src_v, const uint64_t* seg_start, uint32_t nseg,
                            const BatchHybrid& hy, uint32_t* dflags, cudaStream_t s, bool setup) {
#define GI_B(KF) launch_batch<K, KF>(keys, vals, src_k, src_v, seg_start, nseg, hy, dflags, s, setup)
  switch (hy.k) {
    case kBatchMixed: return GI_B(-1);  // each index's own fan-out
    case 0: return GI_B(1);
    case 2: return GI_B(2);
    case 3: return GI_B(3);
    case 5: return GI_B(5);
    case 9: return GI_B(9);
    case 17: return GI_B(17);
    default: return cudaErrorInvalidValue;  // the batch takes k = 2, 3, 5, 9, 17 only
  }
#undef GI_B
}

}  // namespace

uint32_t local_sort_capacity() { return kCapacity; }

// the launch table and the class list that the host groups buckets by agree
#define GI_C(IT, T, MB, LO, HI) +1
static_assert(0 GI_LOCAL_CLASSES_SINGLE(GI_C) == kLocalClasses, "one class per table entry");
#undef GI_C
constexpr bool classes_match() {
  int i = 0;
  bool ok = true;
#define GI_C(IT, T, MB, LO, HI) ok = ok && (HI) == local_class_max(i) && (IT) * (T) == (int)(HI); ++i;
  GI_LOCAL_CLASSES_SINGLE(GI_C)
#undef GI_C
  return ok;
}
static_assert(classes_match(), "local_class_max lists the launch table's bounds");

cudaError_t local_sort(const void* sk, const uint32_t* sv, void* dk, uint32_t* dv,
                       const BatchTile* segs, uint64_t nseg, const uint32_t* nseg_dev,
                       uint64_t max_count, int cls, uint32_t top_shift, uint32_t lsd_mask,
                       bool single, int key_bytes, const Geom& g, bool sorted_layout,
                       uint32_t key_off, uint32_t* dflags, cudaStream_t s) {
  if (nseg == 0) return cudaSuccess;
  if (cls >= kLocalClasses) return cudaErrorInvalidValue;
  if ((cls < 0 && max_count > local_sort_capacity()) || g.n >= (1ull << 32)) return cudaErrorInvalidValue;
  // count ranking costs about one compare per key of the sub-bucket; past this
  // size the remaining ballot passes are cheaper
  const uint32_t limit = 8u * (uint32_t)__builtin_popcount(lsd_mask) + 8u;
  if (key_bytes == 4)
    return launch_kf<uint32_t>(sk, sv, dk, dv, segs, nseg, nseg_dev, max_count, cls, top_shift,
                               lsd_mask, single ? 1u : 0u, limit, g, sorted_layout, key_off,
                               dflags, s);
  return launch_kf<uint64_t>(sk, sv, dk, dv, segs, nseg, nseg_dev, max_count, cls, top_shift,
                             lsd_mask, single ? 1u : 0u, limit, g, sorted_layout, key_off, dflags,
                             s);
}

cudaError_t batch_local_sort(const void* keys, const uint32_t* vals, const void* src_k,
                             const uint32_t* src_v, const uint64_t* seg_start, uint32_t nseg,
                             int key_bytes, const BatchHybrid& hy, uint32_t* dflags,
                             cudaStream_t s) {
  if (nseg == 0) return cudaSuccess;
  cudaError_t e = launch_bucket_lists(seg_start, nseg, hy, s);
  if (e != cudaSuccess) return e;
  if (key_bytes == 4)
    return launch_batch_kf<uint32_t>(keys, vals, src_k, src_v, seg_start, nseg, hy, dflags, s, false);
  return launch_batch_kf<uint64_t>(keys, vals, src_k, src_v, seg_start, nseg, hy, dflags, s, false);
}

cudaError_t batch_local_sort_setup(int key_bytes, uint32_t k) {
  BatchHybrid hy{};
  hy.k = k;
  if (key_bytes == 4)
    return launch_batch_kf<uint32_t>(nullptr, nullptr, nullptr, nullptr, nullptr, 0, hy, nullptr, 0, true);
  return launch_batch_kf<uint64_t>(nullptr, nullptr, nullptr, nullptr, nullptr, 0, hy, nullptr, 0, true);
}

}  // namespace gi
