// Bucket sort in shared memory, the last step of the hybrid build sort.
//
// After the stable MSD scatters on the top digits (gi_sort.cu) the pairs lie in
// buckets: runs whose keys agree on every digit outside `local_mask`.  One CTA
// takes one bucket at a time:
//
//   1. it loads the bucket into shared memory (padding keys ~0 sort last);
//   2. it scatters the bucket stably on its top local digit with the warp-ballot
//      ranking of the radix passes, which splits it into 256 sub-buckets;
//   3. count ranking: every key's final place inside its sub-bucket is the number
//      of keys there that are smaller, or equal and earlier (earlier = first in
//      the input, since every scatter so far was stable).  Sub-buckets hold a few
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
constexpr int kThreads = 256;  // == kRadix: thread d owns digit d in the scans
constexpr int kWarps = kThreads / 32;

struct LocalSmem {
  template <class K>
  static size_t bytes(int items) {
    const size_t tile = (size_t)kThreads * items;
    return tile * sizeof(K) + tile * 4 +            // keys, rowIDs
           sizeof(uint32_t) * kRadix * kWarps +     // per-warp digit counts
           sizeof(uint32_t) * (2 * kRadix + kWarps) +  // sub-bucket starts / ends, warp totals
           sizeof(uint16_t) * tile;                 // sorted position -> current position
  }
};

// One stable scatter of the keys in shared memory on the digit at `shift`.
// Warp w holds the contiguous run [w * 32 * items, (w + 1) * 32 * items), so the
// order inside a warp (item-major, then lane) and across warps is the input order.
// On return s_start[d] is the first position of digit d.
template <class K, int ITEMS>
__device__ __forceinline__ void digit_pass(K* s_k, uint32_t* s_v, uint32_t (*h)[kRadix],
                                           uint32_t* s_start, uint32_t* s_wt, uint32_t items,
                                           uint32_t shift) {
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
  {  // thread d: digit d's count over warps, then a block scan over digits
    const uint32_t d = tid;
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      const uint32_t c = h[w][d];
      h[w][d] = cnt;
      cnt += c;
    }
    uint32_t x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_wt[warp] = x;
    __syncthreads();
    uint32_t wpre = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) wpre += (w < warp) ? s_wt[w] : 0u;
    s_start[d] = wpre + x - cnt;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    if (i < (int)items) {
      const uint32_t d = (uint32_t)(key[i] >> shift) & 0xFF;
      const uint32_t pos = s_start[d] + h[warp][d] + rnk[i];
      s_k[pos] = key[i];
      s_v[pos] = val[i];
    }
  }
  __syncthreads();
}

// KF: 1 = sorted layout (slot = rank); >= 2 = k-ary Eytzinger with that fan-out
// (2 = Eytzinger); 0 = k-ary with the fan-out g.k read at run time.
template <class K, int ITEMS, int MINB, int KF>
__global__ void __launch_bounds__(kThreads, MINB) k_local_sort(
    const K* __restrict__ src_k, const uint32_t* __restrict__ src_v, K* __restrict__ dst_k,
    uint32_t* __restrict__ dst_v, const BatchTile* __restrict__ segs, uint64_t nseg,
    uint32_t local_mask, uint32_t limit, SlotMap sm, uint32_t key_off, uint32_t* __restrict__ flags) {
  constexpr int TILE = kThreads * ITEMS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  K* s_k = (K*)smem_raw;
  uint32_t* s_v = (uint32_t*)(s_k + TILE);
  uint32_t (*h)[kRadix] = (uint32_t (*)[kRadix])(s_v + TILE);  // [warps][256]
  uint32_t* s_start = (uint32_t*)(h + kWarps);
  uint32_t* s_end = s_start + kRadix;
  uint32_t* s_wt = s_end + kRadix;
  uint16_t* s_src = (uint16_t*)(s_wt + kWarps);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t top = local_mask ? 31u - (uint32_t)__clz(local_mask) : 0u;
  const uint32_t top_shift = 8u * top;
  const bool single = __popc(local_mask) <= 1;  // the top pass alone sorts the bucket
  bool dup = false;
  for (uint64_t sg = blockIdx.x; sg < nseg; sg += gridDim.x) {
    const BatchTile seg = segs[sg];
    const uint32_t items = (seg.count + kThreads - 1) / kThreads;  // <= ITEMS
    const uint32_t used = items * kThreads;
    for (uint32_t j = tid; j < used; j += kThreads) {
      const bool in = j < seg.count;
      s_k[j] = in ? src_k[seg.start + j] : ~K(0);  // padding sorts last, stably
      s_v[j] = in ? src_v[seg.start + j] : 0u;
    }
    __syncthreads();
    // the top local digit first; if a sub-bucket is too big for count ranking,
    // every local digit again in LSD order (one pass loop keeps one copy of the
    // pass's code and its registers)
    uint32_t todo = local_mask ? 1u << top : 0u;
    bool first = true, direct = single;
    while (todo) {
      const uint32_t shift = 8u * (uint32_t)(__ffs(todo) - 1);
      todo &= todo - 1;
      digit_pass<K, ITEMS>(s_k, s_v, h, s_start, s_wt, items, shift);
      if (first && !single) {
        first = false;
        // sub-bucket d covers [s_start[d], s_end[d]) of real keys (padding sits
        // after seg.count: it has the largest digit and came last)
        const uint32_t st = s_start[tid];
        const uint32_t en = tid < kRadix - 1 ? s_start[tid + 1] : used;
        const uint32_t en_real = en < seg.count ? en : seg.count;
        s_end[tid] = en_real;
        const bool big = (en_real > st ? en_real - st : 0u) > limit;
        if (__syncthreads_or(big)) {
          todo = local_mask;
          direct = true;
        }
      }
    }
    if (!direct) {
      const uint32_t wofs = (uint32_t)warp * 32 * items + lane;
#pragma unroll 1
      for (uint32_t i = 0; i < items; ++i) {
        const uint32_t p = wofs + i * 32;
        if (p < seg.count) {
          const K x = s_k[p];
          const uint32_t d = (uint32_t)(x >> top_shift) & 0xFF;
          const uint32_t b = s_start[d], e = s_end[d];
          uint32_t r = 0;
          for (uint32_t j = b; j < e; ++j) {
            const K y = s_k[j];
            r += (y < x || (y == x && j < p)) ? 1u : 0u;
          }
          s_src[b + r] = (uint16_t)p;
        }
      }
      __syncthreads();
    }
    // sorted position j -> rank seg.start + j -> its slot in the layout
    for (uint32_t j = tid; j < seg.count; j += kThreads) {
      const uint32_t p = direct ? j : s_src[j];
      const K key = s_k[p];
      if (j > 0) dup |= s_k[direct ? j - 1 : s_src[j - 1]] == key;
      const uint32_t r = (uint32_t)(seg.start + j);
      uint32_t t = r;
      if constexpr (KF != 1) t = slot_of_rank<KF>(r, sm);
      dst_k[t + key_off] = key;
      dst_v[t] = s_v[p];
    }
    __syncthreads();
  }
  if (key_off && blockIdx.x == 0 && tid == 0) dst_k[0] = K(0);  // Eytzinger's empty slot
  if (__any_sync(0xffffffffu, dup) && lane == 0) atomicOr(flags, kFlagDuplicate);
}

template <class K, int KF>
cudaError_t launch(const K* sk, const uint32_t* sv, K* dk, uint32_t* dv, const BatchTile* segs,
                   uint64_t nseg, uint64_t max_count, uint32_t mask, uint32_t limit,
                   const SlotMap& sm, uint32_t key_off, uint32_t* dflags, cudaStream_t s) {
#define GI_LS(IT, MB)                                                                          \
  do {                                                                                         \
    auto kern = k_local_sort<K, IT, MB, KF>;                                                   \
    const size_t smem = LocalSmem::bytes<K>(IT);                                               \
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                                         (int)smem);                                           \
    if (e != cudaSuccess) return e;                                                            \
    const unsigned grid = (unsigned)std::min<uint64_t>(nseg, (uint64_t)sm_count() * MB * 4);   \
    kern<<<grid, kThreads, smem, s>>>(sk, sv, dk, dv, segs, nseg, mask, limit, sm, key_off,    \
                                      dflags);                                                 \
  } while (0)
  if (max_count <= (uint64_t)kThreads * 12)
    GI_LS(12, 3);
  else
    GI_LS(16, 2);
#undef GI_LS
  count_launch();
  return cudaGetLastError();
}

template <class K>
cudaError_t launch_kf(const void* sk, const uint32_t* sv, void* dk, uint32_t* dv,
                      const BatchTile* segs, uint64_t nseg, uint64_t max_count, uint32_t mask,
                      uint32_t limit, const Geom& g, bool sorted, uint32_t key_off,
                      uint32_t* dflags, cudaStream_t s) {
  const K* a = (const K*)sk;
  K* b = (K*)dk;
  const SlotMap sm = make_slot_map(g);
#define GI_L(KF, OFF) launch<K, KF>(a, sv, b, dv, segs, nseg, max_count, mask, limit, sm, OFF, dflags, s)
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

}  // namespace

uint32_t local_sort_capacity() { return kThreads * 16; }

cudaError_t local_sort(const void* sk, const uint32_t* sv, void* dk, uint32_t* dv,
                       const BatchTile* segs, uint64_t nseg, uint64_t max_count,
                       uint32_t local_mask, int key_bytes, const Geom& g, bool sorted_layout,
                       uint32_t key_off, uint32_t* dflags, cudaStream_t s) {
  if (nseg == 0) return cudaSuccess;
  if (max_count > local_sort_capacity() || g.n >= (1ull << 32)) return cudaErrorInvalidValue;
  // count ranking costs about one compare per key of the sub-bucket; past this
  // size the remaining ballot passes are cheaper
  const uint32_t limit = 8u * (uint32_t)__builtin_popcount(local_mask) + 8u;
  if (key_bytes == 4)
    return launch_kf<uint32_t>(sk, sv, dk, dv, segs, nseg, max_count, local_mask, limit, g,
                               sorted_layout, key_off, dflags, s);
  return launch_kf<uint64_t>(sk, sv, dk, dv, segs, nseg, max_count, local_mask, limit, g,
                             sorted_layout, key_off, dflags, s);
}

}  // namespace gi
