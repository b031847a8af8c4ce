// Range-lookup kernels, templated on the key type (Sections 1 and 5).
//
// A range [L, U] (inclusive) selects the ranks [lower_bound(L), upper_bound(U))
// of the sorted order.  The CSR result is built in three passes:
//   count : per range, one descent for L and one for U (interleaved, so the two
//           dependent chains overlap), giving the two ranks; count = difference.
//           The rank of the slot where a descent ends is p'(slot) (Section 6.1).
//   scan  : exclusive prefix sum of the counts -> offsets (reduce, scan of the
//           block sums, down-sweep; no inter-block waits).
//   fill  : rows of rank r come from slot(r), the closed-form inverse of p'.
//           A warp takes 32 consecutive ranges; ranges with at least 32 rows are
//           emitted by the whole warp with coalesced stores, one range at a time;
//           the rows of the shorter ranges are dealt to the lanes together (each
//           lane finds its row's range by a 5-step shuffle search over the
//           running counts), so their stores are coalesced too -- the paper's
//           single-thread / warp switch of Section 5.1 applied to the output
//           pass.  GI_OPT_RANGE_FILL = 1 instead walks each range level by level,
//           one contiguous slot run per level (k_range_fill_levels).
// Rows of a range come out in ascending rank order, i.e. ascending (key, input
// position) order, for every layout.  (The paper's level-by-level scan emits
// them level by level instead; Section 5.)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gi_internal.cuh"
#include "gi_point_impl.cuh"

namespace gi {
namespace rg {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// ---------------------------------------------------------------- bounds per layout
// rank of the first key >= x (upper = false) or > x (upper = true)
template <class K>
__device__ __forceinline__ bool before(K v, K x, bool upper) {
  return upper ? (v <= x) : (v < x);
}

template <class K>
__device__ __forceinline__ uint64_t sorted_bound(const K* __restrict__ keys, uint64_t n, K x,
                                                 bool upper) {
  uint64_t lo = 0, len = n;
  while (len > 0) {
    const uint64_t half = len >> 1;
    if (before(keys[lo + half], x, upper)) {
      lo += half + 1;
      len -= half + 1;
    } else {
      len = half;
    }
  }
  return lo;
}

// keys 1-based; returns the rank (n if no such key).
template <class K>
__device__ __forceinline__ void ebs_bounds(const K* __restrict__ keys, const Geom& g, K L, K U,
                                           uint64_t& rl, uint64_t& ru) {
  uint64_t a = 1, b = 1;
  for (uint32_t lv = 0; lv < g.levels; ++lv) {
    if (a <= g.n) a = 2 * a + (__ldg(keys + a) < L ? 1 : 0);
    if (b <= g.n) b = 2 * b + (__ldg(keys + b) <= U ? 1 : 0);
  }
  a >>= __ffsll((long long)~a);
  b >>= __ffsll((long long)~b);
  rl = a ? slot_to_rank<2>(a - 1, g) : g.n;
  ru = b ? slot_to_rank<2>(b - 1, g) : g.n;
}

// k-ary: a group of G lanes (one key per lane), both descents interleaved.
// Slots past n hold the maximum key, so only lanes past the node end are masked.
template <class K, int KF, int G>
__device__ __forceinline__ void eks_bounds(const K* __restrict__ keys, const Geom& g, K L, K U,
                                           int gl, uint32_t gmask, uint64_t& rl, uint64_t& ru) {
  constexpr int N = KF - 1;
  constexpr int P = (N + G - 1) / G;
  const uint64_t n = g.n;
  uint64_t s[2] = {0, 0}, cand[2] = {~0ull, ~0ull};
  const K x[2] = {L, U};
  for (uint32_t lv = 0; lv < g.levels; ++lv) {
    K piv[2][P];
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      if (s[d] < n) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
          const int j = gl + p * G;
          piv[d][p] = j < N ? __ldg(keys + s[d] + j) : K(0);
        }
      }
    }
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      if (s[d] < n) {
        uint32_t c = 0;
#pragma unroll
        for (int p = 0; p < P; ++p) {
          const int j = gl + p * G;
          c += __popc(__ballot_sync(gmask, j < N && before(piv[d][p], x[d], d == 1)) & gmask);
        }
        if (c < (uint32_t)N && s[d] + c < n) cand[d] = s[d] + c;
        s[d] = s[d] * KF + (uint64_t)(c + 1) * N;
      }
    }
  }
  rl = cand[0] != ~0ull ? slot_to_rank<KF>(cand[0], g) : n;
  ru = cand[1] != ~0ull ? slot_to_rank<KF>(cand[1], g) : n;
}

// k-ary, one thread per range when a node is at most 64 bytes: both descents
// interleaved, whole nodes loaded (vector loads where the node is a power-of-two
// vector), no ballots.
template <class K, int KF>
__device__ __forceinline__ void eks_bounds_single(const K* __restrict__ keys, const Geom& g, K L,
                                                  K U, uint64_t& rl, uint64_t& ru) {
  constexpr int N = KF - 1;
  const uint64_t n = g.n;
  uint64_t s0 = 0, s1 = 0, c0 = ~0ull, c1 = ~0ull;
  for (uint32_t lv = 0; lv < g.levels; ++lv) {
    K a[N], b[N];
    if constexpr (pt::EksShape<K, KF, 1>::VEC) {
      if (s0 < n) pt::vec_load<K, N>(keys + s0, a);
      if (s1 < n) pt::vec_load<K, N>(keys + s1, b);
    } else {  // nodes that are not a power-of-two vector: plain loads
#pragma unroll
      for (int p = 0; p < N; ++p) {
        if (s0 < n) a[p] = __ldg(keys + s0 + p);
        if (s1 < n) b[p] = __ldg(keys + s1 + p);
      }
    }
    if (s0 < n) {
      uint32_t c = 0;
#pragma unroll
      for (int p = 0; p < N; ++p) c += a[p] < L ? 1u : 0u;
      if (c < (uint32_t)N && s0 + c < n) c0 = s0 + c;
      s0 = s0 * KF + (uint64_t)(c + 1) * N;
    }
    if (s1 < n) {
      uint32_t c = 0;
#pragma unroll
      for (int p = 0; p < N; ++p) c += b[p] <= U ? 1u : 0u;
      if (c < (uint32_t)N && s1 + c < n) c1 = s1 + c;
      s1 = s1 * KF + (uint64_t)(c + 1) * N;
    }
  }
  rl = c0 != ~0ull ? slot_to_rank<KF>(c0, g) : n;
  ru = c1 != ~0ull ? slot_to_rank<KF>(c1, g) : n;
}

// Any k at run time, one thread.
template <class K>
__device__ __forceinline__ uint64_t eks_bound_generic(const K* __restrict__ keys, const Geom& g,
                                                      K x, bool upper) {
  const uint64_t n = g.n, k = g.k;
  uint64_t s = 0, cand = ~0ull;
  while (s < n) {
    uint32_t c = 0;
    for (uint32_t j = 0; j + 1 < k && s + j < n; ++j) {
      if (before(keys[s + j], x, upper))
        ++c;
      else
        break;
    }
    if (c < k - 1 && s + c < n) cand = s + c;
    s = s * k + (uint64_t)(c + 1) * (k - 1);
  }
  return cand != ~0ull ? slot_to_rank<0>(cand, g) : n;
}

// ---------------------------------------------------------------- count
// layout: 0 sorted, 1 Eytzinger, 2 k-ary (KF > 0: lane groups of G; KF == 0: generic)
template <class K, int LAYOUT, int KF, int G>
__global__ void __launch_bounds__(256) k_range_count(const K* __restrict__ keys, Geom g,
                                                     const K* __restrict__ lo,
                                                     const K* __restrict__ hi, uint64_t m,
                                                     uint64_t* __restrict__ counts,
                                                     uint64_t* __restrict__ lo_rank) {
  const int lane = threadIdx.x & 31;
  const int gl = lane % G;
  const uint32_t gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane - gl));
  const uint64_t groups = ((uint64_t)gridDim.x * blockDim.x) / G;
  for (uint64_t i = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / G; i < m; i += groups) {
    const K L = lo[i], U = hi[i];
    uint64_t rl = 0, ru = 0;
    if (L <= U) {
      if constexpr (LAYOUT == 0) {
        rl = sorted_bound(keys, g.n, L, false);
        ru = sorted_bound(keys, g.n, U, true);
      } else if constexpr (LAYOUT == 1) {
        ebs_bounds(keys, g, L, U, rl, ru);
      } else if constexpr (KF > 0 && G == 1) {
        eks_bounds_single<K, KF>(keys, g, L, U, rl, ru);
      } else if constexpr (KF > 0) {
        eks_bounds<K, KF, G>(keys, g, L, U, gl, gmask, rl, ru);
      } else {
        rl = eks_bound_generic(keys, g, L, false);
        ru = eks_bound_generic(keys, g, U, true);
      }
    }
    if (gl == 0) {
      counts[i] = ru - rl;
      lo_rank[i] = rl;
    }
  }
}

// ---------------------------------------------------------------- scan (in place, exclusive)
__device__ __forceinline__ uint64_t block_exclusive_scan(uint64_t v, uint64_t* s_warp,
                                                         uint64_t& total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[w] = x;
  __syncthreads();
  uint64_t pre = 0, tot = 0;
  const int nw = blockDim.x >> 5;
  for (int i = 0; i < nw; ++i) {
    if (i < w) pre += s_warp[i];
    tot += s_warp[i];
  }
  __syncthreads();
  total = tot;
  return pre + x - v;
}

static __global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint64_t* __restrict__ a,
                                                              uint64_t m,
                                                              uint64_t* __restrict__ block_sums) {
  __shared__ uint64_t s_warp[kScanThreads / 32];
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
  uint64_t sum = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const uint64_t j = base + (uint64_t)i * kScanThreads + threadIdx.x;
    if (j < m) sum += a[j];
  }
  uint64_t tot;
  block_exclusive_scan(sum, s_warp, tot);
  if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

// One CTA: exclusive scan of the block sums (any count, in chunks), total at [nb].
static __global__ void __launch_bounds__(1024) k_scan_sums(uint64_t* __restrict__ sums, uint64_t nb) {
  __shared__ uint64_t s_warp[32];
  uint64_t carry = 0;
  for (uint64_t base = 0; base < nb; base += blockDim.x) {
    const uint64_t j = base + threadIdx.x;
    const uint64_t v = j < nb ? sums[j] : 0;
    uint64_t tot;
    const uint64_t ex = block_exclusive_scan(v, s_warp, tot);
    if (j < nb) sums[j] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) sums[nb] = carry;
}

static __global__ void __launch_bounds__(kScanThreads) k_scan_down(uint64_t* __restrict__ a, uint64_t m,
                                                            const uint64_t* __restrict__ sums) {
  __shared__ uint64_t s_warp[kScanThreads / 32];
  __shared__ uint64_t s_tile[kScanTile];
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
  // blocked ownership for the scan: thread t holds items t*ITEMS .. t*ITEMS+ITEMS-1
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const uint64_t j = base + (uint64_t)i * kScanThreads + threadIdx.x;
    s_tile[i * kScanThreads + threadIdx.x] = j < m ? a[j] : 0;
  }
  __syncthreads();
  uint64_t v[kScanItems], sum = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = s_tile[threadIdx.x * kScanItems + i];
    sum += v[i];
  }
  uint64_t tot;
  uint64_t run = sums[blockIdx.x] + block_exclusive_scan(sum, s_warp, tot);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    s_tile[threadIdx.x * kScanItems + i] = run;
    run += v[i];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const uint64_t j = base + (uint64_t)i * kScanThreads + threadIdx.x;
    if (j < m) a[j] = s_tile[i * kScanThreads + threadIdx.x];
  }
}

// ---------------------------------------------------------------- fill
// rank -> slot: 32-bit map with a level table when n < 2^32 (IDX = uint32_t), the
// 64-bit closed form otherwise
template <int LAYOUT, int KF, class IDX>
__device__ __forceinline__ uint64_t slot_of(uint64_t r, const Geom& g, const SlotMap& sm) {
  if constexpr (LAYOUT == 0) return r;
  else if constexpr (sizeof(IDX) == 4) return slot_of_rank<LAYOUT == 1 ? 2 : KF>((uint32_t)r, sm);
  else if constexpr (LAYOUT == 1) return rank_to_slot<2>(r, g);
  else return rank_to_slot<KF>(r, g);
}

template <int LAYOUT, int KF, class IDX>
__device__ __forceinline__ uint32_t row_at(const uint32_t* __restrict__ rows, uint64_t r,
                                           const Geom& g, const SlotMap& sm) {
  const uint64_t s = slot_of<LAYOUT, KF, IDX>(r, g, sm);
  return s < g.n ? __ldg(rows + s) : GI_MISS;  // ranks are < n; the bound is a guard
}

// Rows of 32 consecutive ranges per warp.  Ranges of 32 rows or more are filled by
// the whole warp, one at a time (coalesced, the switch of Section 5.1).  The short
// ones are filled cooperatively: their rows, concatenated, are dealt to the lanes
// (32 independent loads in flight), each lane finding its row's range by a 5-step
// search over the lanes' running counts (the last range starting at or before the
// row; an empty range shares its start with the next one, which wins).
template <int LAYOUT, int KF, class IDX>
__global__ void __launch_bounds__(256) k_range_fill(const uint32_t* __restrict__ rows, Geom g,
                                                    SlotMap sm,
                                                    const uint64_t* __restrict__ offsets,
                                                    const uint64_t* __restrict__ lo_rank,
                                                    uint64_t m, uint32_t* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w * 32 < m;
       w += warps) {
    const uint64_t i = w * 32 + lane;
    uint64_t off = 0, cnt = 0, r0 = 0;
    if (i < m) {
      off = offsets[i];
      cnt = offsets[i + 1] - off;
      r0 = lo_rank[i];
    }
    const bool big = cnt >= 32;
    uint32_t bigmask = __ballot_sync(0xffffffffu, big);
    while (bigmask) {
      const int b = __ffs(bigmask) - 1;
      bigmask &= bigmask - 1;
      const uint64_t bo = __shfl_sync(0xffffffffu, off, b);
      const uint64_t bc = __shfl_sync(0xffffffffu, cnt, b);
      const uint64_t br = __shfl_sync(0xffffffffu, r0, b);
      for (uint64_t j = lane; j < bc; j += 32) out[bo + j] = row_at<LAYOUT, KF, IDX>(rows, br + j, g, sm);
    }
    // short ranges: running count of their rows over the lanes
    uint32_t c = big ? 0u : (uint32_t)cnt, x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    const uint32_t rel = x - c;  // rows of the short ranges before this lane's
    const uint32_t total = __shfl_sync(0xffffffffu, x, 31);
    for (uint32_t row0 = 0; row0 < total; row0 += 32) {  // warp-uniform: the shuffles need all lanes
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
      if (row < total) out[o] = row_at<LAYOUT, KF, IDX>(rows, r, g, sm);
    }
  }
}

// ---------------------------------------------------------------- fill by level runs
// Ranks < r that the complete k-ary tree stores on level l.  The bottom level
// holds the ranks r' with r' mod k != k-1 until its b keys are used up, so
// nb(r) = min(b, r - floor(r/k)) of them lie below r.  The other Q = r - nb(r)
// ranks are the upper levels' keys in order; in the perfect upper tree, the
// (x)th of them (x = 1..) sits on level m-1-v, where v is the number of trailing
// zeros of x in base k.  So level l holds floor(Q/k^j) - floor(Q/k^(j+1)) of
// them, with j = m-1-l.
template <int KF>
__device__ __forceinline__ uint64_t level_rank_count(uint64_t r, uint32_t l, const Geom& g) {
  const uint64_t k = KF ? (uint64_t)KF : (uint64_t)g.k;
  uint64_t nb = r - r / k;
  if (nb > g.b) nb = g.b;
  if (l == g.m) return nb;
  const uint64_t Q = r - nb;
  const uint64_t kj = kpow<KF>(g.m - 1 - l, g);
  return Q / kj - Q / (kj * k);
}

// The rows of a range, level by level (Section 5): on every level the keys of
// [lo_rank, hi_rank) occupy one contiguous run of slots, whose ends follow from
// level_rank_count, so no key is read.  Each row goes to its key-order position
// offset + p'(slot) - lo_rank.  A lane handles its own range's short runs; runs
// of 32 slots or more are taken by the whole warp with coalesced reads, one at a
// time -- the single-thread / warp switch of Section 5.1, made per level.
template <int KF>
__global__ void __launch_bounds__(256) k_range_fill_levels(const uint32_t* __restrict__ rows, Geom g,
                                                           const uint64_t* __restrict__ offsets,
                                                           const uint64_t* __restrict__ lo_rank,
                                                           uint64_t m, uint32_t* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w * 32 < m; w += warps) {
    const uint64_t i = w * 32 + lane;
    uint64_t off = 0, cnt = 0, r0 = 0;
    if (i < m) {
      off = offsets[i];
      cnt = offsets[i + 1] - off;
      r0 = lo_rank[i];
    }
    const uint64_t r1 = r0 + cnt;
    for (uint32_t l = 0; l < g.levels; ++l) {
      uint64_t a = 0, len = 0;
      if (cnt) {
        a = level_rank_count<KF>(r0, l, g);
        len = level_rank_count<KF>(r1, l, g) - a;
      }
      const uint64_t start = (l == g.m ? g.top : kpow<KF>(l, g) - 1) + a;
      const bool big = len >= 32;
      if (!big) {
        for (uint64_t j = 0; j < len; ++j) {
          const uint64_t s = start + j;
          out[off + slot_to_rank<KF>(s, g) - r0] = __ldg(rows + s);
        }
      }
      uint32_t bm = __ballot_sync(0xffffffffu, big);
      while (bm) {
        const int b = __ffs(bm) - 1;
        bm &= bm - 1;
        const uint64_t bs = __shfl_sync(0xffffffffu, start, b);
        const uint64_t bl = __shfl_sync(0xffffffffu, len, b);
        const uint64_t bo = __shfl_sync(0xffffffffu, off - r0, b);
        for (uint64_t j = lane; j < bl; j += 32) {
          const uint64_t s = bs + j;
          out[bo + slot_to_rank<KF>(s, g)] = __ldg(rows + s);
        }
      }
    }
  }
}

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace rg
}  // namespace gi
