// Build path: key-value radix sort of (key, rowID) pairs into the sorted order
// and, for the Eytzinger layouts, into the closed-form permutation of that order.
//
// The paper builds the sorted array with a library key-value sort (Section 3)
// and moves it into Eytzinger order with one thread per target slot, each
// computing the source position p'(t) in closed form and copying one entry
// (Section 4, generalised to k in Section 6.1).  Here the sort is our own:
//
//   1. sort_prepare: one read of the keys computes the 256-bin histogram of
//      every 8-bit digit at once and scans each into global digit offsets.
//      Digits that are the same for every key are skipped by every later pass.
//   2. Default for large u64 inputs, the hybrid sort (hybrid_sort): one or two
//      stable MSD scatters on the top non-trivial digits (a plain pass, then a
//      pass segmented by first-level bucket), after which every bucket holds at
//      most 5120 pairs and is sorted by one CTA in shared memory
//      (gi_local_sort.cu), which writes each pair straight to its layout slot.
//   3. Otherwise (small or narrow inputs, or a bucket too large: the LSD
//      fallback) sort_pass once per remaining digit: a single-pass "onesweep"
//      scatter.  Each CTA takes the next tile in launch order, ranks its keys
//      stably by digit with warp ballots, publishes its per-digit counts and
//      finds its global offsets by decoupled look-back over earlier tiles (a
//      bounded wait), then writes keys and rowIDs through shared memory so that
//      each digit's run leaves the SM as consecutive addresses.  Then
//      layout_gather: slot t <- sorted[p'(t)], one read and one write per entry,
//      fused with the duplicate-key check.
//   The batched form (many indexes at once) uses the same passes segmented by
//   index, on plans written on the device (gi_batch.cu).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "gi_internal.cuh"

namespace gi {

namespace {

constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;

template <class K>
struct SortTile;
template <>
struct SortTile<uint32_t> {
  static constexpr int kItems = 16;
};
template <>
struct SortTile<uint64_t> {
  static constexpr int kItems = 12;
};

// Status word of the look-back: [63:62] flag, [61:40] epoch, [39:0] count.
constexpr uint64_t kStatAggregate = 1ull << 62;
constexpr uint64_t kStatInclusive = 2ull << 62;
constexpr uint64_t kValueMask = (1ull << 40) - 1;

// Tickets -> tiles of a subset of a batch's indexes: ticket t < *count is tile
// list[t] (the listed indexes' tiles in index order, written on the device).
// list == NULL: tile = ticket.
struct TileMap {
  const uint32_t* list;
  const uint32_t* count;
};

__device__ __forceinline__ uint64_t ld_volatile_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_volatile_u64(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// The 8-bit window just below the highest bit in which two keys differ: the
// first MSD scatter of the hybrid sort (so that no bit of it is wasted on bits
// every key shares, as the top byte of keys below 2^63 would).
struct Window {
  unsigned long long xor_or;  // OR over the keys of key ^ keys[0]
  uint32_t shift;             // the window is bits [shift, shift + 8)
  uint32_t trivial;           // 1 if every key has the same window value
  unsigned long long hist[kRadix];
  unsigned long long offs[kRadix];
};

__host__ __device__ inline uint32_t window_shift(unsigned long long xor_or) {
  if (!xor_or) return 0;
#ifdef __CUDA_ARCH__
  const int hb = 63 - __clzll((long long)xor_or);
#else
  const int hb = 63 - __builtin_clzll(xor_or);
#endif
  return hb >= 7 ? (uint32_t)(hb - 7) : 0u;
}

// Scratch layout (bytes, each region 256-aligned):
//   hist    [passes][256] u64   digit counts
//   offs    [passes][256] u64   exclusive digit offsets
//   trivial [passes]      u32   1 if one digit holds every key
//   counter [passes + 1]  u32   tile tickets (the last: the window pass)
//   win     Window              the window's counts, offsets and shift
//   status  [tiles][256]  u64   look-back words (epoch = pass + 1)
struct ScratchView {
  unsigned long long* hist;
  unsigned long long* offs;
  uint32_t* trivial;
  uint32_t* counter;
  Window* win;
  uint64_t* status;
};

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

inline uint64_t tiles_for(uint64_t n, int key_bytes) {
  const uint64_t tile = (uint64_t)kSortThreads *
                        (key_bytes == 4 ? SortTile<uint32_t>::kItems : SortTile<uint64_t>::kItems);
  return (n + tile - 1) / tile;
}

inline ScratchView view(void* scratch, int key_bytes) {
  const int passes = key_bytes;  // 8-bit digits
  char* p = (char*)scratch;
  ScratchView v;
  v.hist = (unsigned long long*)p;
  p += align256(sizeof(uint64_t) * passes * kRadix);
  v.offs = (unsigned long long*)p;
  p += align256(sizeof(uint64_t) * passes * kRadix);
  v.trivial = (uint32_t*)p;
  p += align256(sizeof(uint32_t) * passes);
  v.counter = (uint32_t*)p;
  p += align256(sizeof(uint32_t) * (passes + 1));
  v.win = (Window*)p;
  p += align256(sizeof(Window));
  v.status = (uint64_t*)p;
  return v;
}

inline size_t header_bytes(int key_bytes) {
  const int passes = key_bytes;
  return 2 * align256(sizeof(uint64_t) * passes * kRadix) + align256(sizeof(uint32_t) * passes) +
         align256(sizeof(uint32_t) * (passes + 1)) + align256(sizeof(Window));
}

// ---------------------------------------------------------------- histogram
// All digit histograms in one read of the keys.  With copy_to set, the keys are
// read from page-locked host memory and written to copy_to on the way (the
// host-to-device copy and the histogram in one pass over the bus).
template <class K>
__device__ __forceinline__ void count_digits(uint32_t (*sh)[kRadix], K key) {
#pragma unroll
  for (int p = 0; p < (int)sizeof(K); ++p) atomicAdd(&sh[p][(uint32_t)(key >> (8 * p)) & 0xFF], 1u);
}

// COUNT = false: only the OR of key ^ keys[0] (and the copy); the digit counts are
// taken later, and only if the LSD passes need them.
template <class K, bool COUNT = true>
__global__ void __launch_bounds__(256) k_histogram(const K* __restrict__ keys,
                                                   K* __restrict__ copy_to, uint64_t n,
                                                   unsigned long long* __restrict__ hist,
                                                   unsigned long long* __restrict__ xor_or) {
  constexpr int P = sizeof(K);
  constexpr int V = 16 / sizeof(K);  // keys per 16-byte load
  __shared__ uint32_t sh[P][kRadix];
  __shared__ unsigned long long s_or;
  for (int i = threadIdx.x; i < P * kRadix; i += blockDim.x) (&sh[0][0])[i] = 0;
  if (threadIdx.x == 0) s_or = 0;
  __syncthreads();
  const K k0 = n ? keys[0] : K(0);
  K acc = 0;  // OR of key ^ keys[0]: the bits in which two keys differ
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // 16-byte loads, two in flight per thread, when both pointers allow them
  const bool vec = ((uintptr_t)keys % 16 == 0) && ((uintptr_t)copy_to % 16 == 0);
  const uint64_t nv = vec ? n / V : 0;
  const uint4* kv = (const uint4*)keys;
  uint4* cv = (uint4*)copy_to;
  uint64_t i = gtid;
  for (; i + stride < nv; i += 2 * stride) {
    const uint4 a = kv[i], b = kv[i + stride];
    if (copy_to) {
      cv[i] = a;
      cv[i + stride] = b;
    }
    const K* ka = (const K*)&a;
    const K* kb = (const K*)&b;
#pragma unroll
    for (int j = 0; j < V; ++j) {
      if (COUNT) {
        count_digits<K>(sh, ka[j]);
        count_digits<K>(sh, kb[j]);
      }
      acc |= (ka[j] ^ k0) | (kb[j] ^ k0);
    }
  }
  for (; i < nv; i += stride) {
    const uint4 a = kv[i];
    if (copy_to) cv[i] = a;
    const K* ka = (const K*)&a;
#pragma unroll
    for (int j = 0; j < V; ++j) {
      if (COUNT) count_digits<K>(sh, ka[j]);
      acc |= ka[j] ^ k0;
    }
  }
  for (uint64_t t = nv * V + gtid; t < n; t += stride) {  // the rest one key at a time
    const K key = keys[t];
    if (copy_to) copy_to[t] = key;
    if (COUNT) count_digits<K>(sh, key);
    acc |= key ^ k0;
  }
  unsigned long long x = (unsigned long long)acc;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x |= __shfl_xor_sync(0xffffffffu, x, o);
  if ((threadIdx.x & 31) == 0 && x) atomicOr(&s_or, x);
  __syncthreads();
  if (COUNT)
    for (int i = threadIdx.x; i < P * kRadix; i += blockDim.x) {
      const uint32_t c = (&sh[0][0])[i];
      if (c) atomicAdd(&hist[i], (unsigned long long)c);
    }
  if (threadIdx.x == 0 && s_or) atomicOr(xor_or, s_or);
}

// Counts of the window (Window) over all keys; the window's shift comes from
// xor_or, which k_histogram has finished.  Block 0 publishes the shift.
// Keys differing in fewer than min_bytes bytes are not sorted by the hybrid sort:
// block 0 marks the window trivial then, so the window pass queued behind skips.
template <class K>
__global__ void __launch_bounds__(256) k_window_hist(const K* __restrict__ keys, uint64_t n,
                                                     Window* __restrict__ win, uint32_t min_bytes) {
  __shared__ uint32_t sh[kRadix];
  sh[threadIdx.x] = 0;
  __syncthreads();
  const unsigned long long xo = win->xor_or;
  const uint32_t sw = window_shift(xo);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    win->shift = sw;
    uint32_t bytes = 0;
    for (int p = 0; p < (int)sizeof(K); ++p) bytes += ((xo >> (8 * p)) & 0xFF) ? 1u : 0u;
    if (bytes < min_bytes) win->trivial = 1;
  }
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + 3 * stride < n; i += 4 * stride) {  // four loads in flight
    const K a = keys[i], b = keys[i + stride], c = keys[i + 2 * stride], d = keys[i + 3 * stride];
    atomicAdd(&sh[(uint32_t)(a >> sw) & 0xFF], 1u);
    atomicAdd(&sh[(uint32_t)(b >> sw) & 0xFF], 1u);
    atomicAdd(&sh[(uint32_t)(c >> sw) & 0xFF], 1u);
    atomicAdd(&sh[(uint32_t)(d >> sw) & 0xFF], 1u);
  }
  for (; i < n; i += stride) atomicAdd(&sh[(uint32_t)(keys[i] >> sw) & 0xFF], 1u);
  __syncthreads();
  const uint32_t c = sh[threadIdx.x];
  if (c) atomicAdd(&win->hist[threadIdx.x], (unsigned long long)c);
}

// The reserved-rowID check on its own, for a build in which no sort pass reads
// the input rowIDs (every key equal).
__global__ void __launch_bounds__(256) k_check_rows(const uint32_t* __restrict__ rows, uint64_t n,
                                                    uint32_t* __restrict__ flags) {
  bool bad = false;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    bad |= rows[i] == GI_MISS;
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flags, kFlagReservedRowid);
}

// One block per pass: exclusive scan of the 256 digit counts.
__global__ void __launch_bounds__(256) k_scan_hist(const unsigned long long* __restrict__ hist,
                                                   unsigned long long* __restrict__ offs,
                                                   uint32_t* __restrict__ trivial, uint64_t n) {
  __shared__ unsigned long long warp_tot[8];
  __shared__ uint32_t any_full;
  const int p = blockIdx.x, d = threadIdx.x, lane = d & 31, w = d >> 5;
  if (d == 0) any_full = 0;
  __syncthreads();
  const unsigned long long c = hist[p * kRadix + d];
  if (c == n) atomicOr(&any_full, 1u);
  unsigned long long x = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  unsigned long long base = 0;
  for (int i = 0; i < w; ++i) base += warp_tot[i];
  offs[p * kRadix + d] = base + x - c;
  __syncthreads();
  if (d == 0 && any_full) trivial[p] = 1;  // (the flags start zeroed)
}

// ---------------------------------------------------------------- one onesweep pass
template <class K>
__global__ void __launch_bounds__(kSortThreads, 5) k_sort_pass(
    const K* __restrict__ src_k, const uint32_t* __restrict__ src_v, K* __restrict__ dst_k,
    uint32_t* __restrict__ dst_v, uint64_t n, uint32_t shift,
    const unsigned long long* __restrict__ digit_off, uint64_t* __restrict__ status,
    uint32_t* __restrict__ tile_counter, uint32_t epoch, uint32_t* __restrict__ flags,
    uint32_t check_rows, const uint32_t* __restrict__ skip_if,
    const uint32_t* __restrict__ shift_ptr) {
  constexpr int ITEMS = SortTile<K>::kItems;
  constexpr int TILE = kSortThreads * ITEMS;
  if (skip_if && *skip_if) return;  // a speculative pass on a digit that turned out trivial
  if (shift_ptr) shift = *shift_ptr;  // the window pass: its shift was written on the device
  // keys and rowIDs have their own exchange arrays, so one final loop writes both;
  // the per-warp digit counters share space with the rowIDs (dead by then)
  union HistOrVals {
    uint32_t h[kSortWarps][kRadix];
    uint32_t vals[TILE];
  };
  __shared__ K s_keys[TILE];
  __shared__ HistOrVals hv;
  __shared__ uint32_t s_start[kRadix];            // tile-local start of each digit's run
  __shared__ unsigned long long s_gbase[kRadix];  // global position of local position 0 per digit
  __shared__ uint32_t s_warp_tot[kSortWarps];
  __shared__ uint32_t s_tile;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_tile = atomicAdd(tile_counter, 1u);
  for (int i = lane; i < kRadix; i += 32) hv.h[warp][i] = 0;
  __syncthreads();
  const uint64_t tile = s_tile;
  const uint64_t tile_base = tile * TILE;
  const uint32_t valid = (uint32_t)((n - tile_base) < (uint64_t)TILE ? (n - tile_base) : TILE);

  // Warp-striped ownership: item i of lane l in warp w is tile element
  // w*32*ITEMS + i*32 + l, so tile order is (warp, item, lane).
  K key[ITEMS];
  uint32_t rnk[ITEMS];
  const uint64_t wbase = tile_base + (uint64_t)warp * 32 * ITEMS + lane;
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const uint64_t idx = wbase + (uint64_t)i * 32;
    key[i] = idx < n ? src_k[idx] : ~K(0);  // padding sorts last (digit 255, after real keys)
  }
  const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const uint32_t d = (uint32_t)(key[i] >> shift) & 0xFF;
    uint32_t peers = 0xffffffffu;  // lanes holding the same digit, from one ballot per bit
#pragma unroll
    for (int b = 0; b < kRadixBits; ++b) {
      const uint32_t bit = (d >> b) & 1u;
      peers &= ~(__ballot_sync(0xffffffffu, bit) ^ (0u - bit));  // lanes agreeing on bit b
    }
    const uint32_t before = __popc(peers & lt_mask);
    const uint32_t leader = 31 - __clz(peers);
    const uint32_t base = hv.h[warp][d];
    __syncwarp();
    if (lane == leader) hv.h[warp][d] = base + __popc(peers);
    __syncwarp();
    rnk[i] = base + before;
  }
  __syncthreads();

  // Thread d owns digit d: exclusive prefix over warps, tile count.
  const uint32_t d = tid;
  uint32_t cnt = 0;
#pragma unroll
  for (int w = 0; w < kSortWarps; ++w) {
    const uint32_t c = hv.h[w][d];
    hv.h[w][d] = cnt;
    cnt += c;
  }
  const uint32_t cnt_valid = (d == kRadix - 1) ? cnt - (TILE - valid) : cnt;
  uint64_t* my_status = status + tile * kRadix + d;
  const uint64_t ep = (uint64_t)epoch << 40;
  st_volatile_u64(my_status, (tile == 0 ? kStatInclusive : kStatAggregate) | ep | cnt_valid);

  // Block-wide exclusive scan of the per-digit tile counts -> run starts.
  uint32_t x = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp_tot[warp] = x;
  __syncthreads();
  uint32_t wpre = 0;
#pragma unroll
  for (int w = 0; w < kSortWarps; ++w) wpre += (w < warp) ? s_warp_tot[w] : 0u;
  const uint32_t start = wpre + x - cnt;
  s_start[d] = start;

  // Decoupled look-back over earlier tiles for digit d (bounded wait).
  uint64_t excl = 0;
  if (tile > 0) {
    int64_t j = (int64_t)tile - 1;
    uint32_t spins = 0;
    while (j >= 0) {
      const uint64_t s = ld_volatile_u64(status + (uint64_t)j * kRadix + d);
      const bool ready = ((s >> 40) & 0x3FFFFF) == epoch && (s >> 62) != 0;
      if (ready) {
        excl += s & kValueMask;
        if ((s >> 62) == 2) break;
        --j;
      } else {
        if (++spins > kSpinLimit) {
          atomicOr(flags, kFlagTimeout);
          break;
        }
        __nanosleep(64);
      }
    }
    st_volatile_u64(my_status, kStatInclusive | ep | (excl + cnt_valid));
  }
  s_gbase[d] = digit_off[d] + excl - start;
  __syncthreads();

  // Local sorted position of every key: its digit's run start + earlier warps'
  // count of that digit + its rank within its warp.
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const uint32_t dd = (uint32_t)(key[i] >> shift) & 0xFF;
    rnk[i] += s_start[dd] + hv.h[warp][dd];
    s_keys[rnk[i]] = key[i];
  }
  __syncthreads();  // the digit counters are dead: their space takes the rowIDs
  bool bad = false;  // a rowID equal to the reserved miss value (first pass only)
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const uint64_t idx = wbase + (uint64_t)i * 32;
    const uint32_t v = idx < n ? src_v[idx] : 0u;
    bad |= check_rows && idx < n && v == GI_MISS;
    hv.vals[rnk[i]] = v;
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(flags, kFlagReservedRowid);
  __syncthreads();

  // Consecutive threads take consecutive local positions: each digit run goes
  // to consecutive global addresses, keys and rowIDs alike.
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
    const uint32_t j = tid + r * kSortThreads;
    if (j < valid) {
      const K kk = s_keys[j];
      const uint64_t dst = s_gbase[(uint32_t)(kk >> shift) & 0xFF] + j;
      if (dst < n) {  // the bound only guards a failed wait
        dst_k[dst] = kk;
        dst_v[dst] = hv.vals[j];
      }
    }
  }
}

// ---------------------------------------------------------------- layout permutation
// Slot t <- sorted[p'(t)] (Sections 4, 6.1).  key_off = 1 for Eytzinger order,
// whose slot 0 is the empty slot.  Also flags equal neighbours in sorted order.
template <class K, int KF>
__global__ void __launch_bounds__(256) k_layout_gather(const K* __restrict__ sk,
                                                       const uint32_t* __restrict__ sv,
                                                       K* __restrict__ dk, uint32_t* __restrict__ dv,
                                                       Geom g, uint32_t key_off,
                                                       uint32_t* __restrict__ flags) {
  bool dup = false;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < g.n; t += stride) {
    const uint64_t r = slot_to_rank<KF>(t, g);
    const K key = sk[r];
    dk[t + key_off] = key;
    dv[t] = sv[r];
    if (r > 0) dup |= sk[r - 1] == key;
  }
  if (key_off && blockIdx.x == 0 && threadIdx.x == 0) dk[0] = K(0);
  if (__any_sync(0xffffffffu, dup) && (threadIdx.x & 31) == 0) atomicOr(flags, kFlagDuplicate);
}

template <class K>
__global__ void __launch_bounds__(256) k_sorted_dups(const K* __restrict__ sk, uint64_t n,
                                                     uint32_t* __restrict__ flags) {
  bool dup = false;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x + 1; i < n; i += stride)
    dup |= sk[i - 1] == sk[i];
  if (__any_sync(0xffffffffu, dup) && (threadIdx.x & 31) == 0) atomicOr(flags, kFlagDuplicate);
}

inline int grid_for(uint64_t work, int block, int per_sm = 8) {
  const uint64_t want = (work + block - 1) / block;
  const uint64_t cap = (uint64_t)sm_count() * per_sm;
  return (int)(want < cap ? (want ? want : 1) : cap);
}

// ================================================================= batched form
// Many independent indexes sorted at once.  Every tile belongs to one index; the
// look-back stops at its index's first tile, and each index has its own digit
// offsets, so keys never leave their index (a segmented LSD sort).

// plan != NULL: only the indexes of plan kPlanLsd, and no rowID check (their
// first LSD pass checks them)
template <class K>
__global__ void __launch_bounds__(256) k_batch_histogram(const K* __restrict__ keys,
                                                         const uint32_t* __restrict__ rows,
                                                         const BatchTile* __restrict__ chunks,
                                                         uint64_t nchunks,
                                                         unsigned long long* __restrict__ hist,
                                                         uint32_t* __restrict__ flags,
                                                         const BatchPlan* __restrict__ plan) {
  constexpr int P = sizeof(K);
  __shared__ uint32_t sh[P][kRadix];
  bool bad = false;
  for (uint64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const BatchTile t = chunks[c];
    if (plan && plan[t.seg].mode != kPlanLsd) continue;
    for (int i = threadIdx.x; i < P * kRadix; i += blockDim.x) (&sh[0][0])[i] = 0;
    __syncthreads();
    const K* kp = keys + t.start;
    const uint32_t* rp = rows + t.start;
    uint32_t i = threadIdx.x;
    for (; i + 3 * blockDim.x < t.count; i += 4 * blockDim.x) {  // four keys in flight
      K kk[4];
      uint32_t rr[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        kk[u] = kp[i + u * blockDim.x];
        rr[u] = plan ? 0u : rp[i + u * blockDim.x];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
#pragma unroll
        for (int p = 0; p < P; ++p) atomicAdd(&sh[p][(uint32_t)(kk[u] >> (8 * p)) & 0xFF], 1u);
        bad |= rr[u] == GI_MISS;
      }
    }
    for (; i < t.count; i += blockDim.x) {
      const K key = kp[i];
#pragma unroll
      for (int p = 0; p < P; ++p) atomicAdd(&sh[p][(uint32_t)(key >> (8 * p)) & 0xFF], 1u);
      bad |= !plan && rp[i] == GI_MISS;
    }
    __syncthreads();
    unsigned long long* h = hist + (uint64_t)t.seg * P * kRadix;
    for (int i = threadIdx.x; i < P * kRadix; i += blockDim.x) {
      const uint32_t v = (&sh[0][0])[i];
      if (v) atomicAdd(&h[i], (unsigned long long)v);
    }
    __syncthreads();
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flags, kFlagReservedRowid);
}

// one CTA per index: exclusive digit scans of every pass, offset by the index start
__global__ void __launch_bounds__(256) k_batch_scan_hist(const unsigned long long* __restrict__ hist,
                                                         unsigned long long* __restrict__ offs,
                                                         const uint64_t* __restrict__ seg_start,
                                                         int passes) {
  __shared__ unsigned long long warp_tot[8];
  const int d = threadIdx.x, lane = d & 31, w = d >> 5;
  const uint64_t seg = blockIdx.x;
  for (int p = 0; p < passes; ++p) {
    const uint64_t at = (seg * passes + p) * kRadix + d;
    const unsigned long long c = hist[at];
    unsigned long long x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    unsigned long long base = 0;
    for (int i = 0; i < w; ++i) base += warp_tot[i];
    offs[at] = seg_start[seg] + base + x - c;
    __syncthreads();
  }
}

template <class K>
__global__ void __launch_bounds__(kSortThreads, 5) k_batch_sort_pass(
    const K* __restrict__ src_k, const uint32_t* __restrict__ src_v, K* __restrict__ dst_k,
    uint32_t* __restrict__ dst_v, uint64_t n, uint32_t shift, const BatchTile* __restrict__ tiles,
    const unsigned long long* __restrict__ offs, int pass, int passes,
    uint64_t* __restrict__ status, uint32_t* __restrict__ tile_counter, uint32_t epoch,
    uint32_t* __restrict__ flags, const BatchPlan* __restrict__ plan, uint32_t want,
    uint32_t window, TileMap map, uint32_t check_rows) {
  constexpr int ITEMS = SortTile<K>::kItems;
  constexpr int TILE = kSortThreads * ITEMS;
  union HistOrVals {
    uint32_t h[kSortWarps][kRadix];
    uint32_t vals[TILE];
  };
  __shared__ K s_keys[TILE];
  __shared__ HistOrVals hv;
  __shared__ uint32_t s_start[kRadix];
  __shared__ unsigned long long s_gbase[kRadix];
  __shared__ uint32_t s_warp_tot[kSortWarps];
  __shared__ uint32_t s_tile;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t shift0 = shift;
  // Tickets are taken in order; with a map, ticket t is the t-th tile of the
  // indexes the map lists and the grid is persistent (a CTA takes tickets until
  // none is left), else one ticket per CTA.  A CTA waits in the look-back only
  // on tiles of lower tickets, held by CTAs that are running, so it always ends.
  for (;;) {
  if (tid == 0) s_tile = atomicAdd(tile_counter, 1u);
  for (int i = lane; i < kRadix; i += 32) hv.h[warp][i] = 0;
  __syncthreads();
  const uint32_t ticket = s_tile;
  uint64_t tile = ticket;
  if (map.list) {
    if (ticket >= *map.count) return;
    tile = map.list[ticket];
  }
  const BatchTile desc = tiles[tile];
  // with a plan, only the indexes sorted this way take part (a whole index is
  // skipped, so no tile of it is ever waited for)
  if (plan && plan[desc.seg].mode != want) {
    if (!map.list) return;
    __syncthreads();
    continue;
  }
  shift = (plan && window) ? plan[desc.seg].s1 : shift0;  // the index's MSD window
  const uint64_t tile_base = desc.start;
  const uint32_t valid = desc.count;
  const unsigned long long* digit_off = offs + ((uint64_t)desc.seg * passes + pass) * kRadix;

  K key[ITEMS];
  uint32_t rnk[ITEMS];
  const uint32_t wofs = (uint32_t)warp * 32 * ITEMS + lane;
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const uint32_t e = wofs + i * 32;
    key[i] = e < valid ? src_k[tile_base + e] : ~K(0);
  }
  const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const uint32_t d = (uint32_t)(key[i] >> shift) & 0xFF;
    uint32_t peers = 0xffffffffu;
#pragma unroll
    for (int b = 0; b < kRadixBits; ++b) {
      const uint32_t bit = (d >> b) & 1u;
      peers &= ~(__ballot_sync(0xffffffffu, bit) ^ (0u - bit));
    }
    const uint32_t before = __popc(peers & lt_mask);
    const uint32_t leader = 31 - __clz(peers);
    const uint32_t base = hv.h[warp][d];
    __syncwarp();
    if (lane == leader) hv.h[warp][d] = base + __popc(peers);
    __syncwarp();
    rnk[i] = base + before;
  }
  __syncthreads();

  const uint32_t d = tid;
  uint32_t cnt = 0;
#pragma unroll
  for (int w = 0; w < kSortWarps; ++w) {
    const uint32_t c = hv.h[w][d];
    hv.h[w][d] = cnt;
    cnt += c;
  }
  const uint32_t cnt_valid = (d == kRadix - 1) ? cnt - (TILE - valid) : cnt;
  uint64_t* my_status = status + tile * kRadix + d;
  const uint64_t ep = (uint64_t)epoch << 40;
  const bool first = desc.local == 0;
  st_volatile_u64(my_status, (first ? kStatInclusive : kStatAggregate) | ep | cnt_valid);

  uint32_t x = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp_tot[warp] = x;
  __syncthreads();
  uint32_t wpre = 0;
#pragma unroll
  for (int w = 0; w < kSortWarps; ++w) wpre += (w < warp) ? s_warp_tot[w] : 0u;
  const uint32_t start = wpre + x - cnt;
  s_start[d] = start;

  // look-back over the earlier tiles of the same index only
  uint64_t excl = 0;
  if (!first) {
    const int64_t stop = (int64_t)tile - desc.local;
    int64_t j = (int64_t)tile - 1;
    uint32_t spins = 0;
    while (j >= stop) {
      const uint64_t s = ld_volatile_u64(status + (uint64_t)j * kRadix + d);
      const bool ready = ((s >> 40) & 0x3FFFFF) == epoch && (s >> 62) != 0;
      if (ready) {
        excl += s & kValueMask;
        if ((s >> 62) == 2) break;
        --j;
      } else {
        if (++spins > kSpinLimit) {
          atomicOr(flags, kFlagTimeout);
          break;
        }
        __nanosleep(64);
      }
    }
    st_volatile_u64(my_status, kStatInclusive | ep | (excl + cnt_valid));
  }
  s_gbase[d] = digit_off[d] + excl - start;
  __syncthreads();

#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const uint32_t dd = (uint32_t)(key[i] >> shift) & 0xFF;
    rnk[i] += s_start[dd] + hv.h[warp][dd];
    s_keys[rnk[i]] = key[i];
  }
  __syncthreads();
  bool bad = false;  // a rowID equal to the reserved miss value (passes that read the input)
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const uint32_t e = wofs + i * 32;
    const uint32_t v = e < valid ? src_v[tile_base + e] : 0u;
    bad |= check_rows && e < valid && v == GI_MISS;
    hv.vals[rnk[i]] = v;
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(flags, kFlagReservedRowid);
  __syncthreads();
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
    const uint32_t j = tid + r * kSortThreads;
    if (j < valid) {
      const K kk = s_keys[j];
      const uint64_t dst = s_gbase[(uint32_t)(kk >> shift) & 0xFF] + j;
      if (dst < n) {
        dst_k[dst] = kk;
        dst_v[dst] = hv.vals[j];
      }
    }
  }
  if (!map.list) return;
  __syncthreads();  // shared memory is reused by the next ticket
  }
}

// slot t of index s <- sorted position slot_to_rank(t); k = 0: the sorted order itself
template <class K, int KF>
__global__ void __launch_bounds__(256) k_batch_gather(const K* __restrict__ sk,
                                                      const uint32_t* __restrict__ sv,
                                                      K* __restrict__ ok, uint32_t* __restrict__ ov,
                                                      const BatchTile* __restrict__ tiles,
                                                      uint64_t ntiles,
                                                      const uint64_t* __restrict__ seg_start,
                                                      const uint64_t* __restrict__ seg_base,
                                                      uint32_t k, uint32_t* __restrict__ flags,
                                                      const BatchPlan* __restrict__ plan,
                                                      TileMap map, const uint32_t* __restrict__ kidx) {
  bool dup = false;
  const uint64_t total = map.list ? *map.count : ntiles;
  for (uint64_t ti = blockIdx.x; ti < total; ti += gridDim.x) {
    const BatchTile t = tiles[map.list ? map.list[ti] : ti];
    if (plan && plan[t.seg].mode != kPlanLsd) continue;
    const uint64_t s0 = seg_start[t.seg];
    const uint64_t n = seg_start[t.seg + 1] - s0;
    const uint64_t out0 = seg_base[t.seg];
    // KF == 1 marks the sorted order; KF == -1 each index's own fan-out (0: sorted);
    // fan-outs below 2 never reach device_geom
    const uint32_t kk = KF == -1 ? kidx[t.seg] : k;
    const Geom g = device_geom(n, KF > 1 ? (uint32_t)KF : (kk >= 2 ? kk : 2u));
    for (uint32_t i = threadIdx.x; i < t.count; i += blockDim.x) {
      const uint64_t slot = t.start - s0 + i;
      uint64_t r;
      if constexpr (KF == 1) r = slot;
      else if constexpr (KF == -1) r = kk >= 2 ? slot_to_rank<0>(slot, g) : slot;
      else r = slot_to_rank<KF>(slot, g);
      const K key = sk[s0 + r];
      ok[out0 + slot] = key;
      ov[out0 + slot] = sv[s0 + r];
      if (r > 0) dup |= sk[s0 + r - 1] == key;
    }
  }
  if (__any_sync(0xffffffffu, dup) && (threadIdx.x & 31) == 0) atomicOr(flags, kFlagDuplicate);
}

// ---------------------------------------------------------------- hybrid batch build
// OR over every index of key ^ (the index's first key): its set bits are the bits
// in which two keys of the index differ.  One 64-bit atomic per CTA and chunk.
template <class K>
__global__ void __launch_bounds__(256) k_batch_xor(const K* __restrict__ keys,
                                                   const BatchTile* __restrict__ chunks,
                                                   uint64_t nchunks,
                                                   const uint64_t* __restrict__ seg_start,
                                                   unsigned long long* __restrict__ xor_or) {
  __shared__ unsigned long long s_or[8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (uint64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const BatchTile t = chunks[c];
    const K k0 = keys[seg_start[t.seg]];
    const K* kp = keys + t.start;
    K acc = 0;
    uint32_t i = threadIdx.x;
    for (; i + 3 * blockDim.x < t.count; i += 4 * blockDim.x)  // four loads in flight
      acc |= (kp[i] ^ k0) | (kp[i + blockDim.x] ^ k0) | (kp[i + 2 * blockDim.x] ^ k0) |
             (kp[i + 3 * blockDim.x] ^ k0);
    for (; i < t.count; i += blockDim.x) acc |= kp[i] ^ k0;
    unsigned long long x = (unsigned long long)acc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x |= __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) s_or[w] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long y = 0;
      for (int j = 0; j < (int)(blockDim.x >> 5); ++j) y |= s_or[j];
      if (y) atomicOr(&xor_or[t.seg], y);
    }
    __syncthreads();
  }
}

// One thread per index: from the bits in which its keys differ (highest: hb), the
// plan: at most `cap` pairs -> one CTA sorts the whole index (top window = its 8
// highest significant bits); more -> one stable scatter on a window of w bits
// ending at hb (the MSD window), then buckets with the next 8 bits as their top
// window.  The k-ary slot map of the index goes to maps[i].
__global__ void __launch_bounds__(256) k_batch_plan(const unsigned long long* __restrict__ xor_or,
                                                    const uint64_t* __restrict__ seg_start,
                                                    uint32_t nseg, int key_bytes, uint32_t k,
                                                    const uint32_t* __restrict__ kidx,
                                                    uint32_t cap, BatchPlan* __restrict__ plan,
                                                    SlotMap* __restrict__ maps) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nseg) return;
  const uint64_t n = seg_start[i + 1] - seg_start[i];
  const unsigned long long x = n ? xor_or[i] : 0ull;
  BatchPlan pl{};
  for (int p = 0; p < key_bytes; ++p)
    if ((x >> (8 * p)) & 0xFF) pl.lsd_mask |= 1u << p;
  const int hb = x ? 63 - __clzll((long long)x) : -1;  // highest bit in which two keys differ
  if (n == 0) {
    pl.mode = kPlanEmpty;
  } else if (n <= cap) {
    pl.mode = kPlanWhole;
    pl.ts = hb >= 7 ? (uint32_t)hb - 7 : 0u;
  } else {
    // MSD window of w bits, w just large enough for buckets of about 2048 pairs
    // (more buckets only add per-bucket work); bits above hb are common to all
    // keys, so an 8-bit digit at s1 = hb + 1 - w takes 2^w values
    pl.mode = kPlanMsd;  // kPlanLsd if a window bucket turns out larger than cap
    uint32_t w = 1;
    while (w < 8 && (n >> w) > 2048) ++w;
    pl.s1 = hb + 1 >= (int)w ? (uint32_t)(hb + 1 - (int)w) : 0u;
    pl.ts = pl.s1 >= 8 ? pl.s1 - 8 : 0u;
  }
  plan[i] = pl;
  // k == kBatchMixed: each index's own fan-out (its map's k = 0 marks the sorted layout)
  const uint32_t ki = k == kBatchMixed ? kidx[i] : k;
  if (ki >= 2 && n > 0 && n < (1ull << 32)) fill_slot_map(maps[i], device_geom(n, ki));
  else if (k == kBatchMixed) maps[i].k = 0;
}

// Counts of the MSD window per index (indexes of plan kPlanMsd only).
template <class K>
__global__ void __launch_bounds__(256) k_batch_window_hist(const K* __restrict__ keys,
                                                           const BatchTile* __restrict__ chunks,
                                                           uint64_t nchunks,
                                                           const BatchPlan* __restrict__ plan,
                                                           unsigned long long* __restrict__ hist) {
  __shared__ uint32_t sh[kRadix];
  for (uint64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const BatchTile t = chunks[c];
    const BatchPlan pl = plan[t.seg];
    if (pl.mode != kPlanMsd) continue;
    sh[threadIdx.x] = 0;
    __syncthreads();
    const K* kp = keys + t.start;
    uint32_t i = threadIdx.x;
    for (; i + 3 * blockDim.x < t.count; i += 4 * blockDim.x) {  // four loads in flight
      const K a = kp[i], b = kp[i + blockDim.x], c2 = kp[i + 2 * blockDim.x], d = kp[i + 3 * blockDim.x];
      atomicAdd(&sh[(uint32_t)(a >> pl.s1) & 0xFF], 1u);
      atomicAdd(&sh[(uint32_t)(b >> pl.s1) & 0xFF], 1u);
      atomicAdd(&sh[(uint32_t)(c2 >> pl.s1) & 0xFF], 1u);
      atomicAdd(&sh[(uint32_t)(d >> pl.s1) & 0xFF], 1u);
    }
    for (; i < t.count; i += blockDim.x) atomicAdd(&sh[(uint32_t)(kp[i] >> pl.s1) & 0xFF], 1u);
    __syncthreads();
    const uint32_t v = sh[threadIdx.x];
    if (v) atomicAdd(&hist[(uint64_t)t.seg * kRadix + threadIdx.x], (unsigned long long)v);
    __syncthreads();
  }
}

// One CTA: tile-count prefixes of the kPlanMsd and of the kPlanLsd indexes (the
// ticket maps of the MSD pass and of the LSD passes / permutation).
__global__ void __launch_bounds__(1024) k_batch_mode_prefix(const BatchPlan* __restrict__ plan,
                                                            const uint32_t* __restrict__ tile0,
                                                            uint32_t nseg,
                                                            uint32_t* __restrict__ prefix_msd,
                                                            uint32_t* __restrict__ prefix_lsd) {
  __shared__ uint32_t warp_tot[2][32];
  __shared__ uint32_t carry[2];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid == 0) carry[0] = carry[1] = 0;
  __syncthreads();
  for (uint32_t base = 0; base < nseg; base += blockDim.x) {
    const uint32_t s = base + tid;
    uint32_t v[2] = {0, 0};
    if (s < nseg) {
      const uint32_t nt = tile0[s + 1] - tile0[s];
      const uint32_t mode = plan[s].mode;
      v[0] = mode == kPlanMsd ? nt : 0u;
      v[1] = mode == kPlanLsd ? nt : 0u;
    }
    uint32_t x[2] = {v[0], v[1]};
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x[c], o);
        if (lane >= o) x[c] += y;
      }
    }
    if (lane == 31) {
      warp_tot[0][w] = x[0];
      warp_tot[1][w] = x[1];
    }
    __syncthreads();
    uint32_t pre[2] = {carry[0], carry[1]};
    for (int j = 0; j < w; ++j) {
      pre[0] += warp_tot[0][j];
      pre[1] += warp_tot[1][j];
    }
    if (s < nseg) {
      prefix_msd[s] = pre[0] + x[0] - v[0];
      prefix_lsd[s] = pre[1] + x[1] - v[1];
    }
    __syncthreads();
    if (tid == (int)blockDim.x - 1) {  // the block total carries to the next chunk
      carry[0] = pre[0] + x[0];
      carry[1] = pre[1] + x[1];
    }
    __syncthreads();
  }
  if (tid == 0) {
    prefix_msd[nseg] = carry[0];
    prefix_lsd[nseg] = carry[1];
  }
}

// One CTA per index: its tiles into the ticket list of its plan (MSD or LSD).
__global__ void __launch_bounds__(256) k_batch_mode_lists(const BatchPlan* __restrict__ plan,
                                                          const uint32_t* __restrict__ tile0,
                                                          const uint32_t* __restrict__ prefix_msd,
                                                          const uint32_t* __restrict__ prefix_lsd,
                                                          uint32_t* __restrict__ list_msd,
                                                          uint32_t* __restrict__ list_lsd) {
  const uint32_t s = blockIdx.x;
  const uint32_t mode = plan[s].mode;
  if (mode != kPlanMsd && mode != kPlanLsd) return;
  uint32_t* out = mode == kPlanMsd ? list_msd + prefix_msd[s] : list_lsd + prefix_lsd[s];
  const uint32_t t0 = tile0[s], nt = tile0[s + 1] - t0;
  for (uint32_t j = threadIdx.x; j < nt; j += blockDim.x) out[j] = t0 + j;
}

// One CTA per index of plan kPlanMsd: absolute starts of its window buckets, and
// the fallback to the LSD passes if one of them is larger than cap.
__global__ void __launch_bounds__(256) k_batch_window_scan(const unsigned long long* __restrict__ hist,
                                                           unsigned long long* __restrict__ offs,
                                                           const uint64_t* __restrict__ seg_start,
                                                           uint32_t cap, BatchPlan* __restrict__ plan) {
  __shared__ unsigned long long warp_tot[8];
  const uint32_t i = blockIdx.x;
  const int d = threadIdx.x, lane = d & 31, w = d >> 5;
  if (plan[i].mode != kPlanMsd) return;
  const uint64_t at = (uint64_t)i * kRadix + d;
  const unsigned long long c = hist[at];
  unsigned long long x = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  unsigned long long base = 0;
  for (int j = 0; j < w; ++j) base += warp_tot[j];
  offs[at] = seg_start[i] + base + x - c;
  if (__syncthreads_or(c > cap) && d == 0) plan[i].mode = kPlanLsd;
}

// ================================================================= hybrid MSD + bucket sort
// After the stable MSD scatters on the top digits, every bucket is small enough
// for one CTA, which sorts it in shared memory and writes it into the final
// layout (gi_local_sort.cu).

// one digit's histogram per segment (no atomics across segments' counters)
template <class K>
__global__ void __launch_bounds__(256) k_seg_hist1(const K* __restrict__ keys,
                                                   const BatchTile* __restrict__ chunks,
                                                   uint64_t nchunks, uint32_t shift,
                                                   unsigned long long* __restrict__ hist) {
  __shared__ uint32_t sh[kRadix];
  for (uint64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const BatchTile t = chunks[c];
    sh[threadIdx.x] = 0;
    __syncthreads();
    const K* kp = keys + t.start;
    uint32_t i = threadIdx.x;
    for (; i + 3 * blockDim.x < t.count; i += 4 * blockDim.x) {  // four loads in flight
      const K a = kp[i], b = kp[i + blockDim.x], c = kp[i + 2 * blockDim.x], d = kp[i + 3 * blockDim.x];
      atomicAdd(&sh[(uint32_t)(a >> shift) & 0xFF], 1u);
      atomicAdd(&sh[(uint32_t)(b >> shift) & 0xFF], 1u);
      atomicAdd(&sh[(uint32_t)(c >> shift) & 0xFF], 1u);
      atomicAdd(&sh[(uint32_t)(d >> shift) & 0xFF], 1u);
    }
    for (; i < t.count; i += blockDim.x) atomicAdd(&sh[(uint32_t)(kp[i] >> shift) & 0xFF], 1u);
    __syncthreads();
    const uint32_t v = sh[threadIdx.x];
    if (v) atomicAdd(&hist[(uint64_t)t.seg * kRadix + threadIdx.x], (unsigned long long)v);
    __syncthreads();
  }
}

}  // namespace

size_t sort_scratch_bytes(uint64_t n, int key_bytes) {
  // status words for the most tiles any pass launches: a segmented pass over the
  // 256 buckets of one digit cuts at most one extra (partial) tile per bucket
  return header_bytes(key_bytes) +
         align256(sizeof(uint64_t) * kRadix * (tiles_for(n, key_bytes) + kRadix + 1));
}

cudaError_t sort_prepare(const void* keys, void* copy_to, uint64_t n, int key_bytes,
                         void* scratch, cudaStream_t s, uint32_t* host_trivial,
                         unsigned long long* host_win, uint32_t min_bytes) {
  ScratchView v = view(scratch, key_bytes);
  cudaError_t e = cudaMemsetAsync(scratch, 0, sort_scratch_bytes(n, key_bytes), s);
  if (e != cudaSuccess) return e;
  const int grid = grid_for(n, 256, 8);
  if (host_win) {
    // the bits in which keys differ (and the copy over the bus), then the counts
    // of the window below the highest of them; no digit counts (sort_counts
    // takes them if the LSD passes turn out to be needed)
    if (key_bytes == 4)
      k_histogram<uint32_t, false><<<grid, 256, 0, s>>>((const uint32_t*)keys, (uint32_t*)copy_to, n,
                                                        v.hist, &v.win->xor_or);
    else
      k_histogram<uint64_t, false><<<grid, 256, 0, s>>>((const uint64_t*)keys, (uint64_t*)copy_to, n,
                                                        v.hist, &v.win->xor_or);
    const void* src = copy_to ? copy_to : keys;  // the copy when the keys came over the bus
    if (key_bytes == 4)
      k_window_hist<uint32_t><<<grid, 256, 0, s>>>((const uint32_t*)src, n, v.win, min_bytes);
    else
      k_window_hist<uint64_t><<<grid, 256, 0, s>>>((const uint64_t*)src, n, v.win, min_bytes);
    k_scan_hist<<<1, 256, 0, s>>>(v.win->hist, v.win->offs, &v.win->trivial, n);
    count_launch(3);
    // [0] xor_or, [1] shift | trivial << 32, [2..257] counts
    e = cudaMemcpyAsync(host_win, v.win, 16 + sizeof(uint64_t) * kRadix, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
  }
  if (key_bytes == 4)
    k_histogram<uint32_t><<<grid, 256, 0, s>>>((const uint32_t*)keys, (uint32_t*)copy_to, n, v.hist,
                                               &v.win->xor_or);
  else
    k_histogram<uint64_t><<<grid, 256, 0, s>>>((const uint64_t*)keys, (uint64_t*)copy_to, n, v.hist,
                                               &v.win->xor_or);
  k_scan_hist<<<key_bytes, 256, 0, s>>>(v.hist, v.offs, v.trivial, n);
  count_launch(2);
  e = cudaMemcpyAsync(host_trivial, v.trivial, sizeof(uint32_t) * key_bytes, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t sort_counts(const void* keys, uint64_t n, int key_bytes, void* scratch, cudaStream_t s) {
  ScratchView v = view(scratch, key_bytes);
  const int grid = grid_for(n, 256, 8);
  cudaError_t e = cudaMemsetAsync(v.hist, 0, sizeof(uint64_t) * key_bytes * kRadix, s);
  if (e != cudaSuccess) return e;
  // (the OR lands on the window record's, which nothing reads any more)
  unsigned long long* scratch_or = &v.win->xor_or;
  if (key_bytes == 4)
    k_histogram<uint32_t><<<grid, 256, 0, s>>>((const uint32_t*)keys, nullptr, n, v.hist, scratch_or);
  else
    k_histogram<uint64_t><<<grid, 256, 0, s>>>((const uint64_t*)keys, nullptr, n, v.hist, scratch_or);
  k_scan_hist<<<key_bytes, 256, 0, s>>>(v.hist, v.offs, v.trivial, n);
  count_launch(2);
  return cudaGetLastError();
}

cudaError_t sort_window_pass(const void* src_k, const uint32_t* src_v, void* dst_k, uint32_t* dst_v,
                             uint64_t n, int key_bytes, void* scratch, uint32_t* dflags,
                             cudaStream_t s) {
  ScratchView v = view(scratch, key_bytes);
  // its own ticket counter and epoch (30): later passes never mistake its words;
  // skipped on the device when every key has the same window value
  if (key_bytes == 4)
    k_sort_pass<uint32_t><<<(unsigned)tiles_for(n, 4), kSortThreads, 0, s>>>(
        (const uint32_t*)src_k, src_v, (uint32_t*)dst_k, dst_v, n, 0u, v.win->offs, v.status,
        v.counter + key_bytes, 30u, dflags, 1u, &v.win->trivial, &v.win->shift);
  else
    k_sort_pass<uint64_t><<<(unsigned)tiles_for(n, 8), kSortThreads, 0, s>>>(
        (const uint64_t*)src_k, src_v, (uint64_t*)dst_k, dst_v, n, 0u, v.win->offs, v.status,
        v.counter + key_bytes, 30u, dflags, 1u, &v.win->trivial, &v.win->shift);
  count_launch();
  return cudaGetLastError();
}

cudaError_t sort_reset_counters(void* scratch, int key_bytes, cudaStream_t s) {
  ScratchView v = view(scratch, key_bytes);
  return cudaMemsetAsync(v.counter, 0, align256(sizeof(uint32_t) * key_bytes), s);
}

cudaError_t sort_pass(const void* src_k, const uint32_t* src_v, void* dst_k, uint32_t* dst_v,
                      uint64_t n, int key_bytes, int pass, void* scratch, uint32_t* dflags,
                      bool check_rows, cudaStream_t s) {
  ScratchView v = view(scratch, key_bytes);
  const uint64_t tiles = tiles_for(n, key_bytes);
  if (tiles == 0) return cudaSuccess;
  if (tiles > 0x7fffffffull) return cudaErrorInvalidValue;
  // every pass reuses the status array; the epoch (pass + 1) tells its words apart
  if (key_bytes == 4)
    k_sort_pass<uint32_t><<<(unsigned)tiles, kSortThreads, 0, s>>>(
        (const uint32_t*)src_k, src_v, (uint32_t*)dst_k, dst_v, n, 8u * pass,
        v.offs + pass * kRadix, v.status, v.counter + pass, (uint32_t)pass + 1, dflags,
        check_rows ? 1u : 0u, nullptr, nullptr);
  else
    k_sort_pass<uint64_t><<<(unsigned)tiles, kSortThreads, 0, s>>>(
        (const uint64_t*)src_k, src_v, (uint64_t*)dst_k, dst_v, n, 8u * pass,
        v.offs + pass * kRadix, v.status, v.counter + pass, (uint32_t)pass + 1, dflags,
        check_rows ? 1u : 0u, nullptr, nullptr);
  count_launch();
  return cudaGetLastError();
}

cudaError_t check_rowids(const uint32_t* rows, uint64_t n, uint32_t* dflags, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_check_rows<<<grid_for(n, 256, 8), 256, 0, s>>>(rows, n, dflags);
  count_launch();
  return cudaGetLastError();
}

template <class K>
static void launch_gather(const void* sk, const uint32_t* sv, void* dk, uint32_t* dv,
                          const Geom& g, uint32_t key_off, uint32_t* dflags, cudaStream_t s) {
  const int grid = grid_for(g.n, 256, 16);
  const K* a = (const K*)sk;
  K* b = (K*)dk;
  switch (g.k) {
    case 2: k_layout_gather<K, 2><<<grid, 256, 0, s>>>(a, sv, b, dv, g, key_off, dflags); break;
    case 3: k_layout_gather<K, 3><<<grid, 256, 0, s>>>(a, sv, b, dv, g, key_off, dflags); break;
    case 4: k_layout_gather<K, 4><<<grid, 256, 0, s>>>(a, sv, b, dv, g, key_off, dflags); break;
    case 5: k_layout_gather<K, 5><<<grid, 256, 0, s>>>(a, sv, b, dv, g, key_off, dflags); break;
    case 8: k_layout_gather<K, 8><<<grid, 256, 0, s>>>(a, sv, b, dv, g, key_off, dflags); break;
    case 9: k_layout_gather<K, 9><<<grid, 256, 0, s>>>(a, sv, b, dv, g, key_off, dflags); break;
    case 16: k_layout_gather<K, 16><<<grid, 256, 0, s>>>(a, sv, b, dv, g, key_off, dflags); break;
    case 17: k_layout_gather<K, 17><<<grid, 256, 0, s>>>(a, sv, b, dv, g, key_off, dflags); break;
    case 32: k_layout_gather<K, 32><<<grid, 256, 0, s>>>(a, sv, b, dv, g, key_off, dflags); break;
    case 33: k_layout_gather<K, 33><<<grid, 256, 0, s>>>(a, sv, b, dv, g, key_off, dflags); break;
    default: k_layout_gather<K, 0><<<grid, 256, 0, s>>>(a, sv, b, dv, g, key_off, dflags); break;
  }
  count_launch();
}

cudaError_t layout_gather(const void* sk, const uint32_t* sv, void* dk, uint32_t* dv,
                          const Geom& g, int key_bytes, uint32_t key_off, uint32_t* dflags,
                          cudaStream_t s) {
  if (g.n == 0) return cudaSuccess;
  if (key_bytes == 4)
    launch_gather<uint32_t>(sk, sv, dk, dv, g, key_off, dflags, s);
  else
    launch_gather<uint64_t>(sk, sv, dk, dv, g, key_off, dflags, s);
  return cudaGetLastError();
}

cudaError_t check_sorted_dups(const void* sk, uint64_t n, int key_bytes, uint32_t* dflags,
                              cudaStream_t s) {
  if (n < 2) return cudaSuccess;
  const int grid = grid_for(n, 256, 8);
  if (key_bytes == 4)
    k_sorted_dups<uint32_t><<<grid, 256, 0, s>>>((const uint32_t*)sk, n, dflags);
  else
    k_sorted_dups<uint64_t><<<grid, 256, 0, s>>>((const uint64_t*)sk, n, dflags);
  count_launch();
  return cudaGetLastError();
}


// ---------------------------------------------------------------- batched form, host side
uint32_t batch_sort_tile(int key_bytes) {
  return kSortThreads * (key_bytes == 4 ? SortTile<uint32_t>::kItems : SortTile<uint64_t>::kItems);
}

size_t batch_sort_scratch_bytes(uint64_t ntiles, uint32_t nseg, int key_bytes) {
  const int passes = key_bytes;
  return 2 * align256(sizeof(uint64_t) * (uint64_t)nseg * passes * kRadix) +
         align256(sizeof(uint32_t) * passes) +
         align256(sizeof(uint64_t) * kRadix * (ntiles + 1));
}

size_t batch_hybrid_bytes(uint32_t nseg, uint64_t ntiles) {
  return align256(sizeof(BatchPlan) * nseg) + align256(sizeof(SlotMap) * nseg) +
         2 * align256(sizeof(uint64_t) * (uint64_t)nseg * kRadix) + 256 +
         3 * align256(sizeof(uint32_t) * (nseg + 1)) + 2 * align256(sizeof(uint32_t) * (ntiles + 1)) +
         align256(sizeof(uint32_t) * 3 * (uint64_t)nseg * (kRadix + 1)) + 256 +
         align256(sizeof(uint64_t) * nseg);
}

cudaError_t batch_sort(const void* keys, const uint32_t* vals, void* tmp_k[2], uint32_t* tmp_v[2],
                       uint64_t n, int key_bytes, const uint64_t* seg_start, uint32_t nseg,
                       const BatchTile* tiles, uint64_t ntiles, const BatchTile* chunks,
                       uint64_t nchunks, void* scratch, uint32_t* dflags, cudaStream_t s,
                       int* result_buf, const BatchHybrid* hy) {
  const int passes = key_bytes;
  char* p = (char*)scratch;
  unsigned long long* hist = (unsigned long long*)p;
  p += align256(sizeof(uint64_t) * (uint64_t)nseg * passes * kRadix);
  unsigned long long* offs = (unsigned long long*)p;
  p += align256(sizeof(uint64_t) * (uint64_t)nseg * passes * kRadix);
  uint32_t* counter = (uint32_t*)p;
  p += align256(sizeof(uint32_t) * passes);
  uint64_t* status = (uint64_t*)p;
  cudaError_t e = cudaMemsetAsync(scratch, 0, batch_sort_scratch_bytes(ntiles, nseg, key_bytes), s);
  if (e != cudaSuccess) return e;
  if (n == 0 || ntiles == 0) {
    *result_buf = -1;
    return cudaSuccess;
  }
  const int hgrid = (int)std::min<uint64_t>(nchunks, (uint64_t)sm_count() * 8);
  // persistent radix grids: the 5 CTAs per SM the pass fits
  const unsigned pgrid = (unsigned)std::min<uint64_t>(ntiles, (uint64_t)sm_count() * 5);
  const BatchPlan* plan = nullptr;
  if (!hy) {  // the plain segmented LSD sort: digit histograms of every index
    if (key_bytes == 4)
      k_batch_histogram<uint32_t><<<hgrid, 256, 0, s>>>((const uint32_t*)keys, vals, chunks, nchunks, hist, dflags, nullptr);
    else
      k_batch_histogram<uint64_t><<<hgrid, 256, 0, s>>>((const uint64_t*)keys, vals, chunks, nchunks, hist, dflags, nullptr);
    k_batch_scan_hist<<<nseg, 256, 0, s>>>(hist, offs, seg_start, passes);
    count_launch(2);
  } else {
    // per-index plans from the bits in which each index's keys differ, the MSD
    // window counts, then the digit histograms of the indexes that fall back to the
    // LSD passes only; then the MSD scatter into tmp[1] and the bucket sort, which
    // writes the layouts of those indexes.  The rowIDs are checked by the kernels
    // that read the input: the MSD pass, the bucket sort of whole indexes, the
    // first LSD pass.
    plan = hy->plan;
    const uint32_t cap = local_sort_capacity();
    e = cudaMemsetAsync(hy->hist_w, 0, sizeof(uint64_t) * (uint64_t)nseg * kRadix, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(hy->counter, 0, sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(hy->bucket_count, 0, 3 * sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(hy->xor_or, 0, sizeof(uint64_t) * nseg, s);
    if (e != cudaSuccess) return e;
    if (key_bytes == 4)
      k_batch_xor<uint32_t><<<hgrid, 256, 0, s>>>((const uint32_t*)keys, chunks, nchunks, seg_start, hy->xor_or);
    else
      k_batch_xor<uint64_t><<<hgrid, 256, 0, s>>>((const uint64_t*)keys, chunks, nchunks, seg_start, hy->xor_or);
    k_batch_plan<<<(nseg + 255) / 256, 256, 0, s>>>(hy->xor_or, seg_start, nseg, key_bytes, hy->k, hy->kidx, cap,
                                                   hy->plan, hy->slot_maps);
    if (key_bytes == 4)
      k_batch_window_hist<uint32_t><<<hgrid, 256, 0, s>>>((const uint32_t*)keys, chunks, nchunks, hy->plan, hy->hist_w);
    else
      k_batch_window_hist<uint64_t><<<hgrid, 256, 0, s>>>((const uint64_t*)keys, chunks, nchunks, hy->plan, hy->hist_w);
    k_batch_window_scan<<<nseg, 256, 0, s>>>(hy->hist_w, hy->offs_w, seg_start, cap, hy->plan);
    if (key_bytes == 4)
      k_batch_histogram<uint32_t><<<hgrid, 256, 0, s>>>((const uint32_t*)keys, vals, chunks, nchunks, hist, dflags, hy->plan);
    else
      k_batch_histogram<uint64_t><<<hgrid, 256, 0, s>>>((const uint64_t*)keys, vals, chunks, nchunks, hist, dflags, hy->plan);
    k_batch_scan_hist<<<nseg, 256, 0, s>>>(hist, offs, seg_start, passes);
    count_launch(6);
    k_batch_mode_prefix<<<1, 1024, 0, s>>>(hy->plan, hy->tile0, nseg, hy->prefix_msd, hy->prefix_lsd);
    k_batch_mode_lists<<<nseg, 256, 0, s>>>(hy->plan, hy->tile0, hy->prefix_msd, hy->prefix_lsd,
                                            hy->list_msd, hy->list_lsd);
    count_launch(2);
    // persistent grid over the tiles of the kPlanMsd indexes only; the status
    // array is shared with the LSD passes: a distinct epoch (9)
    const TileMap msd_map{hy->list_msd, hy->prefix_msd + nseg};
    if (key_bytes == 4)
      k_batch_sort_pass<uint32_t><<<pgrid, kSortThreads, 0, s>>>(
          (const uint32_t*)keys, vals, (uint32_t*)tmp_k[1], tmp_v[1], n, 0u, tiles, hy->offs_w, 0,
          1, status, hy->counter, 9u, dflags, hy->plan, kPlanMsd, 1u, msd_map, 1u);
    else
      k_batch_sort_pass<uint64_t><<<pgrid, kSortThreads, 0, s>>>(
          (const uint64_t*)keys, vals, (uint64_t*)tmp_k[1], tmp_v[1], n, 0u, tiles, hy->offs_w, 0,
          1, status, hy->counter, 9u, dflags, hy->plan, kPlanMsd, 1u, msd_map, 1u);
    count_launch();
    e = batch_local_sort(keys, vals, tmp_k[1], tmp_v[1], seg_start, nseg, key_bytes, *hy, dflags, s);
    if (e != cudaSuccess) return e;
  }
  // every pass runs (no host round trip to skip trivial digits, so the whole
  // build can be captured in a graph); with a plan, only for kPlanLsd indexes,
  // on a persistent grid over their tiles (usually none)
  const TileMap lsd_map = hy ? TileMap{hy->list_lsd, hy->prefix_lsd + nseg} : TileMap{};
  const unsigned grid = hy ? pgrid : (unsigned)ntiles;
  const void* ck = keys;
  const uint32_t* cv = vals;
  int cur = -1;
  for (int ps = 0; ps < passes; ++ps) {
    const int dst = cur == 0 ? 1 : 0;
    if (key_bytes == 4)
      k_batch_sort_pass<uint32_t><<<grid, kSortThreads, 0, s>>>(
          (const uint32_t*)ck, cv, (uint32_t*)tmp_k[dst], tmp_v[dst], n, 8u * ps, tiles, offs, ps,
          passes, status, counter + ps, (uint32_t)ps + 1, dflags, plan, kPlanLsd, 0u, lsd_map,
          (hy && ps == 0) ? 1u : 0u);
    else
      k_batch_sort_pass<uint64_t><<<grid, kSortThreads, 0, s>>>(
          (const uint64_t*)ck, cv, (uint64_t*)tmp_k[dst], tmp_v[dst], n, 8u * ps, tiles, offs, ps,
          passes, status, counter + ps, (uint32_t)ps + 1, dflags, plan, kPlanLsd, 0u, lsd_map,
          (hy && ps == 0) ? 1u : 0u);
    count_launch();
    ck = tmp_k[dst];
    cv = tmp_v[dst];
    cur = dst;
  }
  *result_buf = cur;
  return cudaGetLastError();
}

template <class K>
static void launch_batch_gather(const void* sk, const uint32_t* sv, void* ok, uint32_t* ov,
                                const BatchTile* tiles, uint64_t ntiles, const uint64_t* seg_start,
                                const uint64_t* seg_base, uint32_t k, uint32_t* dflags,
                                cudaStream_t s, const BatchPlan* plan, TileMap map,
                                const uint32_t* kidx) {
  const int grid = (int)std::min<uint64_t>(ntiles, (uint64_t)sm_count() * 16);
  const K* a = (const K*)sk;
  K* b = (K*)ok;
#define GI_BG(KF) k_batch_gather<K, KF><<<grid, 256, 0, s>>>(a, sv, b, ov, tiles, ntiles, seg_start, seg_base, k, dflags, plan, map, kidx)
  switch (k) {
    case kBatchMixed: GI_BG(-1); break;  // each index's own fan-out
    case 0: GI_BG(1); break;  // sorted order: rank == slot
    case 2: GI_BG(2); break;
    case 3: GI_BG(3); break;
    case 5: GI_BG(5); break;
    case 9: GI_BG(9); break;
    case 17: GI_BG(17); break;
    default: GI_BG(0); break;
  }
#undef GI_BG
  count_launch();
}

cudaError_t batch_gather(const void* sk, const uint32_t* sv, void* ok, uint32_t* ov,
                         const BatchTile* tiles, uint64_t ntiles, const uint64_t* seg_start,
                         const uint64_t* seg_base, uint32_t k, int key_bytes, uint32_t* dflags,
                         cudaStream_t s, const BatchHybrid* hy, uint32_t nseg) {
  if (ntiles == 0) return cudaSuccess;
  const BatchPlan* plan = hy ? hy->plan : nullptr;
  const TileMap map = hy ? TileMap{hy->list_lsd, hy->prefix_lsd + nseg} : TileMap{};
  const uint32_t* kidx = hy ? hy->kidx : nullptr;
  if (k == kBatchMixed && !kidx) return cudaErrorInvalidValue;
  if (key_bytes == 4)
    launch_batch_gather<uint32_t>(sk, sv, ok, ov, tiles, ntiles, seg_start, seg_base, k, dflags, s, plan, map, kidx);
  else
    launch_batch_gather<uint64_t>(sk, sv, ok, ov, tiles, ntiles, seg_start, seg_base, k, dflags, s, plan, map, kidx);
  return cudaGetLastError();
}


// ---------------------------------------------------------------- hybrid sort, host side
// The level-2 buckets of the hybrid sort grouped by size class, on the device:
// bin i (one per level-1 bucket and second-window value) with hist[i] pairs
// starting at offs[i] joins the list of its class (lists + class * nbins, order
// within a list arbitrary); counts[class] ends as each list's length, and
// counts[kLocalClasses] as the number of buckets too large for any class.
__global__ void __launch_bounds__(256) k_bucket_classes(const unsigned long long* __restrict__ hist,
                                                        const unsigned long long* __restrict__ offs,
                                                        uint32_t nbins, BatchTile* __restrict__ lists,
                                                        uint32_t* __restrict__ counts) {
  __shared__ uint32_t s_cnt[kLocalClasses + 1], s_base[kLocalClasses + 1];
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (threadIdx.x <= kLocalClasses) s_cnt[threadIdx.x] = 0;
  __syncthreads();
  const uint64_t c = i < nbins ? hist[i] : 0ull;
  const int cls = c ? local_sort_class(c) : -1;
  uint32_t pos = 0;
  if (cls >= 0) pos = atomicAdd(&s_cnt[cls], 1u);
  __syncthreads();
  if (threadIdx.x <= kLocalClasses && s_cnt[threadIdx.x])
    s_base[threadIdx.x] = atomicAdd(&counts[threadIdx.x], s_cnt[threadIdx.x]);
  __syncthreads();
  if (cls >= 0 && cls < kLocalClasses)
    lists[(uint64_t)cls * nbins + s_base[cls] + pos] = BatchTile{offs[i], 0u, (uint32_t)c, 0u, 0u};
}

cudaError_t hybrid_sort(const void* src_k, const uint32_t* src_v, void* bk[2], uint32_t* bv[2],
                        int first_dst, uint64_t n, int key_bytes, uint32_t nontrivial,
                        const unsigned long long* host_win, void* scratch, const Geom& g,
                        bool sorted_layout, uint32_t key_off, bool force, bool pass1_done,
                        unsigned long long* host_h2, uint32_t* dflags, cudaStream_t s,
                        int* result, bool* used, int* verify_src) {
  *used = false;
  *verify_src = -1;
  *result = pass1_done ? first_dst : -1;
  const int nd = __builtin_popcount(nontrivial);  // bytes in which two keys differ
  // The bucket sort's slot map is 32-bit: larger indexes take the LSD sort.
  if (nd < 2 || n >= (1ull << 32) || !host_win) return cudaSuccess;
  // Measured crossovers (GB300): hybrid_min_pairs / hybrid_min_digits.
  if (!force && (nd < (int)hybrid_min_digits(key_bytes) || n < hybrid_min_pairs(key_bytes)))
    return cudaSuccess;
  if (host_win[1] >> 32) return cudaSuccess;  // one window value only (the pass was skipped)
  const uint64_t cap = local_sort_capacity();
  // MSD windows: the 8 bits just below the highest bit in which two keys differ
  // (s1), then the next 8 (s2), so that no scatter spends a bit every key shares
  const uint32_t s1 = (uint32_t)(host_win[1] & 0xFFFFFFFFu);
  const unsigned long long* hw = host_win + 2;
  // level-1 buckets straight from the window's counts
  std::vector<uint64_t> start1(kRadix + 1, 0);
  uint64_t mx1 = 0;
  for (int d = 0; d < kRadix; ++d) {
    start1[d + 1] = start1[d] + hw[d];
    mx1 = std::max<uint64_t>(mx1, hw[d]);
  }
  // A second window of w2 <= 8 bits just below the first, as wide as it takes to
  // split the largest level-1 bucket into pieces of about 2048 pairs (narrower
  // means fewer, fuller buckets: 2^24..2^27 uniform keys give ~2048-pair buckets,
  // 2^28 ~4096); none if that bucket fits a CTA as it is.
  uint32_t w2 = 0;
  while (w2 < 8 && w2 < s1 && (mx1 >> w2) > 2048) ++w2;
  if ((mx1 >> w2) > cap) return cudaSuccess;  // its level-2 buckets (on average) cannot fit
  const bool two = w2 > 0;
  const uint32_t s2 = s1 - w2;  // the digit at s2 takes the w2 new bits (those above are fixed)
  // keys of one bucket agree on the bits at and above bshift; the bucket sort
  // splits on the 8 bits below, then ranks, or sorts the lower bytes one by one
  const uint32_t bshift = two ? s2 : s1;
  const uint32_t top_shift = bshift >= 8 ? bshift - 8 : 0;
  uint32_t lsd_mask = 0;
  for (int p = 0; p < key_bytes; ++p)
    if ((nontrivial >> p & 1u) && 8u * (uint32_t)p < bshift) lsd_mask |= 1u << p;
  const bool single = bshift <= 8;

  ScratchView v = view(scratch, key_bytes);
  cudaError_t e;
  // pass 1: the window scatter, unless the caller ran it already while the
  // histograms came back
  const int dst1 = first_dst;
  if (!pass1_done) {
    e = sort_window_pass(src_k, src_v, bk[dst1], bv[dst1], n, key_bytes, scratch, dflags, s);
    if (e != cudaSuccess) return e;
  }
  int cur = dst1;
  // the buckets the shared-memory sort takes, by size class (the last: too large)
  std::vector<BatchTile> segs[kLocalClasses + 1];
  if (two) {
    // tables of the level-1 buckets for the segmented pass on s2 (host-built
    // from the window counts while pass 1 runs)
    std::vector<BatchTile> tiles, chunks;
    std::vector<uint64_t> seg_start;
    const uint32_t tile = batch_sort_tile(key_bytes);
    uint32_t nseg1 = 0;
    for (int d = 0; d < kRadix; ++d) {
      const uint64_t a = start1[d], c = start1[d + 1] - a;
      if (!c) continue;
      seg_start.push_back(a);
      for (uint64_t t = 0, l = 0; t < c; t += tile, ++l)
        tiles.push_back(BatchTile{a + t, nseg1, (uint32_t)std::min<uint64_t>(tile, c - t), (uint32_t)l, 0});
      for (uint64_t t = 0; t < c; t += kBatchChunk)
        chunks.push_back(BatchTile{a + t, nseg1, (uint32_t)std::min<uint64_t>(kBatchChunk, c - t), 0, 0});
      ++nseg1;
    }
    seg_start.push_back(n);
    const size_t tbytes = tiles.size() * sizeof(BatchTile), cbytes = chunks.size() * sizeof(BatchTile);
    const size_t hbytes = (size_t)nseg1 * kRadix * 8;
    const uint32_t nbins = nseg1 * kRadix;
    const size_t lbytes = (size_t)kLocalClasses * nbins * sizeof(BatchTile);
    char* blob = nullptr;
    const size_t blob_bytes = 9 * 256 + tbytes + cbytes + 2 * hbytes + (nseg1 + 1) * 8 + 64 + lbytes + 64;
    e = cudaMallocAsync((void**)&blob, blob_bytes, s);
    if (e != cudaSuccess) return e;
    char* q = blob;
    auto take = [&](size_t b) { char* r = q; q += (b + 255) & ~size_t(255); return r; };
    BatchTile* d_tiles = (BatchTile*)take(tbytes);
    BatchTile* d_chunks = (BatchTile*)take(cbytes);
    unsigned long long* d_hist = (unsigned long long*)take(hbytes);
    unsigned long long* d_offs = (unsigned long long*)take(hbytes);
    uint64_t* d_seg_start = (uint64_t*)take((nseg1 + 1) * 8);
    uint32_t* d_counter = (uint32_t*)take(64);
    BatchTile* d_lists = (BatchTile*)take(lbytes);
    uint32_t* d_cls = (uint32_t*)take(64);  // [kLocalClasses + 1] list lengths
    e = cudaMemcpyAsync(d_tiles, tiles.data(), tbytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_chunks, chunks.data(), cbytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_seg_start, seg_start.data(), (nseg1 + 1) * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_hist, 0, hbytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_counter, 0, 64, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_cls, 0, 64, s);
    if (e != cudaSuccess) {
      cudaFreeAsync(blob, s);
      return e;
    }
    // per-bucket counts of the second window and their scan into absolute offsets
    const int hgrid = (int)std::min<uint64_t>(chunks.size(), (uint64_t)sm_count() * 8);
    if (key_bytes == 4)
      k_seg_hist1<uint32_t><<<hgrid, 256, 0, s>>>((const uint32_t*)bk[cur], d_chunks, chunks.size(), s2, d_hist);
    else
      k_seg_hist1<uint64_t><<<hgrid, 256, 0, s>>>((const uint64_t*)bk[cur], d_chunks, chunks.size(), s2, d_hist);
    k_batch_scan_hist<<<nseg1, 256, 0, s>>>(d_hist, d_offs, d_seg_start, 1);
    // the level-2 buckets grouped by size class on the device: no host round trip
    k_bucket_classes<<<(nbins + 255) / 256, 256, 0, s>>>(d_hist, d_offs, nbins, d_lists, d_cls);
    count_launch(3);
    // pass 2: segmented on s2; tiles.size() <= tiles_for(n) + 256, which the
    // status array is sized for
    const int dst2 = 1 - cur;
    if (key_bytes == 4)
      k_batch_sort_pass<uint32_t><<<(unsigned)tiles.size(), kSortThreads, 0, s>>>(
          (const uint32_t*)bk[cur], bv[cur], (uint32_t*)bk[dst2], bv[dst2], n, s2, d_tiles,
          d_offs, 0, 1, v.status, d_counter, 40u, dflags, nullptr, 0u, 0u, TileMap{}, 0u);
    else
      k_batch_sort_pass<uint64_t><<<(unsigned)tiles.size(), kSortThreads, 0, s>>>(
          (const uint64_t*)bk[cur], bv[cur], (uint64_t*)bk[dst2], bv[dst2], n, s2, d_tiles,
          d_offs, 0, 1, v.status, d_counter, 40u, dflags, nullptr, 0u, 0u, TileMap{}, 0u);
    count_launch();
    cur = dst2;
    // every level-2 bucket sorted in shared memory and written into the final
    // layout, one launch per size class (the list lengths read on the device; a
    // launch whose list is empty returns at once).  A bucket too large for any
    // class is left out and counted: the caller reads that count (copied to
    // host_h2) once the stream is done and then falls back to the LSD sort from
    // bk[*verify_src], the data after both scatters, which the bucket sort only read.
    const int dst3 = 1 - cur;
    for (int c = 0; c < kLocalClasses && e == cudaSuccess; ++c)
      e = local_sort(bk[cur], bv[cur], bk[dst3], bv[dst3], d_lists + (size_t)c * nbins, nbins, d_cls + c,
                     local_class_max(c), c, top_shift, lsd_mask, single, key_bytes, g, sorted_layout,
                     key_off, dflags, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(host_h2, d_cls + kLocalClasses, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(blob, s);
    if (e != cudaSuccess) return e;
    *result = dst3;
    *used = true;
    *verify_src = cur;
    return cudaGetLastError();
  } else {
    for (int d = 0; d < kRadix; ++d) {
      const uint64_t c = start1[d + 1] - start1[d];
      if (c) segs[local_sort_class(c)].push_back(BatchTile{start1[d], 0, (uint32_t)c, 0, 0});
    }
  }
  // one level: every bucket sorted in shared memory and written into the final
  // layout, one launch per size class, so that a few large buckets do not put
  // every bucket in the widest class (fewer CTAs per SM)
  if (!segs[kLocalClasses].empty()) return cudaErrorInvalidValue;  // no class fits
  size_t total = 0;
  for (int c = 0; c < kLocalClasses; ++c) total += segs[c].size();
  BatchTile* d_segs = nullptr;
  e = cudaMallocAsync((void**)&d_segs, std::max<size_t>(1, total) * sizeof(BatchTile), s);
  if (e != cudaSuccess) return e;
  const int dst3 = 1 - cur;
  size_t at = 0;
  for (int c = 0; c < kLocalClasses && e == cudaSuccess; ++c) {
    const std::vector<BatchTile>& v = segs[c];
    if (v.empty()) continue;
    uint64_t max_count = 1;
    for (const BatchTile& t : v) max_count = std::max<uint64_t>(max_count, t.count);
    e = cudaMemcpyAsync(d_segs + at, v.data(), v.size() * sizeof(BatchTile), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = local_sort(bk[cur], bv[cur], bk[dst3], bv[dst3], d_segs + at, v.size(), nullptr, max_count, -1,
                     top_shift, lsd_mask, single, key_bytes, g, sorted_layout, key_off, dflags, s);
    at += v.size();
  }
  cudaFreeAsync(d_segs, s);
  if (e != cudaSuccess) return e;
  *result = dst3;
  *used = true;
  return cudaGetLastError();
}

}  // namespace gi
