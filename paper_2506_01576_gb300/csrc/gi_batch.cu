// Batched form: thousands of independent indexes of uneven size, built and
// probed together.
//
// gi_batch_create sizes and allocates everything once from the host-side key
// offsets (tile tables, sort buffers, the padded index arrays, per-index
// descriptors), so gi_batch_build and gi_batch_point_lookup launch kernels only:
// no allocation, no host synchronisation.  The sequence can be captured in a
// CUDA graph and replayed.
//
//   build : every index is sorted by a plan a kernel writes on the device from
//           the bits in which its keys differ (gi_sort.cu): a whole index of at
//           most 5120 pairs by one CTA in shared memory; a larger one by a stable
//           MSD scatter on a window of its highest varying bits, then the same
//           bucket sort on every window bucket; the LSD passes (segmented: each
//           tile stays inside its index, look-back stops at the index's first
//           tile) only when a window bucket is too large.  The bucket sort writes
//           each pair straight into its index's layout -- the index's own fan-out
//           (gi_batch_set_fanouts), sorted or k-ary -- in a padded per-index
//           region (max-key padding after every index, 256-byte aligned starts);
//           after the LSD passes the closed-form permutation does.
//   lookup: one persistent launch over (index, chunk of probes) work items.  A
//           CTA takes a work item, copies the top levels of that index that fit
//           in its shared-memory budget with one bulk asynchronous copy
//           (mbarrier, bounded wait), then every thread runs the descent of the
//           index's layout (binary search, or k-ary with its fan-out) for its
//           probes, reading pinned levels from shared memory and the rest from
//           global memory.  The pinned depth is chosen per index by its size
//           (small indexes are pinned whole).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include "gi_internal.cuh"
#include "gi_point_impl.cuh"
#include "gi_ptr.h"

namespace gi {

struct BatchDesc {
  uint64_t base;         // slot 0 of the index in the padded arrays
  uint64_t n;            // keys
  uint32_t levels;       // tree levels (k-ary) / 0 for sorted
  uint32_t smem_levels;  // top levels pinned in shared memory for this index
  uint32_t smem_slots;   // slots copied to shared memory (0: none)
  uint32_t k;            // fan-out of this index (0: sorted)
};

namespace bt {

// Work item w -> index b: the last b with chunk_start[b] <= w.
__device__ __forceinline__ uint32_t find_index(const uint64_t* cs, uint32_t B, uint64_t w) {
  uint32_t lo = 0, hi = B;  // cs[lo] <= w < cs[hi]
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (cs[mid] <= w) lo = mid; else hi = mid;
  }
  return lo;
}

// chunk_start[b] = sum over c < b of ceil(probes of c / CH); one CTA, any B
__global__ void __launch_bounds__(1024) k_chunk_starts(const uint64_t* __restrict__ qoff, uint32_t B,
                                                       uint32_t CH, uint64_t* __restrict__ cs) {
  __shared__ uint64_t s_warp[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint64_t carry = 0;
  for (uint64_t base = 0; base < B; base += blockDim.x) {
    const uint64_t b = base + threadIdx.x;
    const uint64_t v = b < B ? (qoff[b + 1] - qoff[b] + CH - 1) / CH : 0;
    uint64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    uint64_t pre = 0, tot = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      if (i < w) pre += s_warp[i];
      tot += s_warp[i];
    }
    if (b < B) cs[b] = carry + pre + x - v;
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) cs[B] = carry;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  uint32_t done = 0;
  for (uint32_t spin = 0; spin < kSpinLimit && !done; ++spin) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
  }
  return done != 0;
}

template <class K, int KF>
__device__ __forceinline__ uint32_t eks_one(const K* __restrict__ keys, const uint32_t* __restrict__ rows,
                                            const BatchDesc& d, const K* sm, K x) {
  constexpr int N = KF - 1;
  uint64_t s = 0, cand = ~0ull;
  const K* base = keys + d.base;
  for (uint32_t lv = 0; lv < d.levels; ++lv) {
    if (s >= d.n) break;
    K piv[N];
    if (lv < d.smem_levels) {
#pragma unroll
      for (int p = 0; p < N; ++p) piv[p] = sm[s + p];
    } else if constexpr (pt::EksShape<K, KF, 1>::VEC) {
      pt::vec_load<K, N>(base + s, piv);
    } else {
#pragma unroll
      for (int p = 0; p < N; ++p) piv[p] = __ldg(base + s + p);
    }
    uint32_t c = 0;
#pragma unroll
    for (int p = 0; p < N; ++p) c += piv[p] < x ? 1u : 0u;
    if (c < (uint32_t)N && s + c < d.n) cand = s + c;
    s = s * KF + (uint64_t)(c + 1) * N;
  }
  if (cand != ~0ull && __ldg(base + cand) == x) return __ldg(rows + d.base + cand);
  return GI_MISS;
}

template <class K>
__device__ __forceinline__ uint32_t bs_one(const K* __restrict__ keys, const uint32_t* __restrict__ rows,
                                           const BatchDesc& d, K x) {
  const K* base = keys + d.base;
  uint64_t lo = 0, len = d.n;
  while (len > 0) {
    const uint64_t half = len >> 1;
    if (base[lo + half] < x) {
      lo += half + 1;
      len -= half + 1;
    } else {
      len = half;
    }
  }
  return (lo < d.n && base[lo] == x) ? rows[d.base + lo] : GI_MISS;
}

// One lookup in an index of a batch whose indexes each have their own fan-out
// (d.k; 0 = sorted).  The work item, and so d.k, is the same for the whole CTA.
// WIDE = false: fan-outs up to 5 only (their pivots fit the registers of 8 CTAs
// per SM; the host takes the wide form when an index has k = 9 or 17).
template <class K, bool WIDE>
__device__ __forceinline__ uint32_t any_one(const K* __restrict__ keys, const uint32_t* __restrict__ rows,
                                            const BatchDesc& d, const K* sm, K x) {
  switch (d.k) {
    case 2: return eks_one<K, 2>(keys, rows, d, sm, x);
    case 3: return eks_one<K, 3>(keys, rows, d, sm, x);
    case 5: return eks_one<K, 5>(keys, rows, d, sm, x);
    case 9: if constexpr (WIDE) return eks_one<K, 9>(keys, rows, d, sm, x); else return GI_MISS;
    case 17: if constexpr (WIDE) return eks_one<K, 17>(keys, rows, d, sm, x); else return GI_MISS;
    default: return bs_one<K>(keys, rows, d, x);
  }
}

// CTAs per SM the registers of a lookup variant allow: 8 (the default grid) for
// node widths up to 4 keys, 5 for wider nodes.
template <int KF>
constexpr int batch_point_min_blocks() {
  return (KF == -2 || KF >= 9) ? 5 : 8;
}

// KF == 0: sorted layout (binary search per index, no pinning); KF == -1 / -2:
// each index's own fan-out (-1: up to 5; -2: any)
template <class K, int KF>
__global__ void __launch_bounds__(256, batch_point_min_blocks<KF>()) k_batch_point(const K* __restrict__ keys,
                                                     const uint32_t* __restrict__ rows,
                                                     const BatchDesc* __restrict__ desc,
                                                     const uint64_t* __restrict__ qoff,
                                                     const uint64_t* __restrict__ cs, uint32_t B,
                                                     const K* __restrict__ q,
                                                     uint32_t* __restrict__ out, uint32_t CH,
                                                     uint32_t* __restrict__ flags) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t s_b;
  const K* sm = (const K*)smem_raw;
  const uint32_t bar = pt::smem_u32(&mbar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  uint32_t phase = 0;
  bool in_flight = false, ok = true;
  const uint64_t total = cs[B];
  for (uint64_t w = blockIdx.x; w < total; w += gridDim.x) {
    if (threadIdx.x == 0) s_b = find_index(cs, B, w);
    __syncthreads();
    const uint32_t b = s_b;
    const BatchDesc d = desc[b];
    const uint64_t q0 = qoff[b] + (w - cs[b]) * CH;
    const uint64_t q1 = min(q0 + CH, qoff[b + 1]);
    bool staged = true;
    if (KF != 0 && d.smem_slots) {
      const uint32_t bytes = (uint32_t)(((uint64_t)d.smem_slots * sizeof(K) + 15) & ~15ull);
      if (threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
                "r"(pt::smem_u32(smem_raw)),
            "l"(keys + d.base), "r"(bytes), "r"(bar)
            : "memory");
      }
      const bool landed = mbar_wait(bar, phase & 1);
      phase ^= 1;
      // every thread takes the same decision (a partial timeout must not split the CTA)
      staged = !__syncthreads_or(!landed);
      if (!staged) {
        in_flight = !landed;
        ok = false;
        if (threadIdx.x == 0) atomicOr(flags, kFlagTimeout);
      }
    }
    if (staged) {
      for (uint64_t i = q0 + threadIdx.x; i < q1; i += blockDim.x) {
        const K x = q[i];
        if constexpr (KF < 0)
          out[i] = any_one<K, KF == -2>(keys, rows, d, sm, x);
        else if constexpr (KF > 0)
          out[i] = eks_one<K, KF>(keys, rows, d, sm, x);
        else
          out[i] = bs_one<K>(keys, rows, d, x);
      }
    }
    __syncthreads();  // the staging buffer is reused by the next work item
    if (!ok) break;
  }
  if (in_flight) mbar_wait(bar, phase & 1);  // a copy still in flight: let it land (bounded)
}

}  // namespace bt
}  // namespace gi

// ---------------------------------------------------------------- host side
struct gi_batch {
  int device = 0;
  cudaStream_t stream = nullptr;
  uint32_t B = 0;
  int layout = GI_EYTZINGER_KARY;
  uint32_t k = 0;
  int key_bytes = 8;
  uint64_t n = 0;
  std::vector<uint64_t> key_off;  // host copy, B+1
  std::vector<gi::BatchDesc> desc_host;
  uint64_t* d_seg_start = nullptr;
  uint64_t* d_seg_base = nullptr;
  gi::BatchDesc* d_desc = nullptr;
  gi::BatchTile* d_tiles = nullptr;
  uint64_t ntiles = 0;
  gi::BatchTile* d_chunks = nullptr;
  uint64_t nchunks = 0;
  void* keys = nullptr;
  uint32_t* rows = nullptr;
  size_t keys_bytes = 0;
  void* tmp_k[2] = {nullptr, nullptr};
  uint32_t* tmp_v[2] = {nullptr, nullptr};
  void* scratch = nullptr;
  uint32_t* dflags = nullptr;
  uint64_t* d_cs = nullptr;  // B+1 chunk starts of the last lookup
  void* hy_mem = nullptr;    // tables of the hybrid build
  gi::BatchHybrid hy{};
  std::vector<uint32_t> kidx_host;  // fan-out of every index (0: sorted)
  uint32_t* d_kidx = nullptr;
  int result = -1;
  // defaults: gi_batch_tune's choice on 4096 indexes of 2^8..2^20 u64 keys with
  // 2^10..2^18 probes each (1.41x over 1024 / 4 / 16384)
  uint32_t chunk = 2048;       // probes per work item
  uint32_t smem_budget = 0;    // bytes of pinned levels per CTA
  int blocks_per_sm = 8;
};

namespace {
int bfail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  gi::set_last_error(buf);
  return code;
}

int bcuda(cudaError_t e, const char* what) {
  cudaGetLastError();
  return bfail(e == cudaErrorMemoryAllocation ? GI_ERR_NOMEM : GI_ERR_CUDA, "%s: %s", what,
               cudaGetErrorString(e));
}

// device (or managed) memory that kernels on device `dev` may be given
bool is_device_ptr(const void* p, int dev) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return gi::classify_pointer((int)a.type, a.device, dev) == gi::kPtrDevice;
}

bool batch_kernel_k(uint32_t k) { return k == 2 || k == 3 || k == 5 || k == 9 || k == 17; }

// Fan-outs chosen per size class (floor(log2 n)) by gi_batch_tune_fanouts with
// GI_TUNE_RECORD, per key width; 0 = nothing recorded.  Process-wide.
std::mutex g_fanout_mu;
uint32_t g_fanout_table[2][64] = {};

// The fan-out an index of n keys takes when the caller leaves it to the library:
// the recorded choice of its size class, else k = 3 for at most 32 KB of keys and
// k = 5 above.  Measured in a batch of 1024 indexes of 2^8..2^20 u64 keys
// (gi_batch_tune_fanouts, lookups of each size class alone): k = 3 fastest at
// 2^10..2^12 keys (by 5-10%), k = 5 from 2^15 keys up (by 1-20%), the two within
// 3% elsewhere; Eytzinger order (k = 2) never fastest in a batch, although it is
// for single indexes of 2^15..2^19 keys.  Key bytes set the bound for u32 keys.
uint32_t auto_fanout(int key_bytes, uint64_t n) {
  if (n == 0) return 5;
  const uint32_t cls = 63 - (uint32_t)__builtin_clzll(n);
  {
    std::lock_guard<std::mutex> lk(g_fanout_mu);
    const uint32_t k = g_fanout_table[key_bytes == 8 ? 1 : 0][cls];
    if (k) return k;
  }
  return n * (uint64_t)key_bytes <= (1ull << 15) ? 3u : 5u;
}

// per-index pinning: the top levels whose slots fit in the budget (whole index if small)
void choose_pinning(gi::BatchDesc& d, uint32_t k, int key_bytes, uint32_t budget) {
  d.smem_levels = 0;
  d.smem_slots = 0;
  if (d.n == 0 || k < 2) return;
  uint64_t slots = 0, width = k - 1;
  for (uint32_t l = 0; l < d.levels; ++l) {
    const uint64_t next = slots + width;  // k^(l+1) - 1 slots: whole levels 0..l
    const uint64_t need = std::min<uint64_t>(next, (d.n + k - 2) / (k - 1) * (k - 1));
    if (need * key_bytes > budget) break;
    slots = next;
    d.smem_levels = l + 1;
    d.smem_slots = (uint32_t)need;
    if (need >= d.n) break;
    width *= k;
  }
}

// Per-index descriptors (levels, pinning, fan-out) from b->kidx_host, uploaded
// with the fan-out table; the bucket-sort variant of the layout is made ready.
cudaError_t apply_fanouts(gi_batch* b) {
  bool uniform = true;
  for (uint32_t i = 1; i < b->B; ++i) uniform &= b->kidx_host[i] == b->kidx_host[0];
  b->k = uniform ? b->kidx_host[0] : gi::kBatchMixed;
  b->layout = (uniform && b->k == 0) ? GI_SORTED : GI_EYTZINGER_KARY;
  for (uint32_t i = 0; i < b->B; ++i) {
    gi::BatchDesc& d = b->desc_host[i];
    const uint32_t k = b->kidx_host[i];
    d.k = k;
    d.levels = k >= 2 ? gi::make_geom(d.n, k).levels : 0;
    choose_pinning(d, k, b->key_bytes, b->smem_budget);
  }
  cudaError_t e = cudaMemcpy(b->d_desc, b->desc_host.data(), b->B * sizeof(gi::BatchDesc),
                             cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_kidx, b->kidx_host.data(), b->B * sizeof(uint32_t), cudaMemcpyHostToDevice);
  b->hy.k = b->k;
  b->hy.kidx = b->d_kidx;
  if (e == cudaSuccess) e = gi::batch_local_sort_setup(b->key_bytes, b->hy.k);
  return e;
}

void free_batch(gi_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  void* ptrs[] = {b->d_seg_start, b->d_seg_base, b->d_desc, b->d_tiles, b->d_chunks, b->keys,
                  b->rows, b->tmp_k[0], b->tmp_k[1], b->tmp_v[0], b->tmp_v[1], b->scratch,
                  b->dflags, b->d_cs, b->hy_mem, b->d_kidx};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  cudaGetLastError();
  delete b;
}
}  // namespace

extern "C" {

int gi_batch_create(const uint64_t* key_offsets, uint32_t B, int layout, uint32_t k, gi_batch** out) {
  gi::set_last_error("");
  if (!out) return bfail(GI_ERR_INVALID, "gi_batch_create: out is NULL");
  *out = nullptr;
  if (!key_offsets || B == 0) return bfail(GI_ERR_INVALID, "gi_batch_create: need B >= 1 and key offsets");
  const int lay = layout & 0xFF, kw = layout & ~0xFF;
  if (kw != GI_KEY_U32 && kw != GI_KEY_U64) return bfail(GI_ERR_INVALID, "gi_batch_create: bad key width");
  if (lay == GI_EYTZINGER_KARY) {
    if (!batch_kernel_k(k)) return bfail(GI_ERR_INVALID, "gi_batch_create: k must be 2, 3, 5, 9 or 17");
  } else if (lay == GI_SORTED) {
    k = 0;
  } else {
    return bfail(GI_ERR_INVALID, "gi_batch_create: layout must be GI_EYTZINGER_KARY or GI_SORTED");
  }
  if (key_offsets[0] != 0) return bfail(GI_ERR_INVALID, "gi_batch_create: key_offsets[0] must be 0");
  for (uint32_t i = 0; i < B; ++i) {
    if (key_offsets[i + 1] < key_offsets[i])
      return bfail(GI_ERR_INVALID, "gi_batch_create: key offsets decrease at %u", i);
    if (key_offsets[i + 1] - key_offsets[i] >= (1ull << 31))
      return bfail(GI_ERR_INVALID, "gi_batch_create: index %u has 2^31 keys or more", i);
  }
  gi_batch* b = new gi_batch();
  cudaGetDevice(&b->device);
  b->B = B;
  b->layout = lay;
  b->k = k;
  b->key_bytes = kw == GI_KEY_U64 ? 8 : 4;
  b->key_off.assign(key_offsets, key_offsets + B + 1);
  b->n = key_offsets[B];
  const int kb = b->key_bytes;
  // padded, 256-byte aligned region per index, >= 64 max-key slots after each
  const uint64_t align_slots = 256 / kb;
  std::vector<uint64_t> base(B);
  uint64_t cur = 0;
  b->desc_host.resize(B);
  for (uint32_t i = 0; i < B; ++i) {
    const uint64_t n = key_offsets[i + 1] - key_offsets[i];
    base[i] = cur;
    cur += (n + 64 + align_slots - 1) / align_slots * align_slots;
    gi::BatchDesc& d = b->desc_host[i];
    d = gi::BatchDesc{};
    d.base = base[i];
    d.n = n;
  }
  b->kidx_host.assign(B, lay == GI_SORTED ? 0u : k);
  const uint64_t slots_total = cur + align_slots;
  // tiles (radix) and chunks (histogram), host-built once
  const uint32_t tile = gi::batch_sort_tile(kb);
  std::vector<gi::BatchTile> tiles, chunks;
  std::vector<uint32_t> tile0(B + 1);  // first tile of every index
  for (uint32_t i = 0; i < B; ++i) {
    const uint64_t s0 = key_offsets[i], n = key_offsets[i + 1] - s0;
    tile0[i] = (uint32_t)tiles.size();
    for (uint64_t t = 0, l = 0; t < n; t += tile, ++l)
      tiles.push_back(gi::BatchTile{s0 + t, i, (uint32_t)std::min<uint64_t>(tile, n - t), (uint32_t)l, 0});
    for (uint64_t t = 0, l = 0; t < n; t += gi::kBatchChunk, ++l)
      chunks.push_back(gi::BatchTile{s0 + t, i, (uint32_t)std::min<uint64_t>(gi::kBatchChunk, n - t), (uint32_t)l, 0});
  }
  tile0[B] = (uint32_t)tiles.size();  // device memory bounds the keys far below 2^32 tiles
  b->ntiles = tiles.size();
  b->nchunks = chunks.size();
  auto bail = [&](int rc) {
    free_batch(b);
    return rc;
  };
#define GI_B(call, what)                                      \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return bail(bcuda(e_, what));      \
  } while (0)
  b->keys_bytes = slots_total * kb;
  GI_B(cudaMalloc(&b->keys, b->keys_bytes), "batch keys");
  GI_B(cudaMalloc((void**)&b->rows, slots_total * 4), "batch rows");
  for (int i = 0; i < 2; ++i) {
    GI_B(cudaMalloc(&b->tmp_k[i], (b->n + 64) * kb), "batch sort buffer");
    GI_B(cudaMalloc((void**)&b->tmp_v[i], (b->n + 64) * 4), "batch sort buffer");
  }
  GI_B(cudaMalloc(&b->scratch, gi::batch_sort_scratch_bytes(b->ntiles, B, kb)), "batch sort scratch");
  GI_B(cudaMalloc((void**)&b->d_seg_start, (B + 1) * 8), "batch tables");
  GI_B(cudaMalloc((void**)&b->d_seg_base, B * 8), "batch tables");
  GI_B(cudaMalloc((void**)&b->d_desc, B * sizeof(gi::BatchDesc)), "batch tables");
  GI_B(cudaMalloc((void**)&b->d_tiles, std::max<size_t>(1, tiles.size()) * sizeof(gi::BatchTile)), "batch tables");
  GI_B(cudaMalloc((void**)&b->d_chunks, std::max<size_t>(1, chunks.size()) * sizeof(gi::BatchTile)), "batch tables");
  GI_B(cudaMalloc((void**)&b->d_cs, (B + 1) * 8), "batch tables");
  GI_B(cudaMalloc((void**)&b->d_kidx, B * sizeof(uint32_t)), "batch tables");
  GI_B(cudaMalloc((void**)&b->dflags, 256), "batch status");
  GI_B(cudaMemset(b->dflags, 0, 256), "batch status");
  {  // tables of the hybrid build: per-index plans and slot maps, MSD window counts
    GI_B(cudaMalloc(&b->hy_mem, gi::batch_hybrid_bytes(B, b->ntiles)), "batch tables");
    char* q = (char*)b->hy_mem;
    auto take = [&](size_t bytes) { char* r = q; q += (bytes + 255) & ~size_t(255); return r; };
    b->hy.plan = (gi::BatchPlan*)take(sizeof(gi::BatchPlan) * B);
    b->hy.slot_maps = (gi::SlotMap*)take(sizeof(gi::SlotMap) * B);
    b->hy.hist_w = (unsigned long long*)take(sizeof(uint64_t) * (uint64_t)B * 256);
    b->hy.offs_w = (unsigned long long*)take(sizeof(uint64_t) * (uint64_t)B * 256);
    b->hy.counter = (uint32_t*)take(sizeof(uint32_t));
    uint32_t* d_tile0 = (uint32_t*)take(sizeof(uint32_t) * (B + 1));
    b->hy.tile0 = d_tile0;
    b->hy.prefix_msd = (uint32_t*)take(sizeof(uint32_t) * (B + 1));
    b->hy.prefix_lsd = (uint32_t*)take(sizeof(uint32_t) * (B + 1));
    b->hy.list_msd = (uint32_t*)take(sizeof(uint32_t) * (b->ntiles + 1));
    b->hy.list_lsd = (uint32_t*)take(sizeof(uint32_t) * (b->ntiles + 1));
    b->hy.buckets = (uint32_t*)take(sizeof(uint32_t) * 3 * (uint64_t)B * 257);
    b->hy.bucket_count = (uint32_t*)take(3 * sizeof(uint32_t));
    b->hy.xor_or = (unsigned long long*)take(sizeof(uint64_t) * B);
    GI_B(cudaMemcpy(d_tile0, tile0.data(), sizeof(uint32_t) * (B + 1), cudaMemcpyHostToDevice), "batch tables");
    b->hy.out_k = b->keys;
    b->hy.out_v = b->rows;
    b->hy.seg_base = b->d_seg_base;
  }
  GI_B(apply_fanouts(b), "batch tables");
  GI_B(cudaMemcpy(b->d_seg_start, key_offsets, (B + 1) * 8, cudaMemcpyHostToDevice), "batch tables");
  GI_B(cudaMemcpy(b->d_seg_base, base.data(), B * 8, cudaMemcpyHostToDevice), "batch tables");
  if (!tiles.empty())
    GI_B(cudaMemcpy(b->d_tiles, tiles.data(), tiles.size() * sizeof(gi::BatchTile), cudaMemcpyHostToDevice), "batch tables");
  if (!chunks.empty())
    GI_B(cudaMemcpy(b->d_chunks, chunks.data(), chunks.size() * sizeof(gi::BatchTile), cudaMemcpyHostToDevice), "batch tables");
  // the shared-memory budget stays below 48 KB (option bound), so launches need no
  // attribute change and can be captured in a graph
#undef GI_B
  *out = b;
  return GI_OK;
}

int gi_batch_set_stream(gi_batch* b, void* stream) {
  gi::set_last_error("");
  if (!b) return bfail(GI_ERR_INVALID, "gi_batch_set_stream: NULL batch");
  b->stream = (cudaStream_t)stream;
  return GI_OK;
}

int gi_batch_build(gi_batch* b, const void* keys, const uint32_t* rowids) {
  gi::set_last_error("");
  if (!b) return bfail(GI_ERR_INVALID, "gi_batch_build: NULL batch");
  if (b->n && (!is_device_ptr(keys, b->device) || !is_device_ptr(rowids, b->device)))
    return bfail(GI_ERR_INVALID, "gi_batch_build: keys and rowids must be device memory of the batch's device");
  cudaStream_t s = b->stream;
  // max-key padding after every index first: the bucket sort writes the layouts
  cudaError_t e = cudaMemsetAsync(b->keys, 0xFF, b->keys_bytes, s);
  if (e != cudaSuccess) return bcuda(e, "gi_batch_build: padding");
  e = gi::batch_sort(keys, rowids, b->tmp_k, b->tmp_v, b->n, b->key_bytes, b->d_seg_start, b->B,
                     b->d_tiles, b->ntiles, b->d_chunks, b->nchunks, b->scratch, b->dflags, s,
                     &b->result, &b->hy);
  if (e != cudaSuccess) return bcuda(e, "gi_batch_build: sort");
  if (b->result >= 0) {  // indexes whose plan fell back to the LSD passes
    e = gi::batch_gather(b->tmp_k[b->result], b->tmp_v[b->result], b->keys, b->rows, b->d_tiles,
                         b->ntiles, b->d_seg_start, b->d_seg_base, b->k, b->key_bytes, b->dflags, s,
                         &b->hy, b->B);
    if (e != cudaSuccess) return bcuda(e, "gi_batch_build: permutation");
  }
  return GI_OK;
}

int gi_batch_point_lookup(gi_batch* b, const void* queries, const uint64_t* query_offsets, uint64_t m,
                          uint32_t* out_rowids) {
  gi::set_last_error("");
  if (!b) return bfail(GI_ERR_INVALID, "gi_batch_point_lookup: NULL batch");
  if (m == 0) return GI_OK;
  if (!is_device_ptr(queries, b->device) || !is_device_ptr(query_offsets, b->device) ||
      !is_device_ptr(out_rowids, b->device))
    return bfail(GI_ERR_INVALID, "gi_batch_point_lookup: queries, offsets and output must be device memory of the batch's device");
  cudaStream_t s = b->stream;
  gi::bt::k_chunk_starts<<<1, 1024, 0, s>>>(query_offsets, b->B, b->chunk, b->d_cs);
  const unsigned grid = (unsigned)(gi::sm_count() * b->blocks_per_sm);
  const size_t smem = b->k != 0 ? b->smem_budget + 256 : 0;
#define GI_BP(K, KF)                                                                           \
  gi::bt::k_batch_point<K, KF><<<grid, 256, smem, s>>>((const K*)b->keys, b->rows, b->d_desc, \
                                                       query_offsets, b->d_cs, b->B,         \
                                                       (const K*)queries, out_rowids, b->chunk, \
                                                       b->dflags)
  const bool wide = b->k == gi::kBatchMixed &&
                    std::any_of(b->kidx_host.begin(), b->kidx_host.end(), [](uint32_t k) { return k >= 9; });
  if (b->key_bytes == 8) {
    switch (b->k) {
      case gi::kBatchMixed:
        if (wide) GI_BP(uint64_t, -2); else GI_BP(uint64_t, -1);
        break;
      case 0: GI_BP(uint64_t, 0); break;
      case 2: GI_BP(uint64_t, 2); break;
      case 3: GI_BP(uint64_t, 3); break;
      case 5: GI_BP(uint64_t, 5); break;
      case 9: GI_BP(uint64_t, 9); break;
      default: GI_BP(uint64_t, 17); break;
    }
  } else {
    switch (b->k) {
      case gi::kBatchMixed:
        if (wide) GI_BP(uint32_t, -2); else GI_BP(uint32_t, -1);
        break;
      case 0: GI_BP(uint32_t, 0); break;
      case 2: GI_BP(uint32_t, 2); break;
      case 3: GI_BP(uint32_t, 3); break;
      case 5: GI_BP(uint32_t, 5); break;
      case 9: GI_BP(uint32_t, 9); break;
      default: GI_BP(uint32_t, 17); break;
    }
  }
#undef GI_BP
  gi::count_launch(2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return bcuda(e, "gi_batch_point_lookup");
  return GI_OK;
}

int gi_batch_sync(gi_batch* b) {
  gi::set_last_error("");
  if (!b) return bfail(GI_ERR_INVALID, "gi_batch_sync: NULL batch");
  uint32_t f = 0;
  cudaError_t e = cudaMemcpyAsync(&f, b->dflags, 4, cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(e, "gi_batch_sync");
  if (f) {  // reported once: the next build starts from a clean status
    e = cudaMemsetAsync(b->dflags, 0, 4, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(e, "gi_batch_sync: status reset");
  }
  if (f & gi::kFlagTimeout) return bfail(GI_ERR_TIMEOUT, "a bounded device-side wait gave up");
  if (f & gi::kFlagReservedRowid) return bfail(GI_ERR_INVALID, "a rowID equals the reserved value GI_MISS");
  return GI_OK;
}

int gi_batch_copy_index(const gi_batch* b, uint32_t i, void* keys_out, uint32_t* rowids_out) {
  gi::set_last_error("");
  if (!b || i >= b->B) return bfail(GI_ERR_INVALID, "gi_batch_copy_index: bad batch or index");
  const gi::BatchDesc& d = b->desc_host[i];
  cudaError_t e = cudaSuccess;
  if (keys_out && d.n)
    e = cudaMemcpyAsync(keys_out, (const char*)b->keys + d.base * b->key_bytes, d.n * b->key_bytes,
                        cudaMemcpyDefault, b->stream);
  if (e == cudaSuccess && rowids_out && d.n)
    e = cudaMemcpyAsync(rowids_out, b->rows + d.base, d.n * 4, cudaMemcpyDefault, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(e, "gi_batch_copy_index");
  return GI_OK;
}

int gi_batch_set_fanouts(gi_batch* b, const uint32_t* ks) {
  gi::set_last_error("");
  if (!b) return bfail(GI_ERR_INVALID, "gi_batch_set_fanouts: NULL batch");
  std::vector<uint32_t> next(b->B);
  for (uint32_t i = 0; i < b->B; ++i) {
    next[i] = ks ? ks[i] : auto_fanout(b->key_bytes, b->desc_host[i].n);
    if (!gi::batch_fanout_ok(next[i]))
      return bfail(GI_ERR_INVALID, "gi_batch_set_fanouts: index %u: fan-out %u is not 0, 2, 3, 5, 9 or 17",
                   i, next[i]);
  }
  const std::vector<uint32_t> prev = b->kidx_host;
  b->kidx_host = next;
  cudaError_t e = cudaStreamSynchronize(b->stream);  // no build or lookup may still read the tables
  if (e == cudaSuccess) e = apply_fanouts(b);
  if (e != cudaSuccess) {
    b->kidx_host = prev;
    apply_fanouts(b);
    return bcuda(e, "gi_batch_set_fanouts");
  }
  return GI_OK;
}

int gi_batch_get_fanouts(const gi_batch* b, uint32_t* ks_out) {
  gi::set_last_error("");
  if (!b || !ks_out) return bfail(GI_ERR_INVALID, "gi_batch_get_fanouts: NULL argument");
  std::copy(b->kidx_host.begin(), b->kidx_host.end(), ks_out);
  return GI_OK;
}

int gi_batch_tune_fanouts(gi_batch* b, const void* keys, const uint32_t* rowids, const void* queries,
                          const uint64_t* query_offsets, uint64_t m, uint32_t reps, int flags,
                          uint32_t* ks_out, double* class_ms) {
  gi::set_last_error("");
  if (!b) return bfail(GI_ERR_INVALID, "gi_batch_tune_fanouts: NULL batch");
  if (flags & ~(GI_TUNE_APPLY | GI_TUNE_RECORD)) return bfail(GI_ERR_INVALID, "gi_batch_tune_fanouts: unknown flags");
  if (!is_device_ptr(queries, b->device) || !is_device_ptr(query_offsets, b->device) ||
      (b->n && (!is_device_ptr(keys, b->device) || !is_device_ptr(rowids, b->device))))
    return bfail(GI_ERR_INVALID, "gi_batch_tune_fanouts: keys, rowids, queries and offsets must be device memory");
  if (reps == 0) reps = 5;
  const uint32_t B = b->B;
  const int kb = b->key_bytes;
  const cudaStream_t s = b->stream;
  static const uint32_t cand[5] = {2, 3, 5, 9, 17};
  std::vector<uint64_t> qo(B + 1);
  cudaError_t e = cudaMemcpy(qo.data(), query_offsets, (B + 1) * 8, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return bcuda(e, "gi_batch_tune_fanouts: offsets");
  if (qo[B] != m) return bfail(GI_ERR_INVALID, "gi_batch_tune_fanouts: query_offsets[B] != m");
  // size classes floor(log2 n); the probes of each class gathered into one run
  std::vector<int> cls(B, -1);
  std::vector<uint64_t> cls_probes(64, 0);
  for (uint32_t i = 0; i < B; ++i) {
    const uint64_t n = b->desc_host[i].n;
    if (n) cls[i] = 63 - __builtin_clzll(n);
    if (cls[i] >= 0) cls_probes[cls[i]] += qo[i + 1] - qo[i];
  }
  std::vector<int> present;
  std::vector<uint64_t> cls_base(64, 0);
  uint64_t acc = 0;
  for (int c = 0; c < 64; ++c)
    if (cls_probes[c]) {
      present.push_back(c);
      cls_base[c] = acc;
      acc += cls_probes[c];
    }
  char* qbuf = nullptr;
  uint64_t* offs = nullptr;
  uint32_t* dout = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto cleanup = [&] {
    cudaStreamSynchronize(s);
    cudaFree(qbuf);
    cudaFree(offs);
    cudaFree(dout);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  e = cudaMalloc((void**)&qbuf, std::max<uint64_t>(acc, 1) * kb);
  if (e == cudaSuccess) e = cudaMalloc((void**)&offs, std::max<size_t>(present.size(), 1) * (B + 1) * 8);
  if (e == cudaSuccess) e = cudaMalloc((void**)&dout, std::max<uint64_t>(acc, 1) * 4);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cleanup();
    return bcuda(e, "gi_batch_tune_fanouts: scratch");
  }
  std::vector<uint64_t> oc(B + 1);
  for (size_t ci = 0; ci < present.size() && e == cudaSuccess; ++ci) {
    const int c = present[ci];
    uint64_t run = 0;
    for (uint32_t i = 0; i < B && e == cudaSuccess; ++i) {
      oc[i] = run;
      const uint64_t np = cls[i] == c ? qo[i + 1] - qo[i] : 0;
      if (np)
        e = cudaMemcpyAsync(qbuf + (cls_base[c] + run) * kb, (const char*)queries + qo[i] * kb, np * kb,
                            cudaMemcpyDeviceToDevice, s);
      run += np;
    }
    oc[B] = run;
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(offs + ci * (B + 1), oc.data(), (B + 1) * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // oc is reused by the next class
  }
  if (e != cudaSuccess) {
    cleanup();
    return bcuda(e, "gi_batch_tune_fanouts: gathering the probes");
  }
  const std::vector<uint32_t> orig = b->kidx_host;
  std::vector<double> t(64 * 5, -1.0);
  int rc = GI_OK;
  for (int ki = 0; ki < 5 && rc == GI_OK; ++ki) {
    std::vector<uint32_t> all(B, cand[ki]);
    rc = gi_batch_set_fanouts(b, all.data());
    if (rc == GI_OK) rc = gi_batch_build(b, keys, rowids);
    for (size_t ci = 0; ci < present.size() && rc == GI_OK; ++ci) {
      const int c = present[ci];
      const void* qc = qbuf + cls_base[c] * kb;
      double best = 1e30;
      for (uint32_t r = 0; r <= reps && rc == GI_OK; ++r) {  // the first run is not timed
        cudaEventRecord(e0, s);
        rc = gi_batch_point_lookup(b, qc, offs + ci * (B + 1), cls_probes[c], dout);
        cudaEventRecord(e1, s);
        e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) rc = bcuda(e, "gi_batch_tune_fanouts: timing");
        float ms = 0.f;
        if (rc == GI_OK && r > 0 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) best = std::min(best, (double)ms);
      }
      t[c * 5 + ki] = best;
    }
    if (rc == GI_OK) rc = gi_batch_sync(b);
  }
  cleanup();
  std::vector<uint32_t> choice(64, 0);
  for (int c : present) {
    int bi = 0;
    for (int ki = 1; ki < 5; ++ki)
      if (t[c * 5 + ki] < t[c * 5 + bi]) bi = ki;
    choice[c] = cand[bi];
  }
  std::vector<uint32_t> chosen(B);
  for (uint32_t i = 0; i < B; ++i)
    chosen[i] = cls[i] >= 0 && choice[cls[i]] ? choice[cls[i]] : auto_fanout(kb, b->desc_host[i].n);
  // the batch ends with the chosen fan-outs (APPLY) or those it had, built
  const int rc2 = gi_batch_set_fanouts(b, (flags & GI_TUNE_APPLY) && rc == GI_OK ? chosen.data() : orig.data());
  if (rc == GI_OK) rc = rc2;
  if (rc == GI_OK) rc = gi_batch_build(b, keys, rowids);
  if (rc == GI_OK) rc = gi_batch_sync(b);
  if (rc != GI_OK) return rc;
  if (flags & GI_TUNE_RECORD) {
    std::lock_guard<std::mutex> lk(g_fanout_mu);
    for (int c : present) g_fanout_table[kb == 8 ? 1 : 0][c] = choice[c];
  }
  if (ks_out) std::copy(chosen.begin(), chosen.end(), ks_out);
  if (class_ms) std::copy(t.begin(), t.end(), class_ms);
  return GI_OK;
}

void gi_batch_fanout_table_clear(void) {
  std::lock_guard<std::mutex> lk(g_fanout_mu);
  for (auto& row : g_fanout_table)
    for (uint32_t& k : row) k = 0;
}

int gi_batch_set_option(gi_batch* b, int option, int64_t v) {
  gi::set_last_error("");
  if (!b) return bfail(GI_ERR_INVALID, "gi_batch_set_option: NULL batch");
  switch (option) {
    case GI_BATCH_OPT_CHUNK:
      if (v < 32 || v > (1 << 20)) return bfail(GI_ERR_INVALID, "chunk must be in [32, 2^20]");
      b->chunk = (uint32_t)v;
      return GI_OK;
    case GI_BATCH_OPT_BLOCKS_PER_SM:
      if (v < 1 || v > 32) return bfail(GI_ERR_INVALID, "blocks per SM must be in [1, 32]");
      b->blocks_per_sm = (int)v;
      return GI_OK;
    case GI_BATCH_OPT_SMEM_BUDGET: {
      if (v < 0 || v > 40 * 1024) return bfail(GI_ERR_INVALID, "shared-memory budget must be in [0, 40 KiB]");
      b->smem_budget = (uint32_t)v;
      for (uint32_t i = 0; i < b->B; ++i)
        choose_pinning(b->desc_host[i], b->kidx_host[i], b->key_bytes, b->smem_budget);
      cudaError_t e = cudaMemcpy(b->d_desc, b->desc_host.data(), b->B * sizeof(gi::BatchDesc),
                                 cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return bcuda(e, "gi_batch_set_option");
      return GI_OK;
    }
  }
  return bfail(GI_ERR_INVALID, "gi_batch_set_option: unknown option %d", option);
}

}  // extern "C"

namespace gi {

cudaStream_t batch_stream(const gi_batch* b) { return b->stream; }

int batch_device(const gi_batch* b) { return b->device; }

int64_t batch_option(const gi_batch* b, int option) {
  switch (option) {
    case GI_BATCH_OPT_CHUNK: return b->chunk;
    case GI_BATCH_OPT_BLOCKS_PER_SM: return b->blocks_per_sm;
    case GI_BATCH_OPT_SMEM_BUDGET: return b->smem_budget;
  }
  return -1;
}

}  // namespace gi

extern "C" {

uint64_t gi_batch_footprint_bytes(const gi_batch* b) {
  return b ? b->n * (uint64_t)(b->key_bytes + 4) : 0;
}

void gi_batch_destroy(gi_batch* b) { free_batch(b); }

}  // extern "C"
