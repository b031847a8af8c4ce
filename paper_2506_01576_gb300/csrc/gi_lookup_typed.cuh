// Point- and range-lookup dispatch for one key type; included by
// gi_lookup_u32.cu and gi_lookup_u64.cu, which instantiate it.
#pragma once

#include "gi_point_typed.cuh"
#include "gi_range_impl.cuh"

namespace gi {
namespace rg {

// lanes per range in the count pass of the k-ary layout: one key per lane
inline int range_group(uint32_t k) {
  int g = 1;
  while (g < (int)k - 1 && g < 32) g <<= 1;
  return g;
}

// Range fill: rows of ranges [0, m) at their CSR offsets (absolute, so a caller
// may fill a sub-range by passing offsets + a and lo_rank + a with m = its count).
inline cudaError_t range_fill(const uint32_t* rows, const Geom& g, const LookupCfg& c,
                              const uint64_t* offsets, const uint64_t* lo_rank, uint64_t m,
                              uint32_t* out_rows, cudaStream_t s) {
  if (m == 0) return cudaSuccess;
  const int block = 256;
  uint64_t gr = (m + block - 1) / block;  // one lane per range
  if (gr > 0x7fffffffull) gr = 0x7fffffffull;
  const unsigned grid = (unsigned)(gr ? gr : 1);
  const SlotMap sm = make_slot_map(g);
  const bool narrow = g.n < (1ull << 32);  // 32-bit rank -> slot map
#define GI_F(L, KF)                                                                              \
  do {                                                                                        \
    if (narrow)                                                                               \
      k_range_fill<L, KF, uint32_t><<<grid, block, 0, s>>>(rows, g, sm, offsets, lo_rank, m,  \
                                                           out_rows);                         \
    else                                                                                      \
      k_range_fill<L, KF, uint64_t><<<grid, block, 0, s>>>(rows, g, sm, offsets, lo_rank, m,  \
                                                           out_rows);                         \
  } while (0)
  if (c.layout == GI_SORTED) {
    k_range_fill<0, 0, uint64_t><<<grid, block, 0, s>>>(rows, g, sm, offsets, lo_rank, m, out_rows);
  } else if (c.range_fill == 1) {  // level runs (Section 5)
    switch (c.layout == GI_EYTZINGER ? 2u : g.k) {
#define GI_RL(KF) case KF: k_range_fill_levels<KF><<<grid, block, 0, s>>>(rows, g, offsets, lo_rank, m, out_rows); break;
      GI_RL(2) GI_RL(3) GI_RL(4) GI_RL(5) GI_RL(8) GI_RL(9) GI_RL(16) GI_RL(17) GI_RL(32) GI_RL(33)
#undef GI_RL
      default: k_range_fill_levels<0><<<grid, block, 0, s>>>(rows, g, offsets, lo_rank, m, out_rows); break;
    }
  } else if (c.layout == GI_EYTZINGER) {
    GI_F(1, 2);
  } else {
    switch (g.k) {
#define GI_RF(KF) case KF: GI_F(2, KF); break;
      GI_RF(3) GI_RF(4) GI_RF(5) GI_RF(8) GI_RF(9) GI_RF(16) GI_RF(17) GI_RF(32) GI_RF(33)
#undef GI_RF
      default: GI_F(2, 0); break;
    }
  }
#undef GI_F
  count_launch();
  return cudaGetLastError();
}

template <class K>
cudaError_t range_lookup_typed(const K* keys, const uint32_t* rows, const Geom& g,
                               const LookupCfg& c, const K* lo, const K* hi, uint64_t m,
                               uint64_t* offsets, uint32_t* out_rows, void* scratch,
                               bool counts_ready, cudaStream_t s) {
  uint64_t* lo_rank = (uint64_t*)scratch;
  uint64_t* sums = (uint64_t*)((char*)scratch + align256(sizeof(uint64_t) * (m ? m : 1)));
  const uint64_t nb = (m + kScanTile - 1) / kScanTile;
  if (m == 0) return cudaMemsetAsync(offsets, 0, sizeof(uint64_t), s);
  if (!counts_ready) {
    const int block = 256;
    auto grid_for = [&](uint64_t threads) {
      uint64_t gr = (threads + block - 1) / block;
      return (unsigned)(gr > 0x7fffffffull ? 0x7fffffffull : (gr ? gr : 1));
    };
    if (c.layout == GI_SORTED) {
      k_range_count<K, 0, 0, 1><<<grid_for(m), block, 0, s>>>(keys, g, lo, hi, m, offsets, lo_rank);
    } else if (c.layout == GI_EYTZINGER) {
      k_range_count<K, 1, 0, 1><<<grid_for(m), block, 0, s>>>(keys, g, lo, hi, m, offsets, lo_rank);
    } else {
      bool done = false;
#define GI_RC(KF)                                                                            \
  if (!done && g.k == KF) {                                                                  \
    /* one thread per range when a node is at most 64 bytes, else one key per lane */       \
    constexpr bool SINGLE = (KF - 1) * sizeof(K) <= 64;                                      \
    constexpr int GG = SINGLE ? 1 : (KF - 1 <= 2) ? 2 : (KF - 1 <= 4) ? 4                    \
                     : (KF - 1 <= 8) ? 8 : (KF - 1 <= 16) ? 16 : 32;                         \
    k_range_count<K, 2, KF, GG><<<grid_for(m * GG), block, 0, s>>>(keys, g, lo, hi, m,       \
                                                                   offsets, lo_rank);        \
    done = true;                                                                             \
  }
      GI_RC(3) GI_RC(4) GI_RC(5) GI_RC(8) GI_RC(9) GI_RC(16) GI_RC(17) GI_RC(32) GI_RC(33)
#undef GI_RC
      if (!done)
        k_range_count<K, 2, 0, 1><<<grid_for(m), block, 0, s>>>(keys, g, lo, hi, m, offsets,
                                                                lo_rank);
    }
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(offsets, m, sums);
    k_scan_sums<<<1, 1024, 0, s>>>(sums, nb);
    k_scan_down<<<(unsigned)nb, kScanThreads, 0, s>>>(offsets, m, sums);
    count_launch(4);
    cudaError_t e = cudaMemcpyAsync(offsets + m, sums + nb, sizeof(uint64_t),
                                    cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
  }
  if (out_rows) return range_fill(rows, g, c, offsets, lo_rank, m, out_rows, s);
  return cudaGetLastError();
}

}  // namespace rg
}  // namespace gi
