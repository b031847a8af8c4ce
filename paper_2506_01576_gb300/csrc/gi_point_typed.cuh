// Launch logic of the point-lookup kernels for one key type (included by
// gi_point_u32.cu / gi_point_u64.cu).
#pragma once

#include "gi_point_impl.cuh"

namespace gi {
namespace pt {

// Lane-group k-ary lookups, instantiated in gi_eks_{u32,u64}_{a,b}.cu; each sets
// *handled when it owns the requested (k, group) pair.
#define GI_EKS_DECL(NAME)                                                                      \
  cudaError_t NAME(const void* keys, const uint32_t* rows, const Geom& g, const LookupCfg& c, \
                   const void* q, uint64_t m, uint32_t* out, uint32_t* dflags, cudaStream_t s, \
                   bool* handled);
GI_EKS_DECL(eks_point_u64_a)
GI_EKS_DECL(eks_point_u64_b)
GI_EKS_DECL(eks_point_u32_a)
GI_EKS_DECL(eks_point_u32_b)

template <class Kern>
inline cudaError_t set_smem(Kern kern, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

inline unsigned grid_size(uint64_t threads_needed, int block, int blocks_per_sm) {
  if (blocks_per_sm > 0) return (unsigned)(sm_count() * blocks_per_sm);
  uint64_t g = (threads_needed + block - 1) / block;
  if (g == 0) g = 1;
  if (g > 0x7fffffffull) g = 0x7fffffffull;
  return (unsigned)g;
}

template <class K>
cudaError_t point_lookup_typed(const K* keys, const uint32_t* rows, const Geom& g,
                               const LookupCfg& c, const K* q, uint64_t m, uint32_t* out,
                               uint32_t* dflags, cudaStream_t s) {
  const int block = c.block;
  const int R = c.per_thread;
  if (c.reorder) {  // local lookup reordering (Section 7.4)
    uint64_t tiles = (m + kReorderTile - 1) / kReorderTile;
    const uint64_t cap = (uint64_t)sm_count() * 8;
    const unsigned grid = (unsigned)(tiles < cap ? (tiles ? tiles : 1) : cap);
    const K* kb = keys;
    bool done = true;
    if (c.layout == GI_SORTED) {
      k_point_reorder<K, 0, 2><<<grid, kReorderThreads, 0, s>>>(kb, rows, g.n, g.levels, q, m, out);
    } else if (c.layout == GI_EYTZINGER) {
      k_point_reorder<K, 1, 2><<<grid, kReorderThreads, 0, s>>>(kb, rows, g.n, g.levels, q, m, out);
    } else {
      switch (g.k) {
        case 3: k_point_reorder<K, 2, 3><<<grid, kReorderThreads, 0, s>>>(kb, rows, g.n, g.levels, q, m, out); break;
        case 5: k_point_reorder<K, 2, 5><<<grid, kReorderThreads, 0, s>>>(kb, rows, g.n, g.levels, q, m, out); break;
        case 9: k_point_reorder<K, 2, 9><<<grid, kReorderThreads, 0, s>>>(kb, rows, g.n, g.levels, q, m, out); break;
        case 17: k_point_reorder<K, 2, 17><<<grid, kReorderThreads, 0, s>>>(kb, rows, g.n, g.levels, q, m, out); break;
        default: done = false; break;  // other fan-outs: the plain kernels below
      }
    }
    if (done) {
      count_launch();
      return cudaGetLastError();
    }
  }
  if (c.layout == GI_SORTED) {
    const unsigned grid = grid_size(m, block, c.blocks_per_sm);
    k_bs_point<K><<<grid, block, 0, s>>>(keys, rows, g.n, q, m, out);
    count_launch();
    return cudaGetLastError();
  }
  const uint64_t slots = smem_slots_for_levels(c.layout, g, c.smem_levels, sizeof(K));
  const size_t smem = (size_t)((slots * sizeof(K) + 15) & ~15ull);
  if (c.layout == GI_EYTZINGER) {
    const unsigned grid = grid_size((m + R - 1) / R, block, c.blocks_per_sm);
    cudaError_t e = cudaErrorInvalidValue;
#define GI_EBS(RR, PFF)                                                                        \
  if (R == RR && c.prefetch == PFF) {                                                          \
    auto kern = k_ebs_point<K, RR, PFF>;                                                       \
    e = set_smem(kern, smem);                                                                  \
    if (e != cudaSuccess) return e;                                                            \
    kern<<<grid, block, smem, s>>>(keys, rows, g.n, g.levels, q, m, out, (uint32_t)slots,      \
                                   dflags);                                                    \
    count_launch();                                                                            \
    return cudaGetLastError();                                                                 \
  }
    GI_EBS(1, 0) GI_EBS(1, 2) GI_EBS(1, 3) GI_EBS(1, 4)
    GI_EBS(2, 0) GI_EBS(2, 2) GI_EBS(2, 3) GI_EBS(2, 4)
    GI_EBS(4, 0) GI_EBS(4, 2) GI_EBS(4, 3) GI_EBS(4, 4)
#undef GI_EBS
    return e;
  }
  // k-ary Eytzinger: the compiled (k, group) pairs live in gi_eks_*.cu
  {
    bool handled = false;
    cudaError_t e = sizeof(K) == 8
        ? eks_point_u64_a(keys, rows, g, c, q, m, out, dflags, s, &handled)
        : eks_point_u32_a(keys, rows, g, c, q, m, out, dflags, s, &handled);
    if (handled) return e;
    e = sizeof(K) == 8 ? eks_point_u64_b(keys, rows, g, c, q, m, out, dflags, s, &handled)
                       : eks_point_u32_b(keys, rows, g, c, q, m, out, dflags, s, &handled);
    if (handled) return e;
  }
  // any other k (or group): one thread per lookup
  const uint32_t k = g.k;
  const unsigned ggrid = grid_size(m, block, c.blocks_per_sm);
  k_eks_generic<K><<<ggrid, block, 0, s>>>(keys, rows, g.n, k, q, m, out, c.early_exit);
  count_launch();
  return cudaGetLastError();
}

}  // namespace pt
}  // namespace gi
