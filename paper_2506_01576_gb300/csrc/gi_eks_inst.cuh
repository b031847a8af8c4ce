// Instantiation unit body for the lane-group k-ary lookup kernel.  Included by
// gi_eks_{u32,u64}_{a,b}.cu with GI_EKS_KEY (key type), GI_EKS_LIST(X) (the
// (k, group) pairs of this unit) and GI_EKS_FN (entry point name) defined, so
// the instantiations compile as four parallel units.
#include "gi_point_typed.cuh"

namespace gi {
namespace pt {

cudaError_t GI_EKS_FN(const void* keys, const uint32_t* rows, const Geom& g, const LookupCfg& c,
                      const void* q, uint64_t m, uint32_t* out, uint32_t* dflags, cudaStream_t s,
                      bool* handled) {
  using K = GI_EKS_KEY;
  *handled = false;
  const int G = c.group, R = c.per_thread;
  const uint32_t k = g.k;
  const uint64_t slots = smem_slots_for_levels(c.layout, g, c.smem_levels, sizeof(K));
  const uint32_t smem_levels = slots ? (uint32_t)c.smem_levels : 0u;
  // dynamic shared memory: the staged slots plus slack for whole-group reads
  const size_t smem = slots ? (size_t)(((slots * sizeof(K) + 15) & ~15ull) + 256) : 0;
  // 32-bit slot arithmetic while s*k + k*(k-1) stays below 2^32 - 1
  const bool narrow = (uint64_t)g.n * k + (uint64_t)k * k < 0xFFFFFFFEull;
  const unsigned grid = grid_size((m + R - 1) / R * (uint64_t)G, c.block, c.blocks_per_sm);
  const uint32_t hot = (uint32_t)c.hot_levels, l1 = (uint32_t)c.l1_levels;
#define GI_L(KF, GG, RR, IDX)                                                                  \
  {                                                                                            \
    auto kern = k_eks_point<K, KF, GG, RR, IDX>;                                               \
    cudaError_t e = set_smem(kern, smem);                                                      \
    if (e != cudaSuccess) return e;                                                            \
    kern<<<grid, c.block, smem, s>>>((const K*)keys, rows, (IDX)g.n, g.levels, (const K*)q, m, \
                                     out, smem_levels, (uint32_t)slots, hot, l1, dflags);      \
  }
#define GI_X(KF, GG)                                                                           \
  if (k == KF && G == GG) {                                                                    \
    *handled = true;                                                                           \
    if (narrow) {                                                                              \
      if (R == 1) GI_L(KF, GG, 1, uint32_t) else if (R == 2) GI_L(KF, GG, 2, uint32_t)         \
      else GI_L(KF, GG, 4, uint32_t)                                                           \
    } else {                                                                                   \
      if (R == 1) GI_L(KF, GG, 1, uint64_t) else if (R == 2) GI_L(KF, GG, 2, uint64_t)         \
      else GI_L(KF, GG, 4, uint64_t)                                                           \
    }                                                                                          \
    count_launch();                                                                            \
    return cudaGetLastError();                                                                 \
  }
  GI_EKS_LIST(GI_X)
#undef GI_X
#undef GI_L
  return cudaSuccess;
}

}  // namespace pt
}  // namespace gi
