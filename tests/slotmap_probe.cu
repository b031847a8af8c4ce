// Host-side entry points onto the CUDA path's closed-form slot maps (the
// __host__ __device__ functions of paper_2506_01576_gb300/csrc/gi_internal.cuh),
// so CPU tests can check them against the paper's formulas at sizes no GPU
// test can build.  Test infrastructure; not part of the library.
#include "gi_internal.cuh"

namespace {

template <int KF>
uint32_t slot_of_rank_kf(uint32_t r, const gi::SlotMap& sm) {
  return gi::slot_of_rank<KF>(r, sm);
}

}  // namespace

extern "C" {

// k = 0 in the template: the fan-out read at run time (the generic kernels)
uint64_t sp_slot_to_rank(uint64_t n, uint32_t k, uint64_t t) {
  return gi::slot_to_rank<0>(t, gi::make_geom(n, k));
}

uint64_t sp_rank_to_slot(uint64_t n, uint32_t k, uint64_t r) {
  return gi::rank_to_slot<0>(r, gi::make_geom(n, k));
}

// the 32-bit level-table map (n < 2^32), runtime fan-out and, for the fan-outs
// the kernels compile in, the compile-time one; ~0u for a fan-out not compiled in
uint32_t sp_slot_of_rank(uint64_t n, uint32_t k, uint32_t r, int compiled) {
  const gi::SlotMap sm = gi::make_slot_map(gi::make_geom(n, k));
  if (!compiled) return gi::slot_of_rank<0>(r, sm);
  switch (k) {
    case 2: return slot_of_rank_kf<2>(r, sm);
    case 3: return slot_of_rank_kf<3>(r, sm);
    case 5: return slot_of_rank_kf<5>(r, sm);
    case 9: return slot_of_rank_kf<9>(r, sm);
    case 17: return slot_of_rank_kf<17>(r, sm);
  }
  return ~0u;
}

}  // extern "C"
