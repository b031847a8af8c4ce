// Point and range lookups over uint32_t keys (instantiation unit).
#include "gi_lookup_typed.cuh"

namespace gi {

cudaError_t point_lookup_u32(const void* keys, const uint32_t* rows, const Geom& g,
                            const LookupCfg& c, const void* q, uint64_t m, uint32_t* out,
                            uint32_t* dflags, cudaStream_t s) {
  return pt::point_lookup_typed<uint32_t>((const uint32_t*)keys, rows, g, c, (const uint32_t*)q, m, out,
                                        dflags, s);
}

cudaError_t range_lookup_u32(const void* keys, const uint32_t* rows, const Geom& g,
                            const LookupCfg& c, const void* lo, const void* hi, uint64_t m,
                            uint64_t* offsets, uint32_t* out_rows, void* scratch,
                            bool counts_ready, cudaStream_t s) {
  return rg::range_lookup_typed<uint32_t>((const uint32_t*)keys, rows, g, c, (const uint32_t*)lo,
                                        (const uint32_t*)hi, m, offsets, out_rows, scratch,
                                        counts_ready, s);
}

cudaError_t range_fill_rows(const uint32_t* rows, const Geom& g, const LookupCfg& c,
                            const uint64_t* offsets, const uint64_t* lo_rank, uint64_t m,
                            uint32_t* out_rows, cudaStream_t s) {
  return rg::range_fill(rows, g, c, offsets, lo_rank, m, out_rows, s);
}

}  // namespace gi
