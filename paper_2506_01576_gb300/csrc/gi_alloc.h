// Sizes of a single index's device arrays (host-only, no CUDA, so they are
// checked on the CPU against every read the lookup kernels make).
//
// Key array: the layout's keys (n, plus the empty slot 0 of Eytzinger order)
// followed by max-key padding up to the allocation end.  The lookups read whole
// k-ary nodes (k-1 keys from a node start below n) and stage whole nodes of the
// top levels; slots past the last key compare as "not less" than any probe, so
// no read needs a bounds check as long as it ends inside the allocation.  65
// padding keys cover a node of the widest fan-out (33) from any start below n.
#pragma once

#include <stddef.h>
#include <stdint.h>

namespace gi {

inline size_t round256(size_t x) { return (x + 255) & ~size_t(255); }

// bytes of the keys the layout stores; the padding starts here
inline size_t key_used_bytes(uint64_t n, int key_bytes, bool eytzinger) {
  return (size_t)(n + (eytzinger ? 1 : 0)) * (size_t)key_bytes;
}

inline size_t key_alloc_bytes(uint64_t n, int key_bytes) {
  return round256((size_t)(n + 1 + 64) * (size_t)key_bytes + 64);
}

inline size_t row_alloc_bytes(uint64_t n) { return round256((size_t)(n + 64) * 4); }

}  // namespace gi
