// CPU oracle for the static index (sorted / Eytzinger / k-ary Eytzinger).
//
// TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's
// CPU-baseline leg load this library.  It shares no code, header or table with
// the CUDA library: it is a plain, slow, obviously correct restatement of what
// the index computes.
//
// What the index answers (Section 1 of the paper): given pairs (key_j, rowID_j),
//   * a point lookup of X returns the rowID of the entry whose key is X;
//   * a range lookup [L, U] returns the rowIDs of all entries with L <= key <= U.
// Sorting the pairs and binary searching the sorted array (Section 3) reaches
// exactly that result, so the oracle is that definition written out with the
// standard library:
//   * sort by (key, input position)  -- ties keep input order;
//   * point(x): r = lower_bound(x); rowID[r] if key[r] == x, else MISS;
//   * range(L, U): empty if L > U, else lower_bound(L) then a forward scan while
//     key <= U, emitted in ascending (key, input position) order, as CSR.
// The Eytzinger / k-ary Eytzinger order (Sections 3, 4, 6) is given here by its
// textbook definition: the slots of a complete k-ary search tree stored level by
// level, filled with the sorted keys by an in-order traversal.  It is pinned in
// the tests against the paper's closed forms and printed examples.
//
// Build: g++ -O2 -std=c++17 -shared -fPIC oracle.cpp -o liboracle.so -pthread

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <thread>
#include <utility>
#include <vector>

namespace {

const uint32_t kMiss = 0xFFFFFFFFu;  // rowID reported for a point lookup that misses

template <class K>
void sort_pairs(const K* keys, const uint32_t* rowids, uint64_t n, K* out_keys,
                uint32_t* out_rowids) {
  // Section 3: the sorted array is produced by a key-value sort.
  std::vector<std::pair<K, uint64_t>> v(n);
  for (uint64_t j = 0; j < n; ++j) v[j] = {keys[j], j};
  std::sort(v.begin(), v.end());  // (key, input position): equal keys keep input order
  for (uint64_t i = 0; i < n; ++i) {
    out_keys[i] = v[i].first;
    out_rowids[i] = rowids[v[i].second];
  }
}

template <class F>
void parallel_for(uint64_t m, int threads, F f) {
  if (threads <= 1 || m < 4096) {
    f(0, m);
    return;
  }
  std::vector<std::thread> ts;
  uint64_t chunk = (m + threads - 1) / threads;
  for (int t = 0; t < threads; ++t) {
    uint64_t a = chunk * t, b = std::min<uint64_t>(m, a + chunk);
    if (a >= b) break;
    ts.emplace_back([=] { f(a, b); });
  }
  for (auto& t : ts) t.join();
}

template <class K>
void point_lookup(const K* skeys, const uint32_t* srows, uint64_t n, const K* q,
                  uint64_t m, uint32_t* out, int threads) {
  // Section 3: binary search of the sorted array; the entry found is the first
  // one whose key is not less than the probe (std::lower_bound).
  parallel_for(m, threads, [&](uint64_t a, uint64_t b) {
    for (uint64_t i = a; i < b; ++i) {
      const K* p = std::lower_bound(skeys, skeys + n, q[i]);
      uint64_t r = (uint64_t)(p - skeys);
      out[i] = (r < n && skeys[r] == q[i]) ? srows[r] : kMiss;
    }
  });
}

template <class K>
void range_counts(const K* skeys, uint64_t n, const K* lo, const K* hi, uint64_t m,
                  uint64_t* offsets, int threads) {
  // Section 1: a range lookup [L, U] returns all entries with L <= key <= U.
  // Counted here by the same lower_bound + forward scan that fills the rows.
  std::vector<uint64_t> cnt(m);
  parallel_for(m, threads, [&](uint64_t a, uint64_t b) {
    for (uint64_t i = a; i < b; ++i) {
      if (lo[i] > hi[i]) {
        cnt[i] = 0;
        continue;
      }
      uint64_t r = (uint64_t)(std::lower_bound(skeys, skeys + n, lo[i]) - skeys);
      uint64_t c = 0;
      while (r + c < n && skeys[r + c] <= hi[i]) ++c;
      cnt[i] = c;
    }
  });
  uint64_t run = 0;
  for (uint64_t i = 0; i < m; ++i) {
    offsets[i] = run;
    run += cnt[i];
  }
  offsets[m] = run;
}

template <class K>
void range_fill(const K* skeys, const uint32_t* srows, uint64_t n, const K* lo,
                const K* hi, uint64_t m, const uint64_t* offsets, uint32_t* out,
                int threads) {
  parallel_for(m, threads, [&](uint64_t a, uint64_t b) {
    for (uint64_t i = a; i < b; ++i) {
      if (lo[i] > hi[i]) continue;
      uint64_t r = (uint64_t)(std::lower_bound(skeys, skeys + n, lo[i]) - skeys);
      uint64_t o = offsets[i];
      while (r < n && skeys[r] <= hi[i]) out[o++] = srows[r++];
    }
  });
}

// In-order fill of the complete k-ary search tree (Sections 3, 6, Figs 5, 10).
// Node j (0-based) holds slots j*(k-1) .. j*(k-1)+k-2; its children are nodes
// j*k+1 .. j*k+k; a slot exists iff its index is < n.  Visiting child c, then
// slot c, for c = 0..k-2, then child k-1, hands out ranks in ascending order.
struct InorderFill {
  uint64_t n, k;
  uint64_t* slot_rank;
  uint64_t next = 0;
  void visit(uint64_t node) {
    uint64_t first = node * (k - 1);
    if (first >= n) return;
    for (uint64_t c = 0; c < k; ++c) {
      visit(node * k + 1 + c);
      if (c + 1 < k) {
        uint64_t s = first + c;
        if (s < n) slot_rank[s] = next++;
      }
    }
  }
};

}  // namespace

extern "C" {

int or_sort_pairs(const void* keys, const uint32_t* rowids, uint64_t n, int key_bytes,
                  void* out_keys, uint32_t* out_rowids) {
  if (key_bytes == 4)
    sort_pairs((const uint32_t*)keys, rowids, n, (uint32_t*)out_keys, out_rowids);
  else if (key_bytes == 8)
    sort_pairs((const uint64_t*)keys, rowids, n, (uint64_t*)out_keys, out_rowids);
  else
    return 1;
  return 0;
}

int or_point_lookup(const void* skeys, const uint32_t* srows, uint64_t n, int key_bytes,
                    const void* q, uint64_t m, uint32_t* out, int threads) {
  if (key_bytes == 4)
    point_lookup((const uint32_t*)skeys, srows, n, (const uint32_t*)q, m, out, threads);
  else if (key_bytes == 8)
    point_lookup((const uint64_t*)skeys, srows, n, (const uint64_t*)q, m, out, threads);
  else
    return 1;
  return 0;
}

int or_range_offsets(const void* skeys, uint64_t n, int key_bytes, const void* lo,
                     const void* hi, uint64_t m, uint64_t* offsets, int threads) {
  if (key_bytes == 4)
    range_counts((const uint32_t*)skeys, n, (const uint32_t*)lo, (const uint32_t*)hi, m,
                 offsets, threads);
  else if (key_bytes == 8)
    range_counts((const uint64_t*)skeys, n, (const uint64_t*)lo, (const uint64_t*)hi, m,
                 offsets, threads);
  else
    return 1;
  return 0;
}

int or_range_fill(const void* skeys, const uint32_t* srows, uint64_t n, int key_bytes,
                  const void* lo, const void* hi, uint64_t m, const uint64_t* offsets,
                  uint32_t* out, int threads) {
  if (key_bytes == 4)
    range_fill((const uint32_t*)skeys, srows, n, (const uint32_t*)lo, (const uint32_t*)hi,
               m, offsets, out, threads);
  else if (key_bytes == 8)
    range_fill((const uint64_t*)skeys, srows, n, (const uint64_t*)lo, (const uint64_t*)hi,
               m, offsets, out, threads);
  else
    return 1;
  return 0;
}

// slot_rank[s] = rank (position in sorted order) of the key stored in slot s of
// the k-ary Eytzinger array of n keys (k = 2: Eytzinger order, slot s stored at
// 1-based position s+1 behind the empty slot 0).
int or_layout_slot_rank(uint64_t n, uint32_t k, uint64_t* slot_rank) {
  if (k < 2) return 1;
  InorderFill f{n, k, slot_rank};
  if (n) f.visit(0);
  return f.next == n ? 0 : 2;
}

int or_hardware_threads(void) {
  unsigned h = std::thread::hardware_concurrency();
  return h ? (int)h : 1;
}

}  // extern "C"
