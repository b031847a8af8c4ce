// Point-lookup kernels, templated on the key type.  Included once per key type
// by gi_point_u32.cu / gi_point_u64.cu so the two instantiation sets compile in
// parallel.
//
//   k_bs_point   textbook lower_bound on the sorted array (Section 3, "BS").
//   k_ebs_point  Eytzinger descent i -> 2i + (E[i] < x), branch-free, several
//                independent lookups interleaved per thread, optional prefetch of
//                the descendants a few levels down (Section 3, "EBS").
//   k_eks_point  k-ary Eytzinger descent (Section 6.2, "EKS"): a group of G
//                lanes loads the k-1 pivots of one node in one coalesced access
//                (vector loads of 8, 16 or 32 contiguous bytes per lane), each
//                lane counts its pivots < x and the group sums the counts with a
//                shuffle butterfly (the paper's ballot + popc measured 1.0-2.3x
//                slower here), and the next node starts at s*k + (c+1)*(k-1).
//                G = 1 is "EKS (single)": one thread reads the whole node.
//   k_eks_generic  any k in [2, 33] at run time, one thread per lookup.
//
// The top tree levels can be pinned in shared memory (Section 7.3): each CTA
// copies slots [0, S) with one bulk asynchronous copy (cp.async.bulk, completion
// on an mbarrier, bounded wait) and reads them from there.  With a persistent
// grid (blocks_per_sm > 0) each CTA walks the probes with the static schedule
// of Section 7.2.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gi_internal.cuh"

namespace gi {
namespace pt {

constexpr uint64_t kNone = ~0ull;

// ---------------------------------------------------------------- shared-memory staging
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Copy `bytes` (multiple of 16, <= 227 KB) from global `src` to shared `dst`
// with one bulk copy.  Returns false if the bounded wait gave up.
__device__ __forceinline__ bool stage_bulk(void* dst, const void* src, uint32_t bytes,
                                           uint64_t* mbar, uint32_t* flags) {
  const uint32_t bar = smem_u32(mbar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
  }
  __syncthreads();
  uint32_t done = 0;
  for (uint32_t spin = 0; spin < kSpinLimit; ++spin) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar)
        : "memory");
    if (done) break;
  }
  if (!done) {
    atomicOr(flags, kFlagTimeout);
    // give the copy in flight a second bounded chance before the CTA may exit
    for (uint32_t spin = 0; spin < kSpinLimit && !done; ++spin) {
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n"
          " selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(done)
          : "r"(bar)
          : "memory");
    }
    return false;
  }
  return true;
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

template <class K>
__device__ __forceinline__ K ldg(const K* p) {
  return __ldg(p);
}

// ---------------------------------------------------------------- textbook binary search
template <class K>
__global__ void __launch_bounds__(512) k_bs_point(const K* __restrict__ keys,
                                                  const uint32_t* __restrict__ rows, uint64_t n,
                                                  const K* __restrict__ q, uint64_t m,
                                                  uint32_t* __restrict__ out) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    const K x = q[i];
    uint64_t lo = 0, len = n;
    while (len > 0) {
      const uint64_t half = len >> 1;
      if (keys[lo + half] < x) {
        lo += half + 1;
        len -= half + 1;
      } else {
        len = half;
      }
    }
    out[i] = (lo < n && keys[lo] == x) ? rows[lo] : GI_MISS;
  }
}

// ---------------------------------------------------------------- Eytzinger (k = 2)
// keys: 1-based (keys[0] is the empty slot), rows: 0-based (slot s -> rows[s-1]).
template <class K, int R, int PF>
__global__ void __launch_bounds__(512) k_ebs_point(const K* __restrict__ keys,
                                                   const uint32_t* __restrict__ rows, uint64_t n,
                                                   uint32_t levels, const K* __restrict__ q,
                                                   uint64_t m, uint32_t* __restrict__ out,
                                                   uint32_t smem_slots, uint32_t* flags) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint64_t mbar;
  const K* sm = (const K*)smem_raw;
  if (smem_slots) {
    const uint32_t bytes = (uint32_t)(((uint64_t)smem_slots * sizeof(K) + 15) & ~15ull);
    if (!stage_bulk(smem_raw, keys, bytes, &mbar, flags)) return;
  }
  const uint64_t threads = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (uint64_t first = tid; first < m; first += threads * R) {
    K x[R];
    uint64_t s[R];
    bool eq[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const uint64_t i = first + r * threads;
      x[r] = i < m ? q[i] : K(0);
      s[r] = 1;
      eq[r] = false;
    }
    for (uint32_t lv = 0; lv < levels; ++lv) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (s[r] <= n) {
          if (PF) {
            const uint64_t f = s[r] << PF;
            if (f <= n) prefetch_l2(keys + f);
          }
          const K v = s[r] < smem_slots ? sm[s[r]] : ldg(keys + s[r]);
          const bool right = v < x[r];
          eq[r] = right ? eq[r] : (v == x[r]);  // equality at the last left turn
          s[r] = 2 * s[r] + (right ? 1 : 0);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const uint64_t i = first + r * threads;
      if (i < m) {
        // undo the trailing right turns: the lower bound is the last left turn
        const uint64_t lb = s[r] >> __ffsll((long long)~s[r]);
        out[i] = (lb != 0 && eq[r]) ? ldg(rows + (lb - 1)) : GI_MISS;
      }
    }
  }
}

// ---------------------------------------------------------------- k-ary Eytzinger, lane groups
// P contiguous keys (8, 16, 32 or 64 bytes...) with the widest vector loads:
// 32-byte loads (ld.global.nc.v4.u64 / .v8.u32, sm_100+) where they fit.
template <class K>
__device__ __forceinline__ void ld32(const K* p, K* v) {
  if constexpr (sizeof(K) == 8) {
    unsigned long long a, b, c, d;
    asm volatile("ld.global.nc.v4.u64 {%0,%1,%2,%3}, [%4];"
                 : "=l"(a), "=l"(b), "=l"(c), "=l"(d)
                 : "l"(p));
    v[0] = a; v[1] = b; v[2] = c; v[3] = d;
  } else {
    uint32_t a[8];
    asm volatile("ld.global.nc.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]),
                   "=r"(a[6]), "=r"(a[7])
                 : "l"(p));
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = a[i];
  }
}

template <class K, int P>
__device__ __forceinline__ void vec_load(const K* p, K* v) {
  constexpr int BYTES = P * (int)sizeof(K);
  if constexpr (BYTES == 8) {
    const uint2 t = __ldg((const uint2*)p);
    if constexpr (sizeof(K) == 4) {
      v[0] = t.x;
      v[1] = t.y;
    } else {
      v[0] = ((uint64_t)t.y << 32) | t.x;
    }
  } else if constexpr (BYTES == 16) {
    if constexpr (sizeof(K) == 4) {
      const uint4 t = __ldg((const uint4*)p);
      v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else {
      const ulonglong2 t = __ldg((const ulonglong2*)p);
      v[0] = t.x; v[1] = t.y;
    }
  } else {
    constexpr int PER = 32 / (int)sizeof(K);
#pragma unroll
    for (int i = 0; i < BYTES / 32; ++i) ld32<K>(p + i * PER, v + i * PER);
  }
}

// ---- L2 eviction-priority hints (createpolicy + ld/st ...L2::cache_hint)
__device__ __forceinline__ uint64_t l2_policy(bool keep) {
  uint64_t pol;
  if (keep)
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  else
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

template <class K>
__device__ __forceinline__ K ld_hint(const K* p, uint64_t pol) {
  if constexpr (sizeof(K) == 8) {
    unsigned long long v;
    asm volatile("ld.global.nc.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(v) : "l"(p), "l"(pol));
    return (K)v;
  } else {
    uint32_t v;
    asm volatile("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return (K)v;
  }
}

// a streamed (read-once) value: skip L1, evict first from L2
template <class K>
__device__ __forceinline__ K ld_stream(const K* p, uint64_t pol) {
  if constexpr (sizeof(K) == 8) {
    unsigned long long v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.u64 %0, [%1], %2;"
                 : "=l"(v) : "l"(p), "l"(pol));
    return (K)v;
  } else {
    uint32_t v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.u32 %0, [%1], %2;"
                 : "=r"(v) : "l"(p), "l"(pol));
    return (K)v;
  }
}

__device__ __forceinline__ void st_stream(uint32_t* p, uint32_t v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.u32 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(pol) : "memory");
}

// P contiguous keys with the widest vector loads, under an L2 policy
template <class K, int P>
__device__ __forceinline__ void vec_load_hint(const K* p, K* v, uint64_t pol) {
  constexpr int BYTES = P * (int)sizeof(K);
  if constexpr (BYTES == 8) {
    if constexpr (sizeof(K) == 8) {
      v[0] = ld_hint<K>(p, pol);
    } else {
      uint32_t a, b;
      asm volatile("ld.global.nc.L2::cache_hint.v2.u32 {%0,%1}, [%2], %3;"
                   : "=r"(a), "=r"(b) : "l"(p), "l"(pol));
      v[0] = a; v[1] = b;
    }
  } else if constexpr (BYTES == 16) {
    if constexpr (sizeof(K) == 8) {
      unsigned long long a, b;
      asm volatile("ld.global.nc.L2::cache_hint.v2.u64 {%0,%1}, [%2], %3;"
                   : "=l"(a), "=l"(b) : "l"(p), "l"(pol));
      v[0] = a; v[1] = b;
    } else {
      uint32_t a, b, c, d;
      asm volatile("ld.global.nc.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
                   : "=r"(a), "=r"(b), "=r"(c), "=r"(d) : "l"(p), "l"(pol));
      v[0] = a; v[1] = b; v[2] = c; v[3] = d;
    }
  } else {
#pragma unroll
    for (int i = 0; i < BYTES / 32; ++i) {
      if constexpr (sizeof(K) == 8) {
        unsigned long long a, b, c, d;
        asm volatile("ld.global.nc.L2::cache_hint.v4.u64 {%0,%1,%2,%3}, [%4], %5;"
                     : "=l"(a), "=l"(b), "=l"(c), "=l"(d) : "l"(p + 4 * i), "l"(pol));
        v[4 * i] = a; v[4 * i + 1] = b; v[4 * i + 2] = c; v[4 * i + 3] = d;
      } else {
        uint32_t a[8];
        asm volatile("ld.global.nc.L2::cache_hint.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8], %9;"
                     : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]),
                       "=r"(a[6]), "=r"(a[7])
                     : "l"(p + 8 * i), "l"(pol));
#pragma unroll
        for (int j = 0; j < 8; ++j) v[8 * i + j] = a[j];
      }
    }
  }
}

// The same loads without allocating in L1 (deep tree levels: read once per lookup,
// they would only push the top levels out of L1).
template <class K, int P>
__device__ __forceinline__ void vec_load_hint_na(const K* p, K* v, uint64_t pol) {
  constexpr int BYTES = P * (int)sizeof(K);
  if constexpr (BYTES % 32 == 0) {
#pragma unroll
    for (int i = 0; i < BYTES / 32; ++i) {
      if constexpr (sizeof(K) == 8) {
        unsigned long long a, b, c, d;
        asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u64 {%0,%1,%2,%3}, [%4], %5;"
                     : "=l"(a), "=l"(b), "=l"(c), "=l"(d) : "l"(p + 4 * i), "l"(pol));
        v[4 * i] = a; v[4 * i + 1] = b; v[4 * i + 2] = c; v[4 * i + 3] = d;
      } else {
        uint32_t a[8];
        asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8], %9;"
                     : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]),
                       "=r"(a[6]), "=r"(a[7])
                     : "l"(p + 8 * i), "l"(pol));
#pragma unroll
        for (int j = 0; j < 8; ++j) v[8 * i + j] = a[j];
      }
    }
  } else if constexpr (BYTES == 16 && sizeof(K) == 8) {
    unsigned long long a, b;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.u64 {%0,%1}, [%2], %3;"
                 : "=l"(a), "=l"(b) : "l"(p), "l"(pol));
    v[0] = a; v[1] = b;
  } else if constexpr (BYTES == 16) {
    uint32_t a, b, c, d;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
                 : "=r"(a), "=r"(b), "=r"(c), "=r"(d) : "l"(p), "l"(pol));
    v[0] = a; v[1] = b; v[2] = c; v[3] = d;
  } else {
    vec_load_hint<K, P>(p, v, pol);
  }
}

template <class K>
__device__ __forceinline__ K ld_hint_na(const K* p, uint64_t pol) {
  return ld_stream<K>(p, pol);
}

template <class K, int KF, int G>
struct EksShape {
  static constexpr int N = KF - 1;           // pivots per node
  static constexpr int P = (N + G - 1) / G;  // pivots per lane
  // one contiguous vector per lane when the node splits evenly into 8-byte or
  // 16-byte pieces or whole 32-byte loads
  static constexpr int BYTES = P * (int)sizeof(K);
  static constexpr bool VEC = (N % G == 0) && (P >= 2 || sizeof(K) == 8) && ((P & (P - 1)) == 0) &&
                              (BYTES == 8 || BYTES == 16 || BYTES % 32 == 0);
};

// The lookup loop (Section 6.2).  Each group of G lanes owns R lookups at a
// time and walks all tree levels in lock step, so every warp is at the same
// level and the shared-memory / global choice is warp-uniform.  Slots past n
// hold the maximum key (written at build), so a node needs no per-pivot bounds
// check: c = #{pivots < x}; the lower-bound candidate is slot s+c if it exists;
// the next node starts at s*k + (c+1)*(k-1).  With one lane per lookup the
// candidate's key is kept in a register (pivot c of the node just read), so
// equality is resolved at the end with no further load of the key array; lane
// groups load it once at the end.
// Levels below l1_levels are read through L1 (the top of the tree stays there);
// deeper levels are not allocated in L1, and neither are rowIDs, probes and
// results, each read once.
template <class K, int KF, int G, int R, class IDX>
__global__ void __launch_bounds__(512) k_eks_point(const K* __restrict__ keys,
                                                   const uint32_t* __restrict__ rows, IDX n,
                                                   uint32_t levels, const K* __restrict__ q,
                                                   uint64_t m, uint32_t* __restrict__ out,
                                                   uint32_t smem_levels, uint32_t smem_slots,
                                                   uint32_t hot_levels, uint32_t l1_levels,
                                                   uint32_t* flags) {
  using S = EksShape<K, KF, G>;
  constexpr int N = S::N, P = S::P;
  constexpr IDX kNoCand = ~IDX(0);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint64_t mbar;
  const K* sm = (const K*)smem_raw;
  if (smem_slots) {
    const uint32_t bytes = (uint32_t)(((uint64_t)smem_slots * sizeof(K) + 15) & ~15ull);
    if (!stage_bulk(smem_raw, keys, bytes, &mbar, flags)) return;
  }
  const int lane = threadIdx.x & 31;
  const int gl = lane % G;
  const uint32_t gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane - gl));
  const uint64_t groups = ((uint64_t)gridDim.x * blockDim.x) / G;
  const uint64_t gid = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const IDX lane_off = S::VEC ? (IDX)(gl * P) : (IDX)gl;
  // Top `hot_levels` levels are kept in L2 (evict_last); deeper levels, rowIDs,
  // probes and results are touched once per lookup and evicted first.
  const uint64_t pol_keep = l2_policy(true), pol_stream = l2_policy(false);
  const bool in_l1 = l1_levels >= levels;  // the whole index read through L1

  for (uint64_t first = gid; first < m; first += groups * R) {
    K x[R], ckey[R];
    IDX s[R], cand[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const uint64_t i = first + r * groups;
      x[r] = i < m ? ld_stream<K>(q + i, pol_stream) : K(0);
      s[r] = i < m ? IDX(0) : n;  // s >= n: nothing (more) to do
      cand[r] = kNoCand;
      ckey[r] = K(0);
    }
    for (uint32_t lv = 0; lv < levels; ++lv) {
      K piv[R][P];
      const bool from_smem = lv < smem_levels;
      const uint64_t pol = lv < hot_levels ? pol_keep : pol_stream;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (s[r] < n) {
          const IDX at = s[r] + lane_off;
          if (from_smem) {
            if constexpr (S::VEC && S::BYTES >= 16) {
              // 16-byte shared loads (the staged region is 16-byte aligned)
              constexpr int PER = 16 / (int)sizeof(K);
#pragma unroll
              for (int i = 0; i < P / PER; ++i) {
                const uint4 t = *reinterpret_cast<const uint4*>(sm + at + i * PER);
                if constexpr (sizeof(K) == 8) {
                  piv[r][i * 2] = ((uint64_t)t.y << 32) | t.x;
                  piv[r][i * 2 + 1] = ((uint64_t)t.w << 32) | t.z;
                } else {
                  piv[r][i * 4] = t.x; piv[r][i * 4 + 1] = t.y;
                  piv[r][i * 4 + 2] = t.z; piv[r][i * 4 + 3] = t.w;
                }
              }
            } else {
#pragma unroll
              for (int p = 0; p < P; ++p) {
                const int j = S::VEC ? gl * P + p : gl + p * G;
                piv[r][p] = j < N ? sm[s[r] + j] : K(0);
              }
            }
          } else if constexpr (S::VEC) {
            if (lv < l1_levels) vec_load_hint<K, P>(keys + at, piv[r], pol);
            else vec_load_hint_na<K, P>(keys + at, piv[r], pol);
          } else {
            // one key per load: a node's keys share sectors, so they go through L1
            // at every level (without it each key is its own L2 request)
#pragma unroll
            for (int p = 0; p < P; ++p) {
              const int j = gl + p * G;
              piv[r][p] = j < N ? ld_hint<K>(keys + at + p * G, pol) : K(0);
            }
          }
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (s[r] < n) {
          // pivots < x held by this lane, then summed over the group (butterfly)
          uint32_t c = 0;
#pragma unroll
          for (int p = 0; p < P; ++p) {
            const int j = S::VEC ? gl * P + p : gl + p * G;  // pivot position in the node
            c += (j < N && piv[r][p] < x[r]) ? 1u : 0u;
          }
#pragma unroll
          for (int o = 1; o < G; o <<= 1) c += __shfl_xor_sync(gmask, c, o);
          if (c < (uint32_t)N && s[r] + c < n) {
            cand[r] = s[r] + c;
            if constexpr (G == 1) {  // pivot c of the node: the candidate's key
              if (!in_l1) {
                K mine = piv[r][0];
#pragma unroll
                for (int p = 1; p < P; ++p) mine = c == (uint32_t)p ? piv[r][p] : mine;
                ckey[r] = mine;
              }
            }
          }
          s[r] = s[r] * KF + (IDX)((c + 1) * N);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const uint64_t i = first + r * groups;
      if (i < m && gl == r % G) {
        uint32_t res = GI_MISS;
        // G > 1, or an index held in L1: the candidate's key is read once here
        // (an L1 hit for a small index, cheaper than selecting it at every level;
        // fetching it from its owner lane at every level measured 1.4-1.5x slower
        // for 4- and 8-lane groups)
        if (cand[r] != kNoCand &&
            ((G == 1 && !in_l1) ? ckey[r] : ld_hint<K>(keys + cand[r], pol_stream)) == x[r])
          res = in_l1 ? ld_hint<uint32_t>(rows + cand[r], pol_stream)  // small: via L1
                      : ld_stream<uint32_t>(rows + cand[r], pol_stream);
        st_stream(out + i, res, pol_stream);
      }
    }
  }
}

// ---------------------------------------------------------------- local lookup reordering
// Section 7.4: a CTA takes a tile of probes, sorts them in shared memory (keys
// with their positions, bitonic network), looks them up in sorted order --
// neighbouring lanes then walk nearly the same path and share cache lines --
// and puts each result back at its probe's position before one coalesced store.
constexpr int kReorderItems = 8;
constexpr int kReorderThreads = 256;
constexpr int kReorderTile = kReorderItems * kReorderThreads;

template <class K, int KIND, int KF>  // KIND 0: sorted (BS), 1: Eytzinger, 2: k-ary single
__device__ __forceinline__ uint32_t lookup_one(const K* __restrict__ keys,
                                               const uint32_t* __restrict__ rows, uint64_t n,
                                               uint32_t levels, K x) {
  if constexpr (KIND == 0) {
    uint64_t lo = 0, len = n;
    while (len > 0) {
      const uint64_t half = len >> 1;
      if (ldg(keys + lo + half) < x) {
        lo += half + 1;
        len -= half + 1;
      } else {
        len = half;
      }
    }
    return (lo < n && ldg(keys + lo) == x) ? ldg(rows + lo) : GI_MISS;
  } else if constexpr (KIND == 1) {
    uint64_t s = 1;
    bool eq = false;
    for (uint32_t lv = 0; lv < levels; ++lv) {
      if (s <= n) {
        const K v = ldg(keys + s);
        const bool right = v < x;
        eq = right ? eq : (v == x);
        s = 2 * s + (right ? 1 : 0);
      }
    }
    const uint64_t lb = s >> __ffsll((long long)~s);
    return (lb != 0 && eq) ? ldg(rows + (lb - 1)) : GI_MISS;
  } else {
    constexpr int N = KF - 1;
    uint64_t s = 0, cand = kNone;
    for (uint32_t lv = 0; lv < levels; ++lv) {
      if (s >= n) break;
      K piv[N];
      if constexpr (EksShape<K, KF, 1>::VEC) {
        vec_load<K, N>(keys + s, piv);
      } else {
#pragma unroll
        for (int p = 0; p < N; ++p) piv[p] = ldg(keys + s + p);
      }
      uint32_t c = 0;
#pragma unroll
      for (int p = 0; p < N; ++p) c += piv[p] < x ? 1u : 0u;
      if (c < (uint32_t)N && s + c < n) cand = s + c;
      s = s * KF + (uint64_t)(c + 1) * N;
    }
    return (cand != kNone && ldg(keys + cand) == x) ? ldg(rows + cand) : GI_MISS;
  }
}

template <class K, int KIND, int KF>
__global__ void __launch_bounds__(kReorderThreads) k_point_reorder(const K* __restrict__ keys,
                                                                  const uint32_t* __restrict__ rows,
                                                                  uint64_t n, uint32_t levels,
                                                                  const K* __restrict__ q, uint64_t m,
                                                                  uint32_t* __restrict__ out) {
  __shared__ K s_key[kReorderTile];
  __shared__ uint32_t s_pos[kReorderTile];
  __shared__ uint32_t s_res[kReorderTile];
  const int tid = threadIdx.x;
  for (uint64_t base = (uint64_t)blockIdx.x * kReorderTile; base < m;
       base += (uint64_t)gridDim.x * kReorderTile) {
    const uint32_t cnt = (uint32_t)min((uint64_t)kReorderTile, m - base);
    for (int i = tid; i < kReorderTile; i += kReorderThreads) {
      s_key[i] = i < (int)cnt ? q[base + i] : ~K(0);  // padding sorts last
      s_pos[i] = (uint32_t)i;
    }
    __syncthreads();
    // bitonic sort of (key, position) pairs, ascending
    for (int size = 2; size <= kReorderTile; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int t = tid; t < kReorderTile / 2; t += kReorderThreads) {
          const int lo = 2 * t - (t & (stride - 1));
          const int hi = lo + stride;
          const bool up = (lo & size) == 0;
          const K a = s_key[lo], b = s_key[hi];
          if ((a > b) == up) {
            s_key[lo] = b;
            s_key[hi] = a;
            const uint32_t pa = s_pos[lo];
            s_pos[lo] = s_pos[hi];
            s_pos[hi] = pa;
          }
        }
        __syncthreads();
      }
    }
    // neighbouring lanes take neighbouring sorted probes
    for (int j = 0; j < kReorderItems; ++j) {
      const int p = j * kReorderThreads + tid;
      const uint32_t orig = s_pos[p];
      if (orig < cnt) s_res[orig] = lookup_one<K, KIND, KF>(keys, rows, n, levels, s_key[p]);
    }
    __syncthreads();
    for (int i = tid; i < (int)cnt; i += kReorderThreads) out[base + i] = s_res[i];
    __syncthreads();
  }
}

// Any k, one thread per lookup, pivots scanned in order.
template <class K>
__global__ void __launch_bounds__(512) k_eks_generic(const K* __restrict__ keys,
                                                     const uint32_t* __restrict__ rows,
                                                     uint64_t n, uint32_t k,
                                                     const K* __restrict__ q, uint64_t m,
                                                     uint32_t* __restrict__ out, int early_exit) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    const K x = q[i];
    uint64_t s = 0, cand = kNone;
    bool eqf = false;
    while (s < n) {
      uint32_t c = 0;
      bool eq = false;
      for (uint32_t j = 0; j + 1 < k && s + j < n; ++j) {
        const K v = keys[s + j];
        if (v < x) {
          ++c;
        } else {
          eq = v == x;
          break;
        }
      }
      if (c < k - 1 && s + c < n) {
        cand = s + c;
        eqf = eq;
        if (early_exit && eq) break;
      }
      s = s * k + (uint64_t)(c + 1) * (k - 1);
    }
    out[i] = eqf ? rows[cand] : GI_MISS;
  }
}

}  // namespace pt
}  // namespace gi
