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
//                (vector loads when a lane holds 8 or 16 contiguous bytes), the
//                group counts the pivots < x with ballots, and the next node
//                starts at s*k + (c+1)*(k-1).  G = 1 is "EKS (single)".
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
// P contiguous keys (8 bytes, or a multiple of 16 bytes) with vector loads.
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
  } else {
#pragma unroll
    for (int i = 0; i < BYTES / 16; ++i) {
      if constexpr (sizeof(K) == 4) {
        const uint4 t = __ldg((const uint4*)p + i);
        v[4 * i + 0] = t.x;
        v[4 * i + 1] = t.y;
        v[4 * i + 2] = t.z;
        v[4 * i + 3] = t.w;
      } else {
        const ulonglong2 t = __ldg((const ulonglong2*)p + i);
        v[2 * i + 0] = t.x;
        v[2 * i + 1] = t.y;
      }
    }
  }
}

template <class K, int KF, int G>
struct EksShape {
  static constexpr int N = KF - 1;                 // pivots per node
  static constexpr int P = (N + G - 1) / G;        // pivots per lane
  // contiguous vector per lane when the node splits evenly into 8/16/32/64-byte pieces
  static constexpr bool VEC = (N % G == 0) && (P >= 2) && (P * sizeof(K) >= 8) &&
                              (P * sizeof(K) <= 64) && ((P & (P - 1)) == 0);
};

template <class K, int KF, int G, int R>
__global__ void __launch_bounds__(512) k_eks_point(const K* __restrict__ keys,
                                                   const uint32_t* __restrict__ rows, uint64_t n,
                                                   uint32_t levels, const K* __restrict__ q,
                                                   uint64_t m, uint32_t* __restrict__ out,
                                                   uint32_t smem_slots, int early_exit,
                                                   uint32_t* flags) {
  using S = EksShape<K, KF, G>;
  constexpr int N = S::N, P = S::P;
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

  for (uint64_t first = gid; first < m; first += groups * R) {
    K x[R];
    uint64_t s[R], cand[R];
    bool act[R], eqf[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const uint64_t i = first + r * groups;
      act[r] = i < m && n > 0;
      x[r] = i < m ? q[i] : K(0);
      s[r] = 0;
      cand[r] = kNone;
      eqf[r] = false;
    }
    for (uint32_t lv = 0; lv < levels; ++lv) {
      K piv[R][P];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (act[r]) {
          if (S::VEC) {
            const uint64_t at = s[r] + (uint64_t)gl * P;
            if (s[r] < smem_slots) {
#pragma unroll
              for (int p = 0; p < P; ++p) piv[r][p] = sm[at + p];
            } else {
              vec_load<K, P>(keys + at, piv[r]);
            }
          } else {
#pragma unroll
            for (int p = 0; p < P; ++p) {
              const uint64_t at = s[r] + gl + (uint64_t)p * G;
              const bool ok = (gl + p * G < N) && at < n;
              piv[r][p] = ok ? (s[r] < smem_slots ? sm[at] : ldg(keys + at)) : K(0);
            }
          }
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (act[r]) {
          uint32_t c = 0;
          bool any_eq = false;
#pragma unroll
          for (int p = 0; p < P; ++p) {
            const int j = S::VEC ? gl * P + p : gl + p * G;  // position in the node
            const bool ok = j < N && s[r] + j < n;
            const bool lt = ok && piv[r][p] < x[r];
            any_eq |= ok && piv[r][p] == x[r];
            c += __popc(__ballot_sync(gmask, lt) & gmask);
          }
          any_eq = __any_sync(gmask, any_eq);
          if (c < (uint32_t)N && s[r] + c < n) {
            cand[r] = s[r] + c;
            eqf[r] = any_eq;
          }
          if (early_exit && any_eq) {
            act[r] = false;
          } else {
            s[r] = s[r] * KF + (uint64_t)(c + 1) * N;
            if (s[r] >= n) act[r] = false;
          }
        }
      }
    }
    if (gl == 0) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const uint64_t i = first + r * groups;
        if (i < m) out[i] = eqf[r] ? ldg(rows + cand[r]) : GI_MISS;
      }
    }
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
