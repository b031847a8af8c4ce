// Memory-system probes used as roofline denominators (Section 5.1).
//
//   k_random_chunks   : independent loads of `chunk` contiguous bytes from
//                       uniformly random chunk-aligned offsets of a buffer much
//                       larger than L2; groups of chunk/16 lanes each load 16 B,
//                       8 loads in flight per lane.  Measures random-sector HBM
//                       throughput, the bound of an index lookup beyond L2.
//   k_coalescing      : the micro-benchmark of Section 5.1 / Fig 9: groups of
//                       2^m neighbouring threads, each step a random position p
//                       per group, thread i of the group loads entry p+i.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gi_internal.cuh"

namespace gi {
namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t z) {  // splitmix64 finaliser
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

constexpr int kInFlight = 8;

__global__ void __launch_bounds__(256) k_random_chunks(const uint4* __restrict__ buf,
                                                       uint64_t chunks, uint32_t lanes,
                                                       uint64_t iters, uint64_t loads,
                                                       uint64_t seed, unsigned long long* sink) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t group = tid / lanes;
  const uint64_t groups = ((uint64_t)gridDim.x * blockDim.x) / lanes;
  const uint32_t gl = (uint32_t)(tid % lanes);
  uint32_t acc = 0;
  for (uint64_t it = 0; it < iters; it += kInFlight) {
    uint4 v[kInFlight];
#pragma unroll
    for (int u = 0; u < kInFlight; ++u) {
      const uint64_t h = mix64(seed ^ mix64(group * 0x100000001B3ull + it + u));
      const uint64_t c = __umul64hi(h, chunks);
      // load number group + (it+u)*groups; exactly `loads` loads in total
      v[u] = (group + (it + u) * groups < loads) ? __ldg(buf + c * lanes + gl)
                                                 : make_uint4(0, 0, 0, 0);
    }
#pragma unroll
    for (int u = 0; u < kInFlight; ++u) acc ^= v[u].x ^ v[u].y ^ v[u].z ^ v[u].w;
  }
  if (acc == 0x9E3779B9u) atomicXor(sink, (unsigned long long)acc);  // keeps the loads alive
}

__global__ void __launch_bounds__(256) k_coalescing(const uint32_t* __restrict__ buf,
                                                    uint64_t entries, uint32_t threads,
                                                    uint32_t group, uint32_t steps, uint64_t seed,
                                                    unsigned long long* sink) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= threads) return;
  const uint32_t g = tid / group, gl = tid % group;
  const uint64_t span = entries - group + 1;
  uint32_t acc = 0;
  for (uint32_t st = 0; st < steps; ++st) {
    const uint64_t p = __umul64hi(mix64(seed ^ mix64(((uint64_t)g << 20) + st)), span);
    acc ^= __ldg(buf + p + gl);
  }
  if (acc == 0x9E3779B9u) atomicXor(sink, (unsigned long long)acc);
}

}  // namespace

cudaError_t probe_random_sectors(const void* buf, uint64_t bytes, uint32_t chunk_bytes,
                                 uint64_t loads, uint64_t seed, uint64_t* sink,
                                 cudaStream_t s) {
  const uint32_t lanes = chunk_bytes / 16;
  const uint64_t chunks = bytes / chunk_bytes;
  if (chunks == 0 || loads == 0) return cudaSuccess;
  const int block = 256;
  const uint64_t threads = (uint64_t)sm_count() * 2048;  // a full GPU of resident threads
  const uint64_t groups = threads / lanes;
  const uint64_t iters = (loads + groups - 1) / groups;
  k_random_chunks<<<(unsigned)(threads / block), block, 0, s>>>(
      (const uint4*)buf, chunks, lanes, iters, loads, seed, (unsigned long long*)sink);
  count_launch();
  return cudaGetLastError();
}

cudaError_t coalescing_probe(const uint32_t* buf, uint64_t entries, uint32_t threads,
                             uint32_t group, uint32_t steps, uint64_t seed, uint64_t* sink,
                             cudaStream_t s) {
  const int block = 256;
  k_coalescing<<<(threads + block - 1) / block, block, 0, s>>>(buf, entries, threads, group,
                                                               steps, seed,
                                                               (unsigned long long*)sink);
  count_launch();
  return cudaGetLastError();
}

}  // namespace gi
