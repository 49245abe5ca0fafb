// Shared device helpers: index insertion, launch sizing, complex helpers.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace iqs {

constexpr int kThreads = 256;   // threads per block for streaming kernels
constexpr int kSMs = 152;       // GB300 SM count (grids are multiples of it)

// Index of the k-th element of the set {i : bit b of i is 0}: insert a zero
// bit at position b.  This is the pair enumeration of the one-qubit gate
// equation (Section 2): pair k is (insert_zero(k, q), insert_zero(k, q) | 2^q).
__host__ __device__ __forceinline__ uint64_t insert_zero(uint64_t k, int b) {
  const uint64_t low = k & ((1ull << b) - 1ull);
  return ((k >> b) << (b + 1)) | low;
}

// Two zero bits at positions lo < hi (controlled gates: control and target).
__host__ __device__ __forceinline__ uint64_t insert_two_zeros(uint64_t k, int lo, int hi) {
  return insert_zero(insert_zero(k, lo), hi);
}

// Blocks for a grid-stride kernel over ``work`` items of ``per_thread`` each:
// enough to cover the work, capped at ``max_per_sm`` blocks per SM.
inline unsigned grid_for(uint64_t work, int per_thread, int max_per_sm) {
  const uint64_t threads = (work + per_thread - 1) / per_thread;
  uint64_t blocks = (threads + kThreads - 1) / kThreads;
  const uint64_t cap = (uint64_t)kSMs * (uint64_t)max_per_sm;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return (unsigned)blocks;
}

// Multiply by i^k exactly (k in 0..3): a permutation of components with sign flips.
template <class V>
__device__ __forceinline__ V mul_ipow(V v, int k) {
  V r = v;
  if (k == 1) { r.x = -v.y; r.y = v.x; }
  else if (k == 2) { r.x = -v.x; r.y = -v.y; }
  else if (k == 3) { r.x = v.y; r.y = -v.x; }
  return r;
}

}  // namespace iqs
