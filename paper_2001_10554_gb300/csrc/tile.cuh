// Shared-memory tiles of a state vector (used by the QAOA mixer and the pool
// engine): tile geometry, XOR swizzle, and a one-value block reduction.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace iqs {

// Tile bits: [0, c) and [s, s + m), s >= c.  Local index l = (h << c) | low.
struct Geo {
  int c, s, m;
};

__device__ __forceinline__ uint64_t tile_x(const Geo& g, uint64_t t, unsigned l) {
  const uint64_t low = l & ((1u << g.c) - 1u);
  const uint64_t h = l >> g.c;
  const int mid = g.s - g.c;
  const uint64_t tlo = t & ((1ull << mid) - 1ull);
  const uint64_t thi = t >> mid;
  return (thi << (g.s + g.m)) | (h << g.s) | (tlo << g.c) | low;
}

// ---------------------------------------------------------------- block reduction of one FP64 value
__device__ __forceinline__ void block_partial(double v, double* out) {
  __shared__ double red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    *out = s;
  }
  __syncthreads();
}

// Shared-memory index of tile element l: XOR-swizzled within 128-byte rows so
// that a warp reading a fixed offset of 32 consecutive register blocks (rows
// of stride 2^kSwzBits elements) hits distinct banks.  A traits type may
// instead define kTmaSwizzle to use the layout of the TMA 128-byte swizzle
// (16-byte chunk index XOR row index mod 8), so tiles written by TMA can be
// indexed directly.  Both are linear over GF(2): swz(a ^ b) = swz(a) ^ swz(b).
template <class TR>
__device__ __forceinline__ unsigned swz(unsigned l) {
  if constexpr (TR::kTmaSwizzle) {
    if constexpr (sizeof(typename TR::V) == 8) return l ^ (((l >> 4) & 7u) << 1);  // 8-byte elements
    else return l ^ ((l >> 3) & 7u);                                             // 16-byte elements
  } else {
    return l ^ ((l >> TR::kSwzBits) & ((1u << TR::kSwzBits) - 1u));
  }
}

}  // namespace iqs
