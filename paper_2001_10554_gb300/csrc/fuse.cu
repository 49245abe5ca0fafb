// Queued low-qubit gates (iqs_set_fusion): the one-qubit gates queued on the
// qubits of one shared-memory tile (bits 0..11 for complex64, 0..10 for
// complex128) are applied in ONE pass over the state instead of one pass per
// gate.  The gates queued on a qubit are multiplied in FP64 on the host; this
// pass applies the per-qubit products in register rounds of a 2^K-amplitude
// tile (the pool engine's tile code: FP32 for complex64, double-float for
// complex128), so each amplitude is read and written once.
#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "pool_common.cuh"

namespace iqs {
namespace {

struct FusedMats {
  double u[16][8];  // the matrices of qubits lb0 .. lb0 + ng - 1 (identity where nothing is queued)
};

template <class TR>
__global__ void __launch_bounds__(kThreads) k_fused(typename TR::V* __restrict__ a, uint64_t tiles, int K, int lb0,
                                                    int ng, const FusedMats f, unsigned* __restrict__ flag) {
  using W = typename TR::W;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  W* sp = reinterpret_cast<W*>(smem_raw);
  __shared__ typename TR::Mat mats[16];
  if ((int)threadIdx.x < ng) {
    pool::M2 m;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      m.r[e] = f.u[threadIdx.x][2 * e];
      m.i[e] = f.u[threadIdx.x][2 * e + 1];
    }
    mats[threadIdx.x] = TR::make(m);
  }
  __syncthreads();
  const Geo g{0, 0, K};
  unsigned bad = 0;
  for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) pool::pool_tile<TR>(sp, mats, a, g, t, lb0, ng, 0u, bad);
  if (bad) atomicOr(flag, 1u);
}

}  // namespace

int fuse_bits(const iqs_reg* r) {
  const int K = r->dtype == IQS_C128 ? pool::P128::kTileBits : pool::P64::kTileBits;
  return std::min(K, r->n);
}

cudaError_t launch_fused(iqs_reg* r) {
  if (r->fmask == 0) return cudaSuccess;
  const int K = fuse_bits(r);
  const int lb0 = __builtin_ctz(r->fmask), hi = 31 - __builtin_clz(r->fmask);
  FusedMats f;
  for (int q = lb0; q <= hi; ++q)
    for (int k = 0; k < 8; ++k)
      f.u[q - lb0][k] = (r->fmask >> q) & 1u ? r->fmat[q][k] : (k == 0 || k == 6 ? 1.0 : 0.0);
  const uint64_t tiles = num_amps(r) >> K;
  const unsigned grid = (unsigned)std::min<uint64_t>(tiles, (uint64_t)kSMs * 8);
  if (r->dtype == IQS_C128) {
    const size_t smem = sizeof(pool::P128::W) << K;
    k_fused<pool::P128><<<grid, kThreads, smem, r->stream>>>((double2*)r->data, tiles, K, lb0, hi - lb0 + 1, f, r->flag);
  } else {
    const size_t smem = sizeof(pool::P64::W) << K;
    k_fused<pool::P64><<<grid, kThreads, smem, r->stream>>>((float2*)r->data, tiles, K, lb0, hi - lb0 + 1, f, r->flag);
  }
  return launched(1);
}

}  // namespace iqs
