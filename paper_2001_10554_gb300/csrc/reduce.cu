// Reductions over the state: squared norm, GetProbability(q) (Section 2,
// "Scope and basic use"), P(q=1) for every qubit in one read, expectation of a
// Pauli product, and the Max-Cut energy <C> (Section 4).
//
// Accumulation is FP64-equivalent for both dtypes without using the slow
// FP64 pipe in the loop: every product is formed error-free in FP32 (FMA
// residuals; complex128 inputs are first split into float pairs) and summed
// into double-float accumulators with TwoSum.  Once per thread the
// accumulators become doubles; warps, blocks and finally the grid (a fixed
// number of blocks, summed in a fixed order by one block) reduce in FP64, so
// every result is deterministic run to run.
#include <cmath>

#include "common.cuh"
#include "cut.cuh"
#include "df64.cuh"
#include "internal.h"

namespace iqs {
namespace {

constexpr int kWarps = kThreads / 32;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum v[0..S) over the block; thread 0..S-1 writes partials[blockIdx.x * stride + j].
template <int S>
__device__ __forceinline__ void block_store(double (&v)[S], int count, double* __restrict__ partials, int stride) {
  __shared__ double sm[kWarps][S];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < S; ++j) {
    const double s = warp_sum(v[j]);
    if (lane == 0) sm[warp][j] = s;
  }
  __syncthreads();
  if (threadIdx.x < count) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) s += sm[w][threadIdx.x];
    partials[(uint64_t)blockIdx.x * stride + threadIdx.x] = s;
  }
}

// One block: results[j] = sum over blocks of partials[b * stride + j], fixed order.
__global__ void k_finalize(const double* __restrict__ partials, int nblocks, int count, int stride,
                           double* __restrict__ results) {
  __shared__ double sm[kWarps];
  for (int j = 0; j < count; ++j) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partials[(uint64_t)b * stride + j];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < kWarps; ++w) t += sm[w];
      results[j] = t;
    }
    __syncthreads();
  }
}

// |a|^2 as an unevaluated pair, per dtype.
__device__ __forceinline__ void abs2(float2 a, float& p, float& e, unsigned&) { dfx::abs2_c64(a.x, a.y, p, e); }
__device__ __forceinline__ void abs2(double2 a, float& p, float& e, unsigned& bad) {
  dfx::abs2_c128(a.x, a.y, p, e, bad);
}

// ---------------------------------------------------------------- norm
template <class V>
__global__ void __launch_bounds__(kThreads) k_norm2(const V* __restrict__ a, uint64_t n, double* partials,
                                                     unsigned* flag) {
  dfx::Acc acc;
  unsigned bad = 0;
  // four loads in flight per thread; the sums keep the one-at-a-time order
  const uint64_t S = (uint64_t)gridDim.x * blockDim.x;
  uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  for (; i + 3 * S < n; i += 4 * S) {
    const V v[4] = {a[i], a[i + S], a[i + 2 * S], a[i + 3 * S]};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      float p, e;
      abs2(v[u], p, e, bad);
      acc.add(p, e);
    }
  }
  for (; i < n; i += S) {
    float p, e;
    abs2(a[i], p, e, bad);
    acc.add(p, e);
  }
  if (bad) atomicOr(flag, 1u);
  double v[1] = {acc.value()};
  block_store<1>(v, 1, partials, 1);
}

// complex64: two amplitudes per 16-byte load
__global__ void __launch_bounds__(kThreads) k_norm2_c64v(const float4* __restrict__ a, uint64_t n2, double* partials) {
  dfx::Acc acc;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n2; i += (uint64_t)gridDim.x * blockDim.x) {
    const float4 v = a[i];
    float p, e;
    dfx::abs2_c64(v.x, v.y, p, e);
    acc.add(p, e);
    dfx::abs2_c64(v.z, v.w, p, e);
    acc.add(p, e);
  }
  double v[1] = {acc.value()};
  block_store<1>(v, 1, partials, 1);
}

// ---------------------------------------------------------------- probability of one qubit
template <class V>
__global__ void __launch_bounds__(kThreads) k_prob(const V* __restrict__ a, uint64_t n_half, int q, double* partials,
                                                    unsigned* flag) {
  dfx::Acc acc;
  unsigned bad = 0;
  const uint64_t bit = 1ull << q;
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < n_half; k += (uint64_t)gridDim.x * blockDim.x) {
    float p, e;
    abs2(a[insert_zero(k, q) | bit], p, e, bad);
    acc.add(p, e);
  }
  if (bad) atomicOr(flag, 1u);
  double v[1] = {acc.value()};
  block_store<1>(v, 1, partials, 1);
}

// complex64, q >= 1: two consecutive amplitudes with bit q set per float4.
__global__ void __launch_bounds__(kThreads) k_prob_c64v(const float2* __restrict__ a, uint64_t n_half2, int q,
                                                         double* partials) {
  dfx::Acc acc;
  const uint64_t bit = 1ull << q;
  for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < n_half2; j += (uint64_t)gridDim.x * blockDim.x) {
    const float4 v = *reinterpret_cast<const float4*>(a + (insert_zero(2 * j, q) | bit));
    float p, e;
    dfx::abs2_c64(v.x, v.y, p, e);
    acc.add(p, e);
    dfx::abs2_c64(v.z, v.w, p, e);
    acc.add(p, e);
  }
  double v[1] = {acc.value()};
  block_store<1>(v, 1, partials, 1);
}

// ---------------------------------------------------------------- probability of every qubit
// df + df
__device__ __forceinline__ dfx::Acc dfadd(const dfx::Acc& a, const dfx::Acc& b) {
  dfx::Acc r;
  float t;
  dfx::two_sum(a.h, b.h, r.h, t);
  r.l = a.l + b.l + t;
  return r;
}

__device__ __forceinline__ void acc_add(dfx::Acc& a, const dfx::Acc& b) { a.add(b.h, b.l); }

// n >= 9.  A task is 512 consecutive amplitudes handled by one warp: lane l
// reads amplitudes base + 32 j + l, j = 0..15.  Bits 0..4 of the index are the
// lane, bits 5..8 are j, bits 9.. are the task number.  Per lane the 16
// weights are summed by a binary tree whose right children also feed the
// per-bit sums of bits 5..8; the task total is reduced over the warp and added
// by lane l to the sum of qubit 9 + l when that bit of the task number is set.
template <class V>
__global__ void __launch_bounds__(kThreads) k_probs_all(const V* __restrict__ a, int n, double* partials,
                                                         unsigned* flag) {
  const int lane = threadIdx.x & 31;
  const uint64_t n_tasks = (1ull << n) >> 9;
  const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  dfx::Acc accL, accS[4], accH;
  unsigned bad = 0;
  for (uint64_t task = warp0; task < n_tasks; task += n_warps) {
    const V* base = a + (task << 9) + lane;
    dfx::Acc w[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      float p, e;
      abs2(base[32 * j], p, e, bad);
      w[j].h = p;
      w[j].l = e;
    }
    dfx::Acc pr[8], qd[4], oc[2];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      pr[i] = dfadd(w[2 * i], w[2 * i + 1]);
      acc_add(accS[0], w[2 * i + 1]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      qd[i] = dfadd(pr[2 * i], pr[2 * i + 1]);
      acc_add(accS[1], pr[2 * i + 1]);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      oc[i] = dfadd(qd[2 * i], qd[2 * i + 1]);
      acc_add(accS[2], qd[2 * i + 1]);
    }
    const dfx::Acc W = dfadd(oc[0], oc[1]);
    acc_add(accS[3], oc[1]);
    acc_add(accL, W);
    // warp total of this task
    dfx::Acc T = W;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      dfx::Acc other;
      other.h = __shfl_xor_sync(0xffffffffu, T.h, o);
      other.l = __shfl_xor_sync(0xffffffffu, T.l, o);
      T = dfadd(T, other);
    }
    if (lane < n - 9 && ((task >> lane) & 1)) acc_add(accH, T);
  }
  if (bad) atomicOr(flag, 1u);
  const double L = accL.value(), H = accH.value();
  double v[kRedSlots - 4];
#pragma unroll
  for (int q = 0; q < kRedSlots - 4; ++q) {
    double c = 0.0;
    if (q < 5) c = ((lane >> q) & 1) ? L : 0.0;
    else if (q < 9) c = accS[q - 5].value();
    else c = (lane == q - 9) ? H : 0.0;
    v[q] = c;
  }
  block_store<kRedSlots - 4>(v, n, partials, kRedSlots);
}

// n < 9: one accumulator per qubit per thread.
template <class V>
__global__ void __launch_bounds__(kThreads) k_probs_small(const V* __restrict__ a, int n, double* partials,
                                                           unsigned* flag) {
  dfx::Acc acc[8];
  unsigned bad = 0;
  const uint64_t N = 1ull << n;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x) {
    float p, e;
    abs2(a[i], p, e, bad);
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (q < n && ((i >> q) & 1)) acc[q].add(p, e);
  }
  if (bad) atomicOr(flag, 1u);
  double v[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = acc[q].value();
  block_store<8>(v, n, partials, kRedSlots);
}

// ---------------------------------------------------------------- Pauli expectation
// Unevaluated pair for a*b + s*c*d with s = +-1 (error-free products, TwoSum).
__device__ __forceinline__ void dot2_f32(float a, float b, float c, float d, float& p, float& e) {
  const float p1 = a * b, e1 = fmaf(a, b, -p1);
  const float p2 = c * d, e2 = fmaf(c, d, -p2);
  float t;
  dfx::two_sum(p1, p2, p, t);
  e = e1 + e2 + t;
}

// Product of two split doubles (xh + xl 2^-52)(yh + yl 2^-52) as an unevaluated pair.
__device__ __forceinline__ void mul_df(float xh, float xl, float yh, float yl, float& p, float& e) {
  p = xh * yh;
  e = fmaf(xh, yh, -p);
  e = fmaf(xh * 0x1p-52f, yl, e);
  e = fmaf(yh * 0x1p-52f, xl, e);
}

// z = conj(psi_y) psi_x: Re z = yr xr + yi xi, Im z = yr xi - yi xr.  ``imag``
// selects the component.  Complex64 version.
__device__ __forceinline__ void zterm(float2 x, float2 y, bool imag, float& p, float& e, unsigned&) {
  if (!imag) dot2_f32(y.x, x.x, y.y, x.y, p, e);
  else dot2_f32(y.x, x.y, -y.y, x.x, p, e);
}
__device__ __forceinline__ void zterm(double2 x, double2 y, bool imag, float& p, float& e, unsigned& bad) {
  float xrh, xrl, xih, xil, yrh, yrl, yih, yil;
  dfx::split(x.x, xrh, xrl, bad);
  dfx::split(x.y, xih, xil, bad);
  dfx::split(y.x, yrh, yrl, bad);
  dfx::split(y.y, yih, yil, bad);
  float p1, e1, p2, e2;
  if (!imag) {
    mul_df(yrh, yrl, xrh, xrl, p1, e1);
    mul_df(yih, yil, xih, xil, p2, e2);
  } else {
    mul_df(yrh, yrl, xih, xil, p1, e1);
    mul_df(yih, yil, xrh, xrl, p2, e2);
    p2 = -p2;
    e2 = -e2;
  }
  float t;
  dfx::two_sum(p1, p2, p, t);
  e = e1 + e2 + t;
}

// X-free strings: sum_x (-1)^popc(x & zm) |psi_x|^2.
template <class V>
__global__ void __launch_bounds__(kThreads) k_expect_diag(const V* __restrict__ a, uint64_t n, uint64_t zm,
                                                           double* partials, unsigned* flag) {
  dfx::Acc acc;
  unsigned bad = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    float p, e;
    abs2(a[i], p, e, bad);
    if (__popcll(i & zm) & 1) {
      p = -p;
      e = -e;
    }
    acc.add(p, e);
  }
  if (bad) atomicOr(flag, 1u);
  double v[1] = {acc.value()};
  block_store<1>(v, 1, partials, 1);
}

// Strings with X or Y: each unordered pair {x, y = x ^ xm} (bit h of x clear,
// h the highest bit of xm) contributes s(x) * (Re z or Im z) times a constant
// applied on the host; s(x) = (-1)^popc(x & zm).
template <class V>
__global__ void __launch_bounds__(kThreads) k_expect_pair(const V* __restrict__ a, uint64_t n_half, int h, uint64_t xm,
                                                           uint64_t zm, int imag, double* partials, unsigned* flag) {
  dfx::Acc acc;
  unsigned bad = 0;
  // two pairs (four loads) in flight per thread; the sums keep the
  // one-at-a-time order
  const uint64_t S = (uint64_t)gridDim.x * blockDim.x;
  uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  auto term = [&](uint64_t x, const V& ax, const V& ay) {
    float p, e;
    zterm(ax, ay, imag != 0, p, e, bad);
    if (__popcll(x & zm) & 1) {
      p = -p;
      e = -e;
    }
    acc.add(p, e);
  };
  for (; k + S < n_half; k += 2 * S) {
    const uint64_t x0 = insert_zero(k, h), x1 = insert_zero(k + S, h);
    const V a0 = a[x0], b0 = a[x0 ^ xm], a1 = a[x1], b1 = a[x1 ^ xm];
    term(x0, a0, b0);
    term(x1, a1, b1);
  }
  for (; k < n_half; k += S) {
    const uint64_t x = insert_zero(k, h);
    term(x, a[x], a[x ^ xm]);
  }
  if (bad) atomicOr(flag, 1u);
  double v[1] = {acc.value()};
  block_store<1>(v, 1, partials, 1);
}

// ---------------------------------------------------------------- Max-Cut energy
template <class V, class X>
__global__ void __launch_bounds__(kThreads) k_energy(const V* __restrict__ a, uint64_t n, EdgesU8 E, double* partials,
                                                      unsigned* flag) {
  dfx::Acc acc;
  unsigned bad = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const float c = (float)cut_count((X)i, E);
    float p, e;
    abs2(a[i], p, e, bad);
    const float q = c * p;
    acc.add(q, fmaf(c, p, -q) + c * e);
  }
  if (bad) atomicOr(flag, 1u);
  double v[1] = {acc.value()};
  block_store<1>(v, 1, partials, 1);
}

struct WeightsDF {
  float h[kEdgeChunk + 1], l[kEdgeChunk + 1];
};

template <class V, class X>
__global__ void __launch_bounds__(kThreads) k_energy_w(const V* __restrict__ a, uint64_t n, EdgesU8 E, WeightsDF W,
                                                        double* partials, unsigned* flag) {
  dfx::Acc acc;
  unsigned bad = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const X x = (X)i;
    dfx::Acc c;
    for (int k = 0; k < E.m; ++k)
      if (((x >> E.u[k]) ^ (x >> E.v[k])) & 1) c.add(W.h[k], W.l[k]);
    float p, e;
    abs2(a[i], p, e, bad);
    const float q = c.h * p;
    acc.add(q, fmaf(c.h, p, -q) + c.h * e + c.l * p);
  }
  if (bad) atomicOr(flag, 1u);
  double v[1] = {acc.value()};
  block_store<1>(v, 1, partials, 1);
}

cudaError_t finalize(iqs_reg* r, int count, int stride) {
  k_finalize<<<1, kThreads, 0, r->stream>>>(r->partials, kRedBlocks, count, stride, r->results);
  return launched(1);
}

}  // namespace

cudaError_t launch_norm2(iqs_reg* r) {
  const uint64_t N = num_amps(r);
  if (r->dtype == IQS_C64)
    k_norm2_c64v<<<kRedBlocks, kThreads, 0, r->stream>>>((const float4*)r->data, N / 2, r->partials);
  else
    k_norm2<double2><<<kRedBlocks, kThreads, 0, r->stream>>>((const double2*)r->data, N, r->partials, r->flag);
  cudaError_t e = launched(1);
  return e != cudaSuccess ? e : finalize(r, 1, 1);
}

cudaError_t launch_probability(iqs_reg* r, int q) {
  const uint64_t half = num_amps(r) >> 1;
  if (r->dtype == IQS_C64) {
    if (q >= 1)
      k_prob_c64v<<<kRedBlocks, kThreads, 0, r->stream>>>((const float2*)r->data, half / 2, q, r->partials);
    else
      k_prob<float2><<<kRedBlocks, kThreads, 0, r->stream>>>((const float2*)r->data, half, q, r->partials, r->flag);
  } else {
    k_prob<double2><<<kRedBlocks, kThreads, 0, r->stream>>>((const double2*)r->data, half, q, r->partials, r->flag);
  }
  cudaError_t e = launched(1);
  return e != cudaSuccess ? e : finalize(r, 1, 1);
}

cudaError_t launch_probabilities(iqs_reg* r) {
  if (r->n >= 9) {
    if (r->dtype == IQS_C64)
      k_probs_all<float2><<<kRedBlocks, kThreads, 0, r->stream>>>((const float2*)r->data, r->n, r->partials, r->flag);
    else
      k_probs_all<double2><<<kRedBlocks, kThreads, 0, r->stream>>>((const double2*)r->data, r->n, r->partials, r->flag);
  } else {
    if (r->dtype == IQS_C64)
      k_probs_small<float2><<<kRedBlocks, kThreads, 0, r->stream>>>((const float2*)r->data, r->n, r->partials, r->flag);
    else
      k_probs_small<double2><<<kRedBlocks, kThreads, 0, r->stream>>>((const double2*)r->data, r->n, r->partials,
                                                                      r->flag);
  }
  cudaError_t e = launched(1);
  return e != cudaSuccess ? e : finalize(r, r->n, kRedSlots);
}

// All-qubit probabilities with caller-supplied scratch: ``partials`` holds
// kRedBlocks x kRedSlots doubles, ``results`` receives n doubles (device).
cudaError_t launch_probabilities_raw(const void* data, int n, int dtype, cudaStream_t s, double* partials,
                                     double* results, unsigned* flag) {
  if (n >= 9) {
    if (dtype == IQS_C64)
      k_probs_all<float2><<<kRedBlocks, kThreads, 0, s>>>((const float2*)data, n, partials, flag);
    else
      k_probs_all<double2><<<kRedBlocks, kThreads, 0, s>>>((const double2*)data, n, partials, flag);
  } else {
    if (dtype == IQS_C64)
      k_probs_small<float2><<<kRedBlocks, kThreads, 0, s>>>((const float2*)data, n, partials, flag);
    else
      k_probs_small<double2><<<kRedBlocks, kThreads, 0, s>>>((const double2*)data, n, partials, flag);
  }
  cudaError_t e = launched(1);
  if (e != cudaSuccess) return e;
  k_finalize<<<1, kThreads, 0, s>>>(partials, kRedBlocks, n, kRedSlots, results);
  return launched(1);
}

cudaError_t launch_expectation(iqs_reg* r, uint64_t xm, uint64_t zm) {
  const uint64_t N = num_amps(r);
  if (xm == 0) {
    if (r->dtype == IQS_C64)
      k_expect_diag<float2><<<kRedBlocks, kThreads, 0, r->stream>>>((const float2*)r->data, N, zm, r->partials, r->flag);
    else
      k_expect_diag<double2><<<kRedBlocks, kThreads, 0, r->stream>>>((const double2*)r->data, N, zm, r->partials,
                                                                      r->flag);
  } else {
    const int h = 63 - __builtin_clzll(xm);
    const int nY = __builtin_popcountll(xm & zm);
    const int imag = nY & 1;
    if (r->dtype == IQS_C64)
      k_expect_pair<float2><<<kRedBlocks, kThreads, 0, r->stream>>>((const float2*)r->data, N / 2, h, xm, zm, imag,
                                                                     r->partials, r->flag);
    else
      k_expect_pair<double2><<<kRedBlocks, kThreads, 0, r->stream>>>((const double2*)r->data, N / 2, h, xm, zm, imag,
                                                                      r->partials, r->flag);
  }
  cudaError_t e = launched(1);
  return e != cudaSuccess ? e : finalize(r, 1, 1);
}

cudaError_t launch_energy(iqs_reg* r, int n_edges, const int32_t* edges, const double* w) {
  // Handles one chunk of at most kEdgeChunk edges; the caller loops.
  EdgesU8 E;
  E.m = n_edges;
  for (int e = 0; e < n_edges; ++e) {
    E.u[e] = (uint8_t)edges[2 * e];
    E.v[e] = (uint8_t)edges[2 * e + 1];
  }
  const uint64_t N = num_amps(r);
  const bool narrow = r->n <= 32;
  if (w == nullptr) {
    if (r->dtype == IQS_C64) {
      if (narrow) k_energy<float2, uint32_t><<<kRedBlocks, kThreads, 0, r->stream>>>((const float2*)r->data, N, E, r->partials, r->flag);
      else k_energy<float2, uint64_t><<<kRedBlocks, kThreads, 0, r->stream>>>((const float2*)r->data, N, E, r->partials, r->flag);
    } else {
      if (narrow) k_energy<double2, uint32_t><<<kRedBlocks, kThreads, 0, r->stream>>>((const double2*)r->data, N, E, r->partials, r->flag);
      else k_energy<double2, uint64_t><<<kRedBlocks, kThreads, 0, r->stream>>>((const double2*)r->data, N, E, r->partials, r->flag);
    }
  } else {
    WeightsDF W;
    for (int e = 0; e < n_edges; ++e) {
      W.h[e] = (float)w[e];
      W.l[e] = (float)(w[e] - (double)W.h[e]);
    }
    if (r->dtype == IQS_C64) {
      if (narrow) k_energy_w<float2, uint32_t><<<kRedBlocks, kThreads, 0, r->stream>>>((const float2*)r->data, N, E, W, r->partials, r->flag);
      else k_energy_w<float2, uint64_t><<<kRedBlocks, kThreads, 0, r->stream>>>((const float2*)r->data, N, E, W, r->partials, r->flag);
    } else {
      if (narrow) k_energy_w<double2, uint32_t><<<kRedBlocks, kThreads, 0, r->stream>>>((const double2*)r->data, N, E, W, r->partials, r->flag);
      else k_energy_w<double2, uint64_t><<<kRedBlocks, kThreads, 0, r->stream>>>((const double2*)r->data, N, E, W, r->partials, r->flag);
    }
  }
  cudaError_t e = launched(1);
  return e != cudaSuccess ? e : finalize(r, 1, 1);
}

}  // namespace iqs
