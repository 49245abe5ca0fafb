// Dense k-qubit gates (Section 2, "Scope and basic use": custom multi-qubit
// gates): a 2^k x 2^k matrix U acts on the amplitudes that differ only in the
// k target bits; bit j of U's row/column index is the value of qubits[j].
//
// One thread owns one group of 2^k amplitudes (the other n - k bits fixed):
// it loads the group into registers, forms every output as a dot product with
// a row of U and stores it.  For small k the loops are unrolled completely, so
// every coefficient is a compile-time offset into the kernel's parameter block
// and enters the FMAs as a constant-bank operand.  Where full unrolling would
// make the loop body larger than the instruction cache (complex64 k >= 4,
// double-float k >= 3, native k >= 4), the row loop stays rolled and the
// coefficients are staged once per block in shared memory (all lanes read
// the same address, so the reads broadcast).  complex64 computes in FP32
// (k <= 5); complex128 in the double-float emulation (k <= 4; for k >= 2 on
// paired .f32x2 instructions, two groups per thread) or, by default for
// k = 3..5, as exact digit products on the tensor cores (kgate_tc.cu), or,
// for small states or on request, in native FP64.  One read and one write
// of the state per gate.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "df64.cuh"
#include "f32x2.cuh"
#include "internal.h"

namespace iqs {
namespace {

constexpr int kMaxK64 = 5, kMaxK128 = 5;

// Target positions ascending (zero insertion) and, per element c of a group,
// the index offset sum_j bit_j(c) << qubits[j].
template <int K>
struct Targets {
  int pos[K];
  uint64_t off[1 << K];
};

// Blocks per SM the register budget is sized for (argument: the group's
// register cost in units of 2^K float2 values).  Each thread already keeps
// 2^K amplitudes in flight, so two or four resident blocks hide HBM latency.
template <int L>
constexpr int min_blocks() { return L >= 5 ? 1 : L == 4 ? 2 : 4; }

template <int K>
__device__ __forceinline__ uint64_t group_base(uint64_t g, const Targets<K>& T) {
  uint64_t x = g;
#pragma unroll
  for (int j = 0; j < K; ++j) x = insert_zero(x, T.pos[j]);
  return x;
}

template <int K>
struct UF32 {
  float2 u[1 << (2 * K)];  // row-major
};

template <int K>
__global__ void __launch_bounds__(kThreads, min_blocks<K>()) k_kgate_c64(float2* __restrict__ a, uint64_t n_groups, Targets<K> T,
                                                        UF32<K> U) {
  constexpr int D = 1 << K;
  for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < n_groups; g += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t base = group_base<K>(g, T);
    float2 x[D];
#pragma unroll
    for (int c = 0; c < D; ++c) x[c] = a[base + T.off[c]];
#pragma unroll
    for (int r = 0; r < D; ++r) {
      float yr = 0.f, yi = 0.f;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const float2 u = U.u[r * D + c];
        yr = fmaf(u.x, x[c].x, fmaf(-u.y, x[c].y, yr));
        yi = fmaf(u.x, x[c].y, fmaf(u.y, x[c].x, yi));
      }
      a[base + T.off[r]] = make_float2(yr, yi);
    }
  }
}

// Rolled rows, U in shared memory (two coefficients per 16-byte read).
template <int K>
__global__ void __launch_bounds__(kThreads, 2) k_kgate_c64_rows(float2* __restrict__ a, uint64_t n_groups, Targets<K> T,
                                                                UF32<K> U) {
  constexpr int D = 1 << K;
  __shared__ __align__(16) float2 su[D * D];
  for (int i = threadIdx.x; i < D * D; i += blockDim.x) su[i] = U.u[i];
  __syncthreads();
  const float4* su4 = reinterpret_cast<const float4*>(su);
  for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < n_groups; g += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t base = group_base<K>(g, T);
    float2 x[D];
#pragma unroll
    for (int c = 0; c < D; ++c) x[c] = a[base + T.off[c]];
#pragma unroll 1
    for (int r = 0; r < D; ++r) {
      float yr = 0.f, yi = 0.f;
#pragma unroll
      for (int c = 0; c < D; c += 2) {
        const float4 u = su4[(r * D + c) >> 1];
        yr = fmaf(u.x, x[c].x, fmaf(-u.y, x[c].y, yr));
        yi = fmaf(u.x, x[c].y, fmaf(u.y, x[c].x, yi));
        yr = fmaf(u.z, x[c + 1].x, fmaf(-u.w, x[c + 1].y, yr));
        yi = fmaf(u.z, x[c + 1].y, fmaf(u.w, x[c + 1].x, yi));
      }
      a[base + T.off[r]] = make_float2(yr, yi);
    }
  }
}

template <int K>
struct UF64 {
  double2 u[1 << (2 * K)];
};

template <int K>
__global__ void __launch_bounds__(kThreads, min_blocks<K + 1>()) k_kgate_c128_native(double2* __restrict__ a, uint64_t n_groups, Targets<K> T,
                                                                UF64<K> U) {
  constexpr int D = 1 << K;
  for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < n_groups; g += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t base = group_base<K>(g, T);
    double2 x[D];
#pragma unroll
    for (int c = 0; c < D; ++c) x[c] = a[base + T.off[c]];
#pragma unroll
    for (int r = 0; r < D; ++r) {
      double yr = 0.0, yi = 0.0;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const double2 u = U.u[r * D + c];
        yr = fma(u.x, x[c].x, fma(-u.y, x[c].y, yr));
        yi = fma(u.x, x[c].y, fma(u.y, x[c].x, yi));
      }
      a[base + T.off[r]] = make_double2(yr, yi);
    }
  }
}

template <int K>
__global__ void __launch_bounds__(kThreads, 1) k_kgate_c128_native_rows(double2* __restrict__ a, uint64_t n_groups,
                                                                        Targets<K> T, UF64<K> U) {
  constexpr int D = 1 << K;
  __shared__ double2 su[D * D];
  for (int i = threadIdx.x; i < D * D; i += blockDim.x) su[i] = U.u[i];
  __syncthreads();
  for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < n_groups; g += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t base = group_base<K>(g, T);
    double2 x[D];
#pragma unroll
    for (int c = 0; c < D; ++c) x[c] = a[base + T.off[c]];
#pragma unroll 1
    for (int r = 0; r < D; ++r) {
      double yr = 0.0, yi = 0.0;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const double2 u = su[r * D + c];
        yr = fma(u.x, x[c].x, fma(-u.y, x[c].y, yr));
        yi = fma(u.x, x[c].y, fma(u.y, x[c].x, yi));
      }
      a[base + T.off[r]] = make_double2(yr, yi);
    }
  }
}

// ---------------------------------------------------------------- staged tiles (complex64, low targets)
// When a target lies below bit 5, a thread's group is (partly) contiguous and
// a warp's loads stride across 32 cache lines.  The tiled kernel instead
// moves tiles of S = 2^s amplitudes, s = max(12, 8 + K): bits [0, t)
// contiguous (t >= 8) and the kh targets at or above t, so that a tile holds
// 2^(s - K) groups, a whole number of them per thread.  Tiles move between HBM and shared memory as coalesced
// 16-byte accesses; inside shared memory the target bits below 4 (the bank
// bits of a float2) are XORed with the lowest non-target bits at or above 4,
// which spreads the lanes' reads over the banks and keeps every group on its
// own 2^K positions.
template <int K>
__host__ __device__ constexpr int tile_bits() { return 8 + K > 12 ? 8 + K : 12; }

template <int K>
struct TilePlan {
  int t;                       // contiguous low bits of a tile
  int kh;                      // targets at or above t
  int hpos[K];                 // their global positions, ascending
  uint64_t hoff[1 << K];       // segment id -> global offset of the high targets
  int tt[K];                   // all tile-local target positions, ascending
  uint32_t toff[1 << K];       // element c -> tile-local offset (bit j of c <-> qubits[j])
  int nsw;                     // swizzle: target bits below 4 ...
  int sw_dst[4];               // ... their positions
  int sw_src[4];               // ... the non-target bits that flip them
};

template <int K>
__device__ __forceinline__ uint32_t tile_swz(uint32_t e, const TilePlan<K>& P) {
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (i < P.nsw) s |= ((e >> P.sw_src[i]) & 1u) << P.sw_dst[i];
  return s;
}

template <int K>
__global__ void __launch_bounds__(kThreads) k_kgate_c64_tiled(float2* __restrict__ a, uint64_t n_tiles, TilePlan<K> P,
                                                              UF32<K> U) {
  constexpr int D = 1 << K;
  constexpr int S = 1 << tile_bits<K>();
  constexpr int GPT = (S >> K) / kThreads;  // groups per thread
  extern __shared__ __align__(16) float2 tile[];
  float2* su = tile + S;                                     // U, D * D values
  uint64_t* hoff = reinterpret_cast<uint64_t*>(su + D * D);  // segment offsets
  for (int i = threadIdx.x; i < D * D; i += blockDim.x) su[i] = U.u[i];
#pragma unroll
  for (int h = 0; h < D; ++h)
    if (threadIdx.x == 0) hoff[h] = P.hoff[h];
  const uint32_t tmask = (1u << P.t) - 1u;
  constexpr int LPT = S / 2 / kThreads;  // 16-byte loads per thread per tile
  auto tile_base = [&](uint64_t tau) {
    uint64_t gbase = tau << P.t;
#pragma unroll
    for (int j = 0; j < K; ++j)
      if (j < P.kh) gbase = insert_zero(gbase, P.hpos[j]);
    return gbase;
  };
  // Software pipeline through registers: the next tile's loads are issued
  // before this tile's compute and store phases, so HBM latency overlaps them.
  // (k = 5 keeps its registers for the 32-amplitude groups and loads each
  // tile just before it is used.)
  constexpr bool kPipe = K <= 4;
  float4 pre[LPT];
  __syncthreads();  // hoff is visible
  if (kPipe && blockIdx.x < n_tiles) {
    const uint64_t gbase = tile_base(blockIdx.x);
#pragma unroll
    for (int k = 0; k < LPT; ++k) {
      const uint32_t e = 2 * (threadIdx.x + k * kThreads);
      pre[k] = *reinterpret_cast<const float4*>(a + (gbase | (e & tmask) | hoff[e >> P.t]));
    }
  }
  for (uint64_t tau = blockIdx.x; tau < n_tiles; tau += gridDim.x) {
    const uint64_t gbase = tile_base(tau);
    if constexpr (!kPipe) {
#pragma unroll
      for (int k = 0; k < LPT; ++k) {
        const uint32_t e = 2 * (threadIdx.x + k * kThreads);
        pre[k] = *reinterpret_cast<const float4*>(a + (gbase | (e & tmask) | hoff[e >> P.t]));
      }
    }
    __syncthreads();  // the previous tile's stores have read the buffer
#pragma unroll
    for (int k = 0; k < LPT; ++k) {
      const uint32_t e = 2 * (threadIdx.x + k * kThreads);
      const uint32_t sw = tile_swz<K>(e, P);
      float4 v = pre[k];
      if (sw & 1u) v = make_float4(v.z, v.w, v.x, v.y);
      *reinterpret_cast<float4*>(tile + ((e ^ sw) & ~1u)) = v;
    }
    __syncthreads();
    const uint64_t nxt = tau + gridDim.x;
    if (kPipe && nxt < n_tiles) {
      const uint64_t nbase = tile_base(nxt);
#pragma unroll
      for (int k = 0; k < LPT; ++k) {
        const uint32_t e = 2 * (threadIdx.x + k * kThreads);
        pre[k] = *reinterpret_cast<const float4*>(a + (nbase | (e & tmask) | hoff[e >> P.t]));
      }
    }
#pragma unroll 1
    for (int j = 0; j < GPT; ++j) {
      uint32_t gb = threadIdx.x + j * kThreads;
#pragma unroll
      for (int q = 0; q < K; ++q) gb = (uint32_t)insert_zero(gb, P.tt[q]);
      const uint32_t gsw = tile_swz<K>(gb, P);
      float2 x[D];
#pragma unroll
      for (int c = 0; c < D; ++c) x[c] = tile[gb | (P.toff[c] ^ gsw)];
#pragma unroll(K <= 3 ? D : 1)
      for (int r = 0; r < D; ++r) {
        float yr = 0.f, yi = 0.f;
#pragma unroll
        for (int c = 0; c < D; ++c) {
          const float2 u = su[r * D + c];
          yr = fmaf(u.x, x[c].x, fmaf(-u.y, x[c].y, yr));
          yi = fmaf(u.x, x[c].y, fmaf(u.y, x[c].x, yi));
        }
        tile[gb | (P.toff[r] ^ gsw)] = make_float2(yr, yi);
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < LPT; ++k) {
      const uint32_t e = 2 * (threadIdx.x + k * kThreads);
      const uint32_t sw = tile_swz<K>(e, P);
      float4 v = *reinterpret_cast<const float4*>(tile + ((e ^ sw) & ~1u));
      if (sw & 1u) v = make_float4(v.z, v.w, v.x, v.y);
      *reinterpret_cast<float4*>(a + (gbase | (e & tmask) | hoff[e >> P.t])) = v;
    }
  }
}

// Tile geometry for qubits[0..K) on n qubits; false when the state is
// smaller than a tile.
template <int K>
bool make_tile_plan(int n, const int* qubits, TilePlan<K>& P) {
  constexpr int s = tile_bits<K>();
  if (n < s) return false;
  std::memset(&P, 0, sizeof(P));
  int t = s, kh = 0;
  for (int it = 0; it < 8; ++it) {  // t = s - (targets at or above t), a fixed point
    kh = 0;
    for (int j = 0; j < K; ++j) kh += qubits[j] >= t;
    if (s - kh == t) break;
    t = s - kh;
  }
  P.t = t;
  P.kh = kh;
  int hs[K], nh = 0;
  for (int j = 0; j < K; ++j)
    if (qubits[j] >= t) hs[nh++] = qubits[j];
  std::sort(hs, hs + nh);
  for (int j = 0; j < nh; ++j) P.hpos[j] = hs[j];
  for (int h = 0; h < (1 << kh); ++h) {
    uint64_t o = 0;
    for (int j = 0; j < kh; ++j) o |= (uint64_t)((h >> j) & 1) << hs[j];
    P.hoff[h] = o;
  }
  // tile-local position of each target: below t as is, else t + rank
  int tl[K];
  for (int j = 0; j < K; ++j) {
    if (qubits[j] < t) tl[j] = qubits[j];
    else tl[j] = t + (int)(std::lower_bound(hs, hs + nh, qubits[j]) - hs);
  }
  int srt[K];
  for (int j = 0; j < K; ++j) srt[j] = tl[j];
  std::sort(srt, srt + K);
  for (int j = 0; j < K; ++j) P.tt[j] = srt[j];
  for (int c = 0; c < (1 << K); ++c) {
    uint32_t o = 0;
    for (int j = 0; j < K; ++j) o |= (uint32_t)((c >> j) & 1) << tl[j];
    P.toff[c] = o;
  }
  uint32_t tmask = 0;
  for (int j = 0; j < K; ++j) tmask |= 1u << tl[j];
  int src = 4;
  for (int b = 0; b < 4; ++b) {
    if (!((tmask >> b) & 1u)) continue;
    while ((tmask >> src) & 1u) ++src;
    P.sw_dst[P.nsw] = b;
    P.sw_src[P.nsw] = src;
    ++P.nsw;
    ++src;
  }
  return true;
}

// Emulated complex128: output component (row r, re or im) is a real dot
// product of 2 * 2^k terms over (x_0.re, x_0.im, x_1.re, ...).
template <int K>
struct UDF {
  dfx::Coef c[2 * (1 << K) * 2 * (1 << K)];
};

template <int K>
__global__ void __launch_bounds__(kThreads, min_blocks<K + 2>()) k_kgate_c128_df(double2* __restrict__ a, uint64_t n_groups, Targets<K> T,
                                                            UDF<K> U, unsigned* flag) {
  constexpr int D = 1 << K;
  constexpr int M = 2 * D;  // real terms per output component
  unsigned bad = 0;
  for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < n_groups; g += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t base = group_base<K>(g, T);
    float xh[M], xl[M];
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const double2 v = a[base + T.off[c]];
      dfx::split(v.x, xh[2 * c], xl[2 * c], bad);
      dfx::split(v.y, xh[2 * c + 1], xl[2 * c + 1], bad);
    }
#pragma unroll
    for (int r = 0; r < D; ++r) {
      float p, e;
      dfx::dot<M>(&U.c[(2 * r) * M], xh, xl, p, e);
      const double yr = dfx::join(p, e);
      dfx::dot<M>(&U.c[(2 * r + 1) * M], xh, xl, p, e);
      a[base + T.off[r]] = make_double2(yr, dfx::join(p, e));
    }
  }
  if (bad) atomicOr(flag, 1u);
}

// The double-float k-qubit gate on paired FP32 instructions.  Each thread owns
// two amplitude groups (g and g + S, S = the grid's thread count) and runs
// dfx::dot's operation sequence for both at once, one group per lane of the
// .f32x2 instructions, in half the FP32 instructions.  The coefficients are
// staged in shared memory duplicated into both lanes as (h, h), (h52, h52),
// (l, l).  The error-free transformations need every product rounded on its
// own before it is added: no rounded product feeds a packed add or subtract
// directly (the negated product -fl(h x) is formed by flipping sign bits with
// an integer XOR), so no multiply can be fused into the sums.  The first term
// runs through the same steps from p = e = 0, which gives it exactly the
// scalar first-term values (p = fl(h x), e = the product's residual).
__device__ __forceinline__ f2::P neg_bits(f2::P a) {
  f2::P d;
  asm("xor.b64 %0, %1, 0x8000000080000000;" : "=l"(d) : "l"(a));
  return d;
}

template <int M>
__device__ __forceinline__ void dot2(const ulonglong2* __restrict__ c, const f2::P* X, const f2::P* XL, f2::P& p,
                                     f2::P& e) {
  p = 0ull;
  e = 0ull;
#pragma unroll
  for (int j = 0; j < M; ++j) {
    const ulonglong2 k0 = c[2 * j];  // (h, h), (h52, h52)
    const f2::P kl = reinterpret_cast<const f2::P*>(c)[4 * j + 2];  // (l, l)
    const f2::P qn = neg_bits(f2::mul(k0.x, X[j]));  // -fl(h x)
    const f2::P eq = f2::fma(k0.x, X[j], qn);         // h x - fl(h x), exact
    // TwoSum(p, q) with q = -qn: s = p + q, t = (p - (s - bb)) + (q - bb)
    const f2::P s = f2::sub(p, qn);
    const f2::P bb = f2::sub(s, p);
    const f2::P t = f2::sub(f2::sub(p, f2::sub(s, bb)), f2::add(qn, bb));
    p = s;
    e = f2::add(e, f2::add(eq, t));
    e = f2::fma(k0.y, XL[j], e);
    e = f2::fma(kl, X[j], e);
  }
}

template <int K>
__global__ void __launch_bounds__(kThreads, K <= 3 ? 2 : 1) k_kgate_c128_df2(double2* __restrict__ a, uint64_t n_groups,
                                                                Targets<K> T, UDF<K> U, unsigned* flag) {
  constexpr int D = 1 << K;
  constexpr int M = 2 * D;
  __shared__ ulonglong2 sc[2 * (2 * D * M)];
  for (int i = threadIdx.x; i < 2 * D * M; i += blockDim.x) {
    const dfx::Coef k = U.c[i];
    sc[2 * i] = make_ulonglong2(f2::pack(k.h, k.h), f2::pack(k.h52, k.h52));
    sc[2 * i + 1] = make_ulonglong2(f2::pack(k.l, k.l), 0ull);
  }
  __syncthreads();
  unsigned bad = 0;
  const uint64_t S = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t g0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g0 < n_groups; g0 += 2 * S) {
    const bool two = g0 + S < n_groups;  // the last round may hold one group: lane 1 repeats it, unstored
    const uint64_t b0 = group_base<K>(g0, T);
    const uint64_t b1 = two ? group_base<K>(g0 + S, T) : b0;
    f2::P X[M], XL[M];
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const double2 v0 = a[b0 + T.off[c]];
      const double2 v1 = a[b1 + T.off[c]];
      float h0, l0, h1, l1;
      dfx::split(v0.x, h0, l0, bad);
      dfx::split(v1.x, h1, l1, bad);
      X[2 * c] = f2::pack(h0, h1);
      XL[2 * c] = f2::pack(l0, l1);
      dfx::split(v0.y, h0, l0, bad);
      dfx::split(v1.y, h1, l1, bad);
      X[2 * c + 1] = f2::pack(h0, h1);
      XL[2 * c + 1] = f2::pack(l0, l1);
    }
#pragma unroll(K >= 3 ? 1 : D)
    for (int r = 0; r < D; ++r) {
      f2::P p, e;
      float p0, p1, e0, e1;
      dot2<M>(&sc[2 * (2 * r) * M], X, XL, p, e);
      f2::unpack(p, p0, p1);
      f2::unpack(e, e0, e1);
      const double re0 = dfx::join(p0, e0), re1 = dfx::join(p1, e1);
      dot2<M>(&sc[2 * (2 * r + 1) * M], X, XL, p, e);
      f2::unpack(p, p0, p1);
      f2::unpack(e, e0, e1);
      a[b0 + T.off[r]] = make_double2(re0, dfx::join(p0, e0));
      if (two) a[b1 + T.off[r]] = make_double2(re1, dfx::join(p1, e1));
    }
  }
  if (bad) atomicOr(flag, 1u);
}

template <int K>
Targets<K> make_targets(const int* qubits) {
  Targets<K> T;
  int pos[K];
  for (int j = 0; j < K; ++j) pos[j] = qubits[j];
  std::sort(pos, pos + K);
  for (int j = 0; j < K; ++j) T.pos[j] = pos[j];
  for (int c = 0; c < (1 << K); ++c) {
    uint64_t o = 0;
    for (int j = 0; j < K; ++j) o |= (uint64_t)((c >> j) & 1) << qubits[j];
    T.off[c] = o;
  }
  return T;
}

// Kernel choices of iqs_kq_autotune, per (dtype, emulated arithmetic, k,
// targets below bit 5): the variant (kVarAuto: the fixed rule below) and the
// grid size in blocks per SM of the grid-stride variants.
enum { kVarAuto = 0, kVarTiled = 1, kVarUnrolled = 2, kVarRows = 3, kVarTensor = 4 };
struct KqChoice {
  int variant = kVarAuto;
  int per_sm = 8;
};
std::mutex g_kq_mutex;
std::map<std::tuple<int, int, int, int>, KqChoice> g_kq_choice;
bool g_kq_cache_loaded = false;

std::tuple<int, int, int, int> kq_key(const iqs_reg* r, int k, const int* qubits) {
  bool low = false;
  for (int j = 0; j < k; ++j) low |= qubits[j] < 5;
  return std::make_tuple(r->dtype, use_emulated(r) ? 1 : 0, k, low ? 1 : 0);
}

// Lines "kq <dtype> <emulated> <k> <low> <variant> <per_sm>" of IQS_AUTOTUNE_CACHE.
void load_kq_cache_locked() {
  if (g_kq_cache_loaded) return;
  g_kq_cache_loaded = true;
  const char* path = std::getenv("IQS_AUTOTUNE_CACHE");
  if (path == nullptr) return;
  FILE* f = std::fopen(path, "r");
  if (f == nullptr) return;
  char line[256];
  while (std::fgets(line, sizeof(line), f)) {
    char kind[16];
    int dt, em, k, low, var, per_sm;
    if (std::sscanf(line, "%15s %d %d %d %d %d %d", kind, &dt, &em, &k, &low, &var, &per_sm) == 7 &&
        std::strcmp(kind, "kq") == 0 && var >= 0 && var <= 4 && per_sm >= 1 && per_sm <= 64)
      g_kq_choice[std::make_tuple(dt, em, k, low)] = KqChoice{var, per_sm};
  }
  std::fclose(f);
}

KqChoice kq_choice(const iqs_reg* r, int k, const int* qubits) {
  std::lock_guard<std::mutex> lock(g_kq_mutex);
  load_kq_cache_locked();
  auto it = g_kq_choice.find(kq_key(r, k, qubits));
  return it == g_kq_choice.end() ? KqChoice() : it->second;
}

template <int K>
cudaError_t launch_k(iqs_reg* r, const int* qubits, const double* U, KqChoice ch) {
  constexpr int D = 1 << K;
  const uint64_t n_groups = num_amps(r) >> K;
  const unsigned grid = grid_for(n_groups, 1, ch.per_sm);
  const Targets<K> T = make_targets<K>(qubits);
  if (r->dtype == IQS_C64) {
    if constexpr (K <= kMaxK64) {
      UF32<K> u;
      for (int i = 0; i < D * D; ++i) u.u[i] = make_float2((float)U[2 * i], (float)U[2 * i + 1]);
      bool low = false;
      for (int j = 0; j < K; ++j) low |= qubits[j] < 5;
      TilePlan<K> P;
      if (low && ch.variant != kVarUnrolled && ch.variant != kVarRows && make_tile_plan<K>(r->n, qubits, P)) {
        const size_t smem = sizeof(float2) * ((size_t)(1 << tile_bits<K>()) + (size_t)(D * D)) + sizeof(uint64_t) * D;
        static PerDevice resident;  // per K instantiation: resident blocks per SM
        int per_sm = 0;
        cudaError_t e = resident.get(&per_sm, [&](int* x) {
          cudaError_t f = cudaFuncSetAttribute(k_kgate_c64_tiled<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
          if (f == cudaSuccess) f = cudaOccupancyMaxActiveBlocksPerMultiprocessor(x, k_kgate_c64_tiled<K>, kThreads, smem);
          return f;
        });
        if (e != cudaSuccess) return e;
        const uint64_t n_tiles = num_amps(r) >> tile_bits<K>();
        const unsigned tg = (unsigned)std::min<uint64_t>(n_tiles, (uint64_t)per_sm * kSMs);
        k_kgate_c64_tiled<K><<<tg, kThreads, smem, r->stream>>>((float2*)r->data, n_tiles, P, u);
        return launched(1);
      }
      if (K >= 4 || ch.variant == kVarRows)
        k_kgate_c64_rows<K><<<grid, kThreads, 0, r->stream>>>((float2*)r->data, n_groups, T, u);
      else if constexpr (K < 4)
        k_kgate_c64<K><<<grid, kThreads, 0, r->stream>>>((float2*)r->data, n_groups, T, u);
      return launched(1);
    }
  } else if (!use_emulated(r)) {
    if constexpr (K <= kMaxK128) {
      UF64<K> u;
      for (int i = 0; i < D * D; ++i) u.u[i] = make_double2(U[2 * i], U[2 * i + 1]);
      if (K >= 4 || ch.variant == kVarRows)
        k_kgate_c128_native_rows<K><<<grid, kThreads, 0, r->stream>>>((double2*)r->data, n_groups, T, u);
      else if constexpr (K < 4)
        k_kgate_c128_native<K><<<grid, kThreads, 0, r->stream>>>((double2*)r->data, n_groups, T, u);
      return launched(1);
    }
  } else {
    if constexpr (K <= kMaxK128) {
      // the fixed rule: k >= 3 on the tensor cores (k = 2 is faster as paired
      // FP32 below; k = 5 has only the tensor-core kernel)
      if (kq_tensor_supported(K) && (K == 5 || ch.variant == kVarTensor || (ch.variant == kVarAuto && K >= 3)))
        return launch_kq_c128_tensor(r, K, qubits, U);
    }
    if constexpr (K <= 4) {
      constexpr int M = 2 * D;
      UDF<K> u;
      for (int row = 0; row < D; ++row)
        for (int c = 0; c < D; ++c) {
          const double ur = U[2 * (row * D + c)], ui = U[2 * (row * D + c) + 1];
          u.c[(2 * row) * M + 2 * c] = dfx::make_coef(ur);           // re += Re(u) Re(x)
          u.c[(2 * row) * M + 2 * c + 1] = dfx::make_coef(-ui);      // re -= Im(u) Im(x)
          u.c[(2 * row + 1) * M + 2 * c] = dfx::make_coef(ui);       // im += Im(u) Re(x)
          u.c[(2 * row + 1) * M + 2 * c + 1] = dfx::make_coef(ur);   // im += Re(u) Im(x)
        }
      if constexpr (K >= 2) {
        const unsigned grid2 = grid_for((n_groups + 1) / 2, 1, ch.per_sm);
        k_kgate_c128_df2<K><<<grid2, kThreads, 0, r->stream>>>((double2*)r->data, n_groups, T, u, r->flag);
      } else {
        k_kgate_c128_df<K><<<grid, kThreads, 0, r->stream>>>((double2*)r->data, n_groups, T, u, r->flag);
      }
      return launched(1);
    }
  }
  return cudaErrorInvalidValue;  // unreachable: k is checked against the dtype's limit by the caller
}

}  // namespace

int max_kq(int dtype) { return dtype == IQS_C64 ? kMaxK64 : kMaxK128; }

namespace {
cudaError_t launch_kq_with(iqs_reg* r, int k, const int* qubits, const double* U, KqChoice ch) {
  switch (k) {
    case 1: return launch_k<1>(r, qubits, U, ch);
    case 2: return launch_k<2>(r, qubits, U, ch);
    case 3: return launch_k<3>(r, qubits, U, ch);
    case 4: return launch_k<4>(r, qubits, U, ch);
    case 5: return launch_k<5>(r, qubits, U, ch);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace

cudaError_t launch_kq(iqs_reg* r, int k, const int* qubits, const double* U) {
  return launch_kq_with(r, k, qubits, U, kq_choice(r, k, qubits));
}

void set_kq_choice(const iqs_reg* r, int k, const int* qubits, int variant, int per_sm) {
  std::lock_guard<std::mutex> lock(g_kq_mutex);
  load_kq_cache_locked();
  g_kq_choice[kq_key(r, k, qubits)] = KqChoice{variant, per_sm};
}

// Times every variant and grid size of a k-qubit gate on these targets on the
// register's state (applying U and then its conjugate transpose, so the state
// comes back up to rounding), and keeps the fastest for (dtype, arithmetic,
// k, low targets).  Returns the best time of one gate in ms.
cudaError_t tune_kq(iqs_reg* r, int k, const int* qubits, const double* U, double* best_ms, int* variant, int* per_sm) {
  const int D = 1 << k;
  std::vector<double> Uh((size_t)2 * D * D);
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) {
      Uh[2 * (i * D + j)] = U[2 * (j * D + i)];
      Uh[2 * (i * D + j) + 1] = -U[2 * (j * D + i) + 1];
    }
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return e;
  std::vector<KqChoice> cands;
  const int vars[4] = {kVarAuto, kVarTiled, kVarUnrolled, kVarRows};
  for (int v : vars)
    for (int ps : {4, 8, 16, 32}) cands.push_back(KqChoice{v, ps});
  if (use_emulated(r) && kq_tensor_supported(k)) cands.push_back(KqChoice{kVarTensor, 1});  // one CTA per SM
  double best = 1e300;
  KqChoice pick;
  for (const KqChoice& c : cands) {
    float tot = 0.f;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // U then U^dagger, timed together
      e = launch_kq_with(r, k, qubits, U, c);
      if (e == cudaSuccess) e = cudaEventRecord(e0, r->stream);
      if (e == cudaSuccess) e = launch_kq_with(r, k, qubits, Uh.data(), c);
      if (e == cudaSuccess) e = launch_kq_with(r, k, qubits, U, c);
      if (e == cudaSuccess) e = cudaEventRecord(e1, r->stream);
      if (e == cudaSuccess) e = launch_kq_with(r, k, qubits, Uh.data(), c);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      tot += ms;
    }
    if (e != cudaSuccess) break;
    const double per_gate = tot / 4.0;
    if (per_gate < best) {
      best = per_gate;
      pick = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  {
    std::lock_guard<std::mutex> lock(g_kq_mutex);
    load_kq_cache_locked();
    g_kq_choice[kq_key(r, k, qubits)] = pick;
  }
  if (const char* path = std::getenv("IQS_AUTOTUNE_CACHE")) {
    if (FILE* f = std::fopen(path, "a")) {
      const auto key = kq_key(r, k, qubits);
      std::fprintf(f, "kq %d %d %d %d %d %d\n", std::get<0>(key), std::get<1>(key), std::get<2>(key),
                   std::get<3>(key), pick.variant, pick.per_sm);
      std::fclose(f);
    }
  }
  *best_ms = best;
  *variant = pick.variant;
  *per_sm = pick.per_sm;
  return cudaSuccess;
}

}  // namespace iqs
