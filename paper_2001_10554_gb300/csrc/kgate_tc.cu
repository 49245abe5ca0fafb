// Dense k-qubit gates (Section 2, "Scope and basic use": custom multi-qubit
// gates) on complex128 states, with the contraction on the tcgen05 tensor
// cores.
//
// A k-qubit gate is a batched matrix product: every group of D = 2^k
// amplitudes (the other n - k bits fixed) is multiplied by U.  In real form
// each group is a row x of R = 2D reals (re, im interleaved) and the output
// row is y = W x with the R x R real matrix
//   W[2r][2c] = Re u_rc, W[2r][2c+1] = -Im u_rc, W[2r+1][2c] = Im u_rc,
//   W[2r+1][2c+1] = Re u_rc.
// FP64 accuracy on bf16 tensor cores comes from exact digit splitting (the
// error-free splitting of Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication", 2012):
//   * each group takes the largest biased FP64 exponent e_max of its reals;
//     every real becomes a signed fixed-point integer
//     F = sign(x) floor(|x| 2^(1075 - e_max)) with |F| < 2^53, written in six balanced
//     radix-2^9 digits f_0..f_5 in [-256, 256]
//     (x 2^(1030 - e_max) = sum_l f_l 2^(-9 l));
//   * each row of W is scaled the same way and split into six digits
//     b_0..b_5, exactly in FP64, by every CTA in its prologue;
//   * a digit times 2^(-9 l) is exact in bf16 (at most 8 significant bits),
//     a product of two digits exact in FP32, and the tensor cores' FP32 sums
//     over the R terms of one digit level d = l + j are exact integers times
//     2^(-9 d) for d <= 3 (|sum| <= (d + 1) R 2^16 <= 2^24 for R <= 64);
//   * levels 4 and 5 share one accumulator (its rounding is below 2^-56 of
//     the row's scale) and levels above 5 are dropped (at most 7 * 2^-52 of
//     max|W| max|x| per term; the balanced digits make it far smaller in
//     practice).
// The five accumulators are added in double-float and rounded to FP64, then
// rescaled by the two powers of two.  Result: at most 19 * 2^-53 * R *
// max|W| * max|x| per output (max over the row and the group), the order of
// an FP64 dot product's error, with the FP64 pipe unused.
//
// Kernel: one CTA per SM, split into teams that each work on one 128-group
// tile at a time (k = 5: one team of 512 threads, four threads per group;
// k = 4: two teams of 256 threads, two threads per group; k = 3: five teams
// of 128; k = 2: six teams of 128).  Each thread stages its
// part of the next tile's groups into shared memory with cp.async while the
// current tile is computed (one read of the state), splits its reals into
// six digit slices written as bf16 into the team's A operand (K-major core
// matrices), and after the team's barrier one thread issues the 21
// digit-pair products (x R/16 K-steps) of M = 128, N = max(R, 16) into the
// team's five TMEM accumulators and commits them to an mbarrier.  Each thread
// then reads its own TMEM lane, rounds the sums to FP64 and writes its part
// of the group back (one write).  The teams of a CTA take turns on the
// tensor cores while the others load, split or write.  With a target below
// bit 7 a warp moves its 32 groups together so that the copies stay
// coalesced.  Waits on the mbarrier are bounded: a wait that gives up sets
// bit 1 of the error flag (IQS_ETIMEOUT) and the CTA frees its tensor memory
// and returns.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "df64.cuh"
#include "internal.h"
#include "tc.cuh"

namespace iqs {
namespace {

constexpr int kSlices = 6;  // balanced radix-2^9 digits per operand
constexpr int kAcc = 5;     // accumulators: digit levels 0, 1, 2, 3, and 4..5
constexpr int kRows = 128;  // groups per tile (the MMA's M)
constexpr uint32_t kWaitPolls = 1u << 22;

template <int K>
struct TcShape {
  static constexpr int D = 1 << K;
  static constexpr int R = 2 * D;             // reals per group
  static constexpr int KP = R < 16 ? 16 : R;  // MMA K extent (zero-padded)
  static constexpr int NP = R < 16 ? 16 : R;  // MMA N extent (padded rows of W are zero)
  // A team of TPG warpgroups works on one 128-group tile: thread (sub, m)
  // owns reals [sub RT, (sub + 1) RT) of group row m.  TEAMS teams per CTA.
  static constexpr int TPG = K >= 5 ? 4 : K == 4 ? 2 : 1;
  static constexpr int RT = R / TPG;
  static constexpr int DT = D / TPG;
  static constexpr int TEAMS = K >= 5 ? 1 : K == 4 ? 2 : K == 3 ? 5 : 6;
  static constexpr int TEAM_THREADS = TPG * 128;
  static constexpr int THREADS = TEAMS * TEAM_THREADS;
  static constexpr uint32_t SBO = (KP / 8) * 128;
  static constexpr uint32_t A_SLICE = kRows * KP * 2;
  static constexpr uint32_t A_BYTES = kSlices * A_SLICE;
  static constexpr uint32_t B_SLICE = NP * KP * 2;
  static constexpr uint32_t B_BYTES = kSlices * B_SLICE;
  static constexpr uint32_t X_BYTES = kRows * D * 16;  // staged input of one tile: [element c][row m]
  // shared memory: TMEM address slot at 0, mbarriers from 8, partial group
  // exponents from 1024 (TEAMS x TPG x 128 words), then B, A, X
  static_assert(8 + 8 * TEAMS <= 1024, "header area");
  static constexpr uint32_t EMX_OFF = 1024;
  static constexpr uint32_t B_OFF = 4096;
  static_assert(EMX_OFF + TEAMS * TPG * 128 * 4 <= B_OFF, "exponent exchange area");
  static constexpr uint32_t A_OFF = B_OFF + (B_BYTES + 1023) / 1024 * 1024;
  static constexpr uint32_t X_OFF = A_OFF + TEAMS * A_BYTES;
  static constexpr uint32_t SMEM = X_OFF + TEAMS * X_BYTES;
  static_assert(SMEM <= 227 * 1024, "shared memory per CTA");
  static constexpr int TCOLS = kAcc * NP;  // TMEM columns per team
  static_assert(TEAMS * TCOLS <= 512, "tensor memory holds 512 columns");
  static_assert(RT % 8 == 0, "a thread writes whole core-matrix rows");
};

template <int K>
struct TcParams {
  int pos[K];                    // target positions, ascending
  uint64_t off[1 << K];          // index offset of group element c
  int ro[TcShape<K>::NP];        // per row o of W: max_i |W[o][i]| in [2^(ro - 1), 2^ro); 0 for a zero row
  double u[2 << (2 * K)];        // U row-major, (re, im) pairs
};

template <int K>
__device__ __forceinline__ uint64_t group_base(uint64_t g, const TcParams<K>& P) {
  uint64_t x = g;
#pragma unroll
  for (int j = 0; j < K; ++j) x = insert_zero(x, P.pos[j]);
  return x;
}

// The six digits of the real x with FP64 bits (hi:lo) in a group whose
// largest biased exponent is ``emax``: F = sign(x) floor(|x| 2^(1075 - emax)),
// so that x 2^(1030 - emax) = F 2^-45 = sum_l f_l 2^(-9 l) up to the
// truncation of F (less than one unit of 2^-45, against
// |x 2^(1030 - emax)| < 2^8).  Zeros and subnormals give F = 0.
// out[l] = f_l 2^(-9 l).
//
// Balanced digits without a carry chain: G = F + 256 (2^36 + 2^27 + 2^18 +
// 2^9 + 1) has plain 9-bit fields g_1..g_5 and top part g_0 = floor(G / 2^45),
// and f_l = g_l - 256 (l >= 1), f_0 = g_0.  A field g is turned into the
// float 2^23 + g by OR-ing in the exponent of 2^23, and one FMA removes
// 2^23 + 256 and applies the level's power of two, exactly.
constexpr unsigned long long kDigitBias = 256ull * ((1ull << 36) + (1ull << 27) + (1ull << 18) + (1ull << 9) + 1ull);

__device__ __forceinline__ float field_value(uint32_t g9, float w) {
  return fmaf(__uint_as_float(g9 | 0x4B000000u), w, -8388864.0f * w);  // (g - 256) w
}

__device__ __forceinline__ void digits(uint32_t lo, uint32_t hi, uint32_t emax, float (&out)[kSlices]) {
  const uint32_t e = (hi >> 20) & 0x7ffu;
  const uint32_t sh = emax - e;
  unsigned long long T = 0;  // |F|
  if (e != 0u && sh < 54u) T = (((unsigned long long)((hi & 0xfffffu) | 0x100000u) << 32) | lo) >> sh;
  const unsigned long long G = (hi >> 31) ? kDigitBias - T : kDigitBias + T;
  const uint32_t gl = (uint32_t)G, gh = (uint32_t)(G >> 32);
  out[0] = __int_as_float(0x4B400000 + ((int)gh >> 13)) - 12582912.0f;
  out[1] = field_value((gh >> 4) & 511u, 0x1p-9f);
  out[2] = field_value(__funnelshift_r(gl, gh, 27) & 511u, 0x1p-18f);
  out[3] = field_value((gl >> 18) & 511u, 0x1p-27f);
  out[4] = field_value((gl >> 9) & 511u, 0x1p-36f);
  out[5] = field_value(gl & 511u, 0x1p-45f);
}

// Two floats that are exact in bf16 as one bf16x2 word (x in the low half).
__device__ __forceinline__ uint32_t pack_bf16(float x, float y) {
  return __byte_perm(__float_as_uint(x), __float_as_uint(y), 0x7632);
}

// y * 2^adj for a double y from join(); results below the normal range flush
// to zero, results above it raise the flag.  (The careful path, for groups
// whose scale is near either end of the FP64 range.)
__device__ __forceinline__ double scale_out(double y, int adj, unsigned& bad) {
  const uint32_t yh = (uint32_t)__double2hiint(y), yl = (uint32_t)__double2loint(y);
  const int e = (int)((yh >> 20) & 0x7ffu);
  const int ne = e + adj;
  bad |= (e != 0 && ne >= 0x7ff) ? 1u : 0u;
  if (e == 0 || ne <= 0) return __hiloint2double((int)(yh & 0x80000000u), 0);
  return __hiloint2double((int)(yh + ((uint32_t)adj << 20)), (int)yl);
}

// The five accumulators of output real q as an unevaluated pair s + lo:
// levels 0..3 are exact, so the TwoSum chain keeps their sum exactly.
__device__ __forceinline__ void combine(const uint32_t (&v)[kAcc][8], int q, float& s, float& lo) {
  float t1, t2, t3;
  dfx::two_sum(__uint_as_float(v[0][q]), __uint_as_float(v[1][q]), s, t1);
  dfx::two_sum(s, __uint_as_float(v[2][q]), s, t2);
  dfx::two_sum(s, __uint_as_float(v[3][q]), s, t3);
  lo = t1 + (t2 + (t3 + __uint_as_float(v[4][q])));
}

// dfx::join(p, e) * 2^adj in one pass: the power of two goes into the
// exponent that join assembles.  Valid when every nonzero result stays a
// normal double: the caller checks that for the whole group (a nonzero |p|
// here lies in [2^-126, 2^24], so 2^adj in [2^-895, 2^998] suffices).
__device__ __forceinline__ double join_scaled(float p, float e, int adj) {
  const float h = p + e;
  const float l = e - (h - p);
  const unsigned hb = __float_as_uint(h);
  const unsigned rb = __float_as_uint(__fadd_rz(h, l));
  unsigned dhi = (((hb & 0x7fffffffu) >> 3) + ((unsigned)(896 + adj) << 20)) | (hb & 0x80000000u);
  dhi = (hb << 1) ? dhi : (hb & 0x80000000u);
  const unsigned dlo = hb << 29;
  const unsigned er = max(rb & 0x7f800000u, 52u << 23);
  const unsigned sb = ((306u << 23) - er) | (hb & 0x80000000u);
  const int k = __float2int_rn(l * __uint_as_float(sb));
  unsigned long long bits = ((unsigned long long)dhi << 32) | dlo;
  bits += (unsigned long long)(long long)k;
  return __longlong_as_double((long long)bits);
}

// Thread 0 of a warpgroup: every digit pair (l, j) with l + j <= 5 into the
// accumulator of level min(l + j, 4); the first product of each accumulator
// overwrites it.
template <int K>
__device__ __forceinline__ void issue_mmas(uint32_t tacc, uint32_t a_s, uint32_t b_s) {
  using S = TcShape<K>;
  constexpr uint32_t idesc = tc::idesc_bf16_f32(kRows, S::NP);
#pragma unroll
  for (int d = 0; d < kSlices; ++d) {
#pragma unroll
    for (int l = 0; l <= d; ++l) {
      const int j = d - l;
      const int acc = d < kAcc - 1 ? d : kAcc - 1;
      const bool first = l == 0 && d <= kAcc - 1;
#pragma unroll
      for (int ks = 0; ks < S::KP / 16; ++ks) {
        const uint64_t ad = tc::sdesc(a_s + l * S::A_SLICE + ks * 256, 128, S::SBO);
        const uint64_t bd = tc::sdesc(b_s + j * S::B_SLICE + ks * 256, 128, S::SBO);
        tc::mma_bf16(tacc + (uint32_t)(acc * S::NP), ad, bd, idesc, (first && ks == 0) ? 0u : 1u);
      }
    }
  }
}

// Entry (o, i) of U's real form W.
template <int K>
__device__ __forceinline__ double w_entry(const TcParams<K>& P, int o, int i) {
  constexpr int D = 1 << K;
  const int r = o >> 1, c = i >> 1;
  const double ur = P.u[2 * (r * D + c)], ui = P.u[2 * (r * D + c) + 1];
  return (o & 1) == 0 ? ((i & 1) == 0 ? ur : -ui) : ((i & 1) == 0 ? ui : ur);
}

__device__ __forceinline__ float digit_weight(int j) {
  return __uint_as_float((uint32_t)(127 - 9 * j) << 23);  // 2^(-9 j), j <= 5
}

// Stage elements [c0, c0 + DT) of group ``g`` into the team's input buffer
// (layout [element c][row m], 16 bytes each).
template <int K>
__device__ __forceinline__ void stage_group(uint8_t* X, int m, int c0, const double2* a, uint64_t base,
                                            const TcParams<K>& P) {
#pragma unroll
  for (int c = 0; c < TcShape<K>::DT; ++c) {
    const uint32_t dst = tc::smem_u32(X + ((size_t)(c0 + c) * kRows + m) * 16);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(a + base + P.off[c0 + c]) : "memory");
  }
}

// With a target below bit 7 the elements of neighbouring groups interleave
// in memory, and one thread per group would read and write them strided.
// There a warp moves its 32 groups together: in round j lane i handles
// element c0 + i % DT of the warp's group j 32/DT + i / DT, so consecutive
// lanes touch consecutive elements; the group's base index comes from its
// owner lane by shuffle.  ``mw`` is the warp's first row in the tile.
template <int K>
__device__ __forceinline__ void stage_warp(uint8_t* X, int mw, int lane, int c0, const double2* a, uint64_t base_own,
                                           bool act_own, uint64_t off_lane) {
  constexpr int DT = TcShape<K>::DT;
  const int cl = lane % DT;
#pragma unroll
  for (int j = 0; j < DT; ++j) {
    const int src = j * (32 / DT) + lane / DT;
    const uint64_t b = __shfl_sync(0xffffffffu, base_own, src);
    const int act = __shfl_sync(0xffffffffu, (int)act_own, src);
    if (act) {
      const uint32_t dst = tc::smem_u32(X + ((size_t)(c0 + cl) * kRows + mw + src) * 16);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(a + b + off_lane) : "memory");
    }
  }
}

// Staging slot of output element c of row ``ml`` of a warp (ml < 32) for the
// strided write-back: the warp's own rows of the A operand (its 4 row groups
// and its columns, in slices 0..3), which no other warp touches and which the
// finished products no longer need.  Element c of a row sits at c ^ (ml % DT),
// so the 8 lanes of one store phase hit 8 different 16-byte bank groups.
template <int K>
__device__ __forceinline__ uint8_t* out_slot(uint8_t* A, int wq, int sub, int ml, int c) {
  using S = TcShape<K>;
  const int q = ml * S::DT + (c ^ (ml % S::DT));
  const int chunk = q / S::RT, idx = q % S::RT;
  return A + (chunk >> 2) * S::A_SLICE + (4 * wq + (chunk & 3)) * S::SBO + sub * S::RT * 16 + idx * 16;
}

template <int K, bool LOW>
__global__ void __launch_bounds__(TcShape<K>::THREADS, 1)
    k_kgate_c128_tc(double2* __restrict__ a, uint64_t n_groups, const __grid_constant__ TcParams<K> P,
                    unsigned* flag) {
  using S = TcShape<K>;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem);
  const uint32_t mbar0 = tc::smem_u32(smem + 8);
  uint32_t* emx = reinterpret_cast<uint32_t*>(smem + S::EMX_OFF);  // [team][sub][m] partial group exponents
  uint8_t* Bs = smem + S::B_OFF;
  uint8_t* As = smem + S::A_OFF;
  const int tid = threadIdx.x, team = tid / S::TEAM_THREADS, sub = (tid / 128) % S::TPG, m = tid & 127;

  // W's digit slices (zero padding included) and row exponents; the A slices
  // zeroed once, so that their padding columns (k = 2: 8 reals padded to
  // K = 16) stay zero.
  for (int i = tid; i < (int)(S::B_BYTES / 16); i += blockDim.x) reinterpret_cast<uint4*>(Bs)[i] = make_uint4(0u, 0u, 0u, 0u);
  for (int i = tid; i < (int)(S::TEAMS * S::A_BYTES / 16); i += blockDim.x)
    reinterpret_cast<uint4*>(As)[i] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  for (int e = tid; e < S::R * S::R; e += blockDim.x) {
    const int o = e / S::R, i = e % S::R;
    double rem = ldexp(w_entry<K>(P, o, i), 8 - P.ro[o]);
    uint16_t* at = reinterpret_cast<uint16_t*>(Bs + (o / 8) * S::SBO + (i / 8) * 128 + (o % 8) * 16 + (i % 8) * 2);
#pragma unroll
    for (int j = 0; j < kSlices; ++j) {
      const double b = rint(rem);
      rem = (rem - b) * 512.0;
      at[j * (S::B_SLICE / 2)] = (uint16_t)(__float_as_uint(__double2float_rn(b) * digit_weight(j)) >> 16);
    }
  }
  if (tid == 0) {
    for (int w = 0; w < S::TEAMS; ++w) tc::mbar_init(mbar0 + 8 * w, 1);
    tc::mbar_init_fence();
  }
  tc::fence_async_smem();
  if (tid < 32) {
    tc::tmem_alloc(tc::smem_u32(tslot), 512);
    tc::tmem_relinquish();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = *tslot;

  uint8_t* A = As + team * S::A_BYTES;
  uint8_t* X = smem + S::X_OFF + team * S::X_BYTES;
  const uint32_t a_s = tc::smem_u32(A), b_s = tc::smem_u32(Bs);
  const uint32_t mbar = mbar0 + 8 * team;
  const uint32_t tacc = tbase + (uint32_t)(team * S::TCOLS);
  const uint32_t tlane = (uint32_t)(tid & 96) << 16;  // this warp's 32 TMEM lanes
  const int bar_id = 1 + team, c0 = sub * S::DT;
  const uint64_t n_tiles = (n_groups + kRows - 1) / kRows;
  const uint64_t stride = (uint64_t)gridDim.x * S::TEAMS;
  // row exponent range of W (the fast epilogue needs every output normal)
  int adj_lo = P.ro[0] - 1038, adj_hi = adj_lo;
#pragma unroll
  for (int o = 1; o < S::R; ++o) {
    adj_lo = min(adj_lo, P.ro[o] - 1038);
    adj_hi = max(adj_hi, P.ro[o] - 1038);
  }
  uint32_t phase = 0;
  unsigned bad = 0;
  bool stalled = false;
  uint64_t tile = (uint64_t)blockIdx.x * S::TEAMS + team;
  const int lane = tid & 31, wq = m >> 5, mw = m & 96;
  const uint64_t off_lane = LOW ? P.off[c0 + lane % S::DT] : 0;
  // the first tile's input; each later tile's is requested while this one is computed
  if constexpr (LOW) {
    if (tile < n_tiles) {
      const uint64_t g1 = tile * kRows + m;
      stage_warp<K>(X, mw, lane, c0, a, g1 < n_groups ? group_base<K>(g1, P) : 0, g1 < n_groups, off_lane);
    }
  } else if (tile < n_tiles && tile * kRows + m < n_groups) {
    stage_group<K>(X, m, c0, a, group_base<K>(tile * kRows + m, P), P);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  for (; tile < n_tiles; tile += stride) {
    const uint64_t g = tile * kRows + m;
    const bool act = g < n_groups;
    const uint64_t base = act ? group_base<K>(g, P) : 0;
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if constexpr (LOW) __syncwarp();  // the warp's copies landed in each other's rows
    uint32_t lo[S::RT], hi[S::RT];
#pragma unroll
    for (int c = 0; c < S::DT; ++c) {
      uint4 w = *reinterpret_cast<const uint4*>(X + ((size_t)(c0 + c) * kRows + m) * 16);
      if (!act) w = make_uint4(0u, 0u, 0u, 0u);
      lo[2 * c] = w.x;
      hi[2 * c] = w.y;
      lo[2 * c + 1] = w.z;
      hi[2 * c + 1] = w.w;
    }
    uint32_t emax = 0;
#pragma unroll
    for (int i = 0; i < S::RT; ++i) emax = max(emax, hi[i] & 0x7ff00000u);
    emax >>= 20;
    // the next tile's input goes into the same buffer: this thread's own
    // elements only, whose values are now in registers (emax used them all;
    // emax is at most 0x7ff, so its test below only orders the copies after
    // those reads)
    {
      const uint64_t gn = g + stride * kRows;
      if constexpr (LOW) {
        __syncwarp();  // every lane has read its rows before any lane refills them
        if (tile + stride < n_tiles)
          stage_warp<K>(X, mw, lane, c0, a, gn < n_groups ? group_base<K>(gn, P) : 0, gn < n_groups, off_lane);
      } else if (tile + stride < n_tiles && gn < n_groups && emax != 0x800u) {
        stage_group<K>(X, m, c0, a, group_base<K>(gn, P), P);
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
    if constexpr (S::TPG > 1) {  // the group's exponent from the team's partial ones
      emx[(team * S::TPG + sub) * 128 + m] = emax;
      tc::bar_sync(bar_id, S::TEAM_THREADS);
#pragma unroll
      for (int t = 0; t < S::TPG; ++t) emax = max(emax, emx[(team * S::TPG + t) * 128 + m]);
    }
    bad |= emax == 0x7ffu ? 1u : 0u;
#pragma unroll
    for (int ch = 0; ch < S::RT / 8; ++ch) {
      uint32_t pk[kSlices][4];
#pragma unroll
      for (int q = 0; q < 8; q += 2) {
        float d0[kSlices], d1[kSlices];
        digits(lo[8 * ch + q], hi[8 * ch + q], emax, d0);
        digits(lo[8 * ch + q + 1], hi[8 * ch + q + 1], emax, d1);
#pragma unroll
        for (int l = 0; l < kSlices; ++l) pk[l][q / 2] = pack_bf16(d0[l], d1[l]);
      }
      uint8_t* row = A + (m >> 3) * S::SBO + (sub * S::RT / 8 + ch) * 128 + (m & 7) * 16;
#pragma unroll
      for (int l = 0; l < kSlices; ++l)
        *reinterpret_cast<uint4*>(row + l * S::A_SLICE) = make_uint4(pk[l][0], pk[l][1], pk[l][2], pk[l][3]);
    }
    tc::fence_async_smem();
    tc::bar_sync(bar_id, S::TEAM_THREADS);
    if (sub == 0 && m == 0) {
      tc::fence_after();
      issue_mmas<K>(tacc, a_s, b_s);
      tc::commit(mbar);
    }
    // a group whose outputs all stay normal doubles (every group of a
    // state of ordinary scale) takes the fast epilogue; the warp decides
    const int e0 = (int)emax;
    const bool fast_ok = !act || emax == 0u || (e0 + adj_lo > -895 && e0 + adj_hi < 998);
    const bool fast = __all_sync(0xffffffffu, fast_ok);
    const bool ok = tc::mbar_wait(mbar, phase, kWaitPolls);
    phase ^= 1u;
    if (tc::bar_or(bar_id, S::TEAM_THREADS, !ok)) {
      stalled = true;
      break;
    }
    tc::fence_after();
#pragma unroll
    for (int ch = 0; ch < S::RT / 8; ++ch) {
      const int col = sub * S::RT + ch * 8;
      uint32_t v[kAcc][8];
#pragma unroll
      for (int acc = 0; acc < kAcc; ++acc) tc::tmem_ld8(tacc + tlane + (uint32_t)(acc * S::NP + col), v[acc]);
      tc::tmem_wait_ld();
      if (act || LOW) {
#pragma unroll
        for (int q = 0; q < 8; q += 2) {
          const int o = col + q;
          float s0, l0, s1, l1;
          combine(v, q, s0, l0);
          combine(v, q + 1, s1, l1);
          double2 y;
          if (fast) {
            y.x = join_scaled(s0, l0, e0 + P.ro[o] - 1038);
            y.y = join_scaled(s1, l1, e0 + P.ro[o + 1] - 1038);
          } else {
            y.x = scale_out(dfx::join(s0, l0), e0 + P.ro[o] - 1038, bad);
            y.y = scale_out(dfx::join(s1, l1), e0 + P.ro[o + 1] - 1038, bad);
          }
          if constexpr (LOW)
            *reinterpret_cast<double2*>(out_slot<K>(A, wq, sub, lane, ch * 4 + q / 2)) = y;
          else
            a[base + P.off[o / 2]] = y;
        }
      }
    }
    if constexpr (LOW) {  // write-back in element order, as the loads
      __syncwarp();
      const int cl = lane % S::DT;
#pragma unroll
      for (int j = 0; j < S::DT; ++j) {
        const int src = j * (32 / S::DT) + lane / S::DT;
        const uint64_t b = __shfl_sync(0xffffffffu, base, src);
        const int ok_src = __shfl_sync(0xffffffffu, (int)act, src);
        const double2 y = *reinterpret_cast<const double2*>(out_slot<K>(A, wq, sub, src, cl));
        if (ok_src) a[b + off_lane] = y;
      }
      __syncwarp();  // the slots are this warp's A rows again for the next tile
    }
    tc::fence_before();
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  if (stalled) {
    if (sub == 0 && m == 0) atomicOr(flag, 2u);
    tc::mbar_wait(mbar, phase ^ 1u, kWaitPolls);  // the products in flight, once more bounded
  }
  if (bad) atomicOr(flag, 1u);
  tc::fence_before();
  __syncthreads();
  if (tid < 32) {
    tc::fence_after();
    tc::tmem_dealloc(tbase, 512);
  }
}

template <int K>
void make_params(const int* qubits, const double* U, TcParams<K>& P) {
  using S = TcShape<K>;
  std::memset(&P, 0, sizeof(P));
  int pos[K];
  for (int j = 0; j < K; ++j) pos[j] = qubits[j];
  std::sort(pos, pos + K);
  for (int j = 0; j < K; ++j) P.pos[j] = pos[j];
  for (int c = 0; c < S::D; ++c) {
    uint64_t o = 0;
    for (int j = 0; j < K; ++j) o |= (uint64_t)((c >> j) & 1) << qubits[j];
    P.off[c] = o;
  }
  std::memcpy(P.u, U, sizeof(P.u));
  for (int o = 0; o < S::R; ++o) {  // row exponents (the digits themselves are formed on the device)
    const int r = o >> 1;
    double mx = 0.0;
    for (int c = 0; c < S::D; ++c) {
      const double ur = U[2 * (r * S::D + c)], ui = U[2 * (r * S::D + c) + 1];
      mx = std::max(mx, std::max(std::fabs(ur), std::fabs(ui)));  // W's rows 2r and 2r + 1 hold the same magnitudes
    }
    int ro = 0;
    if (mx > 0.0) std::frexp(mx, &ro);
    P.ro[o] = ro;
  }
}

template <int K>
cudaError_t launch_tc(iqs_reg* r, const int* qubits, const double* U) {
  using S = TcShape<K>;
  static TcParams<K> P;  // large (up to 16.6 KiB): kept off the host stack, filled under the lock below
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  make_params<K>(qubits, U, P);
  const size_t smem = std::max<size_t>(S::SMEM, 120 * 1024);  // > half an SM's shared memory: one CTA per SM
  bool low = false;
  for (int j = 0; j < K; ++j) low |= qubits[j] < 7;
  auto kern = low ? k_kgate_c128_tc<K, true> : k_kgate_c128_tc<K, false>;
  static PerDevice attr[2];
  int dummy = 0;
  cudaError_t e = attr[low ? 1 : 0].get(&dummy, [&](int* x) {
    *x = 1;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (e != cudaSuccess) return e;
  const uint64_t n_groups = num_amps(r) >> K;
  const uint64_t n_tiles = (n_groups + kRows - 1) / kRows;
  const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((n_tiles + S::TEAMS - 1) / S::TEAMS, kSMs));
  kern<<<grid, S::THREADS, smem, r->stream>>>((double2*)r->data, n_groups, P, r->flag);
  return launched(1);
}

}  // namespace

bool kq_tensor_supported(int k) { return k >= 2 && k <= 5; }

cudaError_t launch_kq_c128_tensor(iqs_reg* r, int k, const int* qubits, const double* U) {
  switch (k) {
    case 2: return launch_tc<2>(r, qubits, U);
    case 3: return launch_tc<3>(r, qubits, U);
    case 4: return launch_tc<4>(r, qubits, U);
    case 5: return launch_tc<5>(r, qubits, U);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace iqs
