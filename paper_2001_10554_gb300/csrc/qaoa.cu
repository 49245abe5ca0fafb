// QAOA Max-Cut engine: energy and adjoint gradient for a batch of B parameter
// sets on one graph, complex64 or complex128 (Section 4: L(theta) =
// <0|U^dagger H_MaxCut U|0> evaluated per particle; Section 2 "Pool of multiple
// states": many parameter sets of one circuit simulated side by side).
//
// States are stored as B contiguous vectors of 2^n amplitudes.  Every kernel
// takes the state index from blockIdx.y, so one launch advances all B states
// by one layer operation.
//
// Forward:  uniform |+>^n; per layer l the cost phase exp(-i gamma_l C) (a
//           per-state FP64-built table exp(-i gamma k) indexed by the
//           precomputed cut count C(x), one byte per basis state) and the
//           mixer RX(2 beta_l) on every qubit, applied in shared-memory tiles
//           of up to 12 qubits per pass.
// Energy:   E = sum C |psi|^2, accumulated in double-float, finished in FP64.
// Backward: adjoint by uncompute (no stored states): lambda = C psi, then for
//           l = p..1 the fused mixer step (accumulate Im<lambda|X_j|phi> for
//           every qubit and apply RX(2 beta)^dagger to both vectors) and the
//           fused phase step (accumulate Im<lambda|C|phi> and apply
//           exp(+i gamma C) to both); dE/dtheta = 2 Im <lambda|G|phi>.
//           Optional periodic renormalisation restores |phi| = 1 and |lambda|
//           to its initial value (both invariant under the exact uncompute).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <thread>
#include <new>
#include <tuple>
#include <type_traits>
#include <utility>
#include <vector>

#include "common.cuh"
#include "cut.cuh"
#include "df64.cuh"
#include "internal.h"
#include "qaoa_ops.cuh"
#include "tile.cuh"

#include <cuda.h>
#include <type_traits>

namespace iqs {
namespace {

using qops::S2;

constexpr int kMaxP = 64;

// ---------------------------------------------------------------- storage traits
struct T64 {
  using V = float2;   // HBM element
  using W = float2;   // working (shared-memory) element
  using RX = float2;  // (cos beta, sin beta)
  using PH = float2;  // exp(-i gamma k)
  static constexpr int kTileBits = 12;  // 4096 x 8 B = 32 KiB per vector
  static constexpr int kRowBits = 4;    // 16 contiguous amplitudes (128 B) per tile row
  static constexpr int kRegBits = 4;    // gates per register round (16 amplitudes per thread)
  static constexpr int kSwzBits = 4;    // 16 elements of 8 B per 128-byte smem row
  // Gradient terms of one register round (at most 32) are summed in FP32
  // before the double-float accumulation: their rounding (<= 32 * 2^-24 of the
  // terms) stays below the complex64 state's own error.
  static constexpr bool kBlockSum = true;
  static constexpr bool kTmaSwizzle = false;
  __device__ static W load(V v, unsigned&) { return v; }
  __device__ static V store(const W& w) { return w; }
  __device__ static RX rx_inv(RX k) { return make_float2(k.x, -k.y); }
  __device__ static void rx(W& a, W& b, const RX& k) { qops::rx_pair(a, b, k.x, k.y); }
  __device__ static PH conj(PH t) { return make_float2(t.x, -t.y); }
  __device__ static W mul(const PH& t, const W& x) { return qops::cmul(t, x); }
};

struct T128 {
  using V = double2;
  using W = S2;
  using RX = qops::RXc;
  using PH = qops::Ph;
  static constexpr int kTileBits = 11;  // 2048 x 16 B = 32 KiB per vector
  static constexpr int kRowBits = 3;    // 8 contiguous amplitudes (128 B) per tile row
  static constexpr int kRegBits = 3;    // gates per register round (8 amplitudes per thread)
  static constexpr int kSwzBits = 3;    // 8 elements of 16 B per 128-byte smem row
  static constexpr bool kBlockSum = false;  // every gradient term goes to the double-float accumulator
  static constexpr bool kTmaSwizzle = false;
  __device__ static W load(V v, unsigned& bad) { return qops::to_split(v, bad); }
  __device__ static V store(const W& w) { return qops::from_split(w); }
  __device__ static RX rx_inv(RX k) {
    RX r = k;
    r.s = k.ns;
    r.ns = k.s;
    return r;
  }
  __device__ static void rx(W& a, W& b, const RX& k) { qops::rx_pair(a, b, k); }
  __device__ static PH conj(PH t) {
    PH r = t;
    r.ti = t.nti;
    r.nti = t.ti;
    return r;
  }
  __device__ static W mul(const PH& t, const W& x) { return qops::cmul(t, x); }
};

// ---------------------------------------------------------------- kernels
template <class V>
__global__ void k_fill_uniform(V* a, uint64_t total, V v) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total; i += (uint64_t)gridDim.x * blockDim.x)
    a[i] = v;
}

template <class X>
__global__ void k_cut_table(uint8_t* cut, uint64_t N, EdgesU8 E) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x)
    cut[i] = (uint8_t)cut_count((X)i, E);
}

// Largest cut count of each graph (grid (blocks, n_graphs)); out[g] must be 0 on entry.
__global__ void k_cut_max(const uint8_t* __restrict__ cut, uint64_t N, unsigned* __restrict__ out) {
  const uint8_t* c = cut + (uint64_t)blockIdx.y * N;
  unsigned m = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x)
    m = max(m, (unsigned)c[i]);
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0) atomicMax(out + blockIdx.y, m);
}

// Mixer pass: RX on the qubits [s, s+m) of every tile (or its inverse, with the
// gradient term, on two vectors when ADJ).  The tile is staged in shared
// memory; the gate bits are processed in rounds of up to kRegBits bits, each
// thread holding the 2^kRegBits amplitudes of one register block and applying
// that round's gates in registers.
template <class TR, bool ADJ>
__global__ void __launch_bounds__(kThreads) k_mixer(typename TR::V* __restrict__ phi, typename TR::V* __restrict__ lam,
                                                    uint64_t N, Geo g, const typename TR::RX* __restrict__ rx,
                                                    double* __restrict__ partials, int part_stride, unsigned* flag) {
  using W = typename TR::W;
  constexpr int R = TR::kRegBits;
  constexpr int RB = 1 << R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  W* sp = reinterpret_cast<W*>(smem_raw);
  const unsigned K = g.c + g.m;
  const unsigned T = 1u << K;
  W* sl = sp + T;
  const unsigned b = blockIdx.y;
  typename TR::V* P = phi + (uint64_t)b * N;
  typename TR::V* L = ADJ ? lam + (uint64_t)b * N : nullptr;
  const typename TR::RX k = ADJ ? TR::rx_inv(rx[b]) : rx[b];
  const uint64_t tiles = N >> K;
  unsigned bad = 0;
  dfx::Acc acc;
  for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    for (unsigned l = threadIdx.x; l < T; l += blockDim.x) {
      const uint64_t x = tile_x(g, t, l);
      sp[swz<TR>(l)] = TR::load(P[x], bad);
      if (ADJ) sl[swz<TR>(l)] = TR::load(L[x], bad);
    }
    __syncthreads();
    for (int pos = g.c; pos < (int)K; pos += R) {
      const int gb = min(R, (int)K - pos);
      const unsigned nsub = T >> gb;
      for (unsigned sb = threadIdx.x; sb < nsub; sb += blockDim.x) {
        const unsigned base = ((sb >> pos) << (pos + gb)) | (sb & ((1u << pos) - 1u));
        W a[RB];
        W y[ADJ ? RB : 1];
#pragma unroll
        for (int j = 0; j < RB; ++j) {
          if (j < (1 << gb)) {
            const unsigned idx = swz<TR>(base | ((unsigned)j << pos));
            a[j] = sp[idx];
            if (ADJ) y[j] = sl[idx];
          }
        }
        float rsum = 0.f;  // FP32 block sum of this round's gradient terms (complex64)
#pragma unroll
        for (int bit = 0; bit < R; ++bit) {
          if (bit < gb) {
#pragma unroll
            for (int j = 0; j < RB; ++j) {
              if (!(j & (1 << bit)) && j < (1 << gb)) {
                const int j1 = j | (1 << bit);
                if (ADJ) {
                  if constexpr (TR::kBlockSum) {
                    rsum = qops::im_conj_mul_fma(y[j], a[j1], rsum);
                    rsum = qops::im_conj_mul_fma(y[j1], a[j], rsum);
                  } else {
                    float p, e;
                    qops::im_conj_mul(y[j], a[j1], p, e);
                    acc.add(p, e);
                    qops::im_conj_mul(y[j1], a[j], p, e);
                    acc.add(p, e);
                  }
                  TR::rx(y[j], y[j1], k);
                }
                TR::rx(a[j], a[j1], k);
              }
            }
          }
        }
        if (ADJ && TR::kBlockSum) acc.add(rsum, 0.f);
#pragma unroll
        for (int j = 0; j < RB; ++j) {
          if (j < (1 << gb)) {
            const unsigned idx = swz<TR>(base | ((unsigned)j << pos));
            sp[idx] = a[j];
            if (ADJ) sl[idx] = y[j];
          }
        }
      }
      __syncthreads();
    }
    for (unsigned l = threadIdx.x; l < T; l += blockDim.x) {
      const uint64_t x = tile_x(g, t, l);
      P[x] = TR::store(sp[swz<TR>(l)]);
      if (ADJ) L[x] = TR::store(sl[swz<TR>(l)]);
    }
    __syncthreads();
  }
  if (bad) atomicOr(flag, 1u);
  if (ADJ) block_partial(acc.value(), partials + (uint64_t)b * part_stride + blockIdx.x);
}

// The same pass for the two common tile shapes with everything but the tile
// placement known at compile time: C row bits, then M gate bits, K = C + M =
// kTileBits.  C = 0 is the low pass (tile = 2^K contiguous amplitudes); C > 0
// is a high pass whose gate bits start at s.  Since swz() is linear over
// GF(2), the shared-memory index of (base | j << POS) is swz(base) ^ swz(j << POS),
// one XOR with a compile-time constant per element.
// The gates of one register round on a register block of 2^GB amplitudes
// (element j differs from element 0 in the round's bits by j), with the
// adjoint pass's gradient terms: complex64 sums a round's terms in FP32 before
// the double-float accumulator, complex128 adds every term to it.
template <class TR, bool ADJ, int GB>
__device__ __forceinline__ void round_in_regs(typename TR::W* a, typename TR::W* y, const typename TR::RX& k,
                                              dfx::Acc& acc) {
  constexpr int RB = 1 << GB;
  float rsum = 0.f;
#pragma unroll
  for (int bit = 0; bit < GB; ++bit) {
#pragma unroll
    for (int j = 0; j < RB; ++j) {
      if (!(j & (1 << bit))) {
        const int j1 = j | (1 << bit);
        if (ADJ) {
          if constexpr (TR::kBlockSum) {
            rsum = qops::im_conj_mul_fma(y[j], a[j1], rsum);
            rsum = qops::im_conj_mul_fma(y[j1], a[j], rsum);
          } else {
            float p, e;
            qops::im_conj_mul(y[j], a[j1], p, e);
            acc.add(p, e);
            qops::im_conj_mul(y[j1], a[j], p, e);
            acc.add(p, e);
          }
          TR::rx(y[j], y[j1], k);
        }
        TR::rx(a[j], a[j1], k);
      }
    }
  }
  if (ADJ && TR::kBlockSum) acc.add(rsum, 0.f);
}

// First element of register block sb in a round whose gate bits start at POS.
template <int POS, int GB>
__device__ __forceinline__ unsigned block_base(unsigned sb) {
  return ((sb >> POS) << (POS + GB)) | (sb & ((1u << POS) - 1u));
}

template <class TR, bool ADJ, int C, int POS, int GB>
__device__ __forceinline__ void mixer_round(typename TR::W* sp, typename TR::W* sl, const typename TR::RX& k,
                                            float& rsum_out, dfx::Acc& acc) {
  using W = typename TR::W;
  constexpr int K = TR::kTileBits;
  constexpr unsigned NSUB = 1u << (K - GB);
  constexpr int RB = 1 << GB;
  for (unsigned sb = threadIdx.x; sb < NSUB; sb += blockDim.x) {
    const unsigned sbase = swz<TR>(block_base<POS, GB>(sb));
    W a[RB];
    W y[ADJ ? RB : 1];
#pragma unroll
    for (int j = 0; j < RB; ++j) {
      const unsigned idx = sbase ^ swz<TR>((unsigned)j << POS);
      a[j] = sp[idx];
      if (ADJ) y[j] = sl[idx];
    }
    round_in_regs<TR, ADJ, GB>(a, y, k, acc);
#pragma unroll
    for (int j = 0; j < RB; ++j) {
      const unsigned idx = sbase ^ swz<TR>((unsigned)j << POS);
      sp[idx] = a[j];
      if (ADJ) sl[idx] = y[j];
    }
  }
  (void)rsum_out;
}

// Register rounds in shared memory for the gate bits [POS, END), each followed
// by a block barrier.
template <class TR, bool ADJ, int C, int POS, int END>
__device__ __forceinline__ void mixer_rounds_to(typename TR::W* sp, typename TR::W* sl, const typename TR::RX& k,
                                                dfx::Acc& acc) {
  if constexpr (POS < END) {
    constexpr int GB = (TR::kTileBits - POS) < TR::kRegBits ? (TR::kTileBits - POS) : TR::kRegBits;
    float dummy = 0.f;
    mixer_round<TR, ADJ, C, POS, GB>(sp, sl, k, dummy, acc);
    __syncthreads();
    mixer_rounds_to<TR, ADJ, C, POS + GB, END>(sp, sl, k, acc);
  }
}

template <class TR, bool ADJ, int C, int POS>
__device__ __forceinline__ void mixer_rounds(typename TR::W* sp, typename TR::W* sl, const typename TR::RX& k,
                                             dfx::Acc& acc) {
  mixer_rounds_to<TR, ADJ, C, POS, TR::kTileBits>(sp, sl, k, acc);
}

// Global index of tile element l: C = 0 tiles are 2^K contiguous amplitudes,
// C > 0 tiles are rows of 2^C contiguous amplitudes, 2^s apart.
template <int C>
__device__ __forceinline__ uint64_t fast_x(uint64_t tbase, unsigned l, int s) {
  if constexpr (C == 0)
    return tbase + l;
  else
    return tbase + ((uint64_t)(l >> C) << s) + (l & ((1u << C) - 1u));
}

// Renormalisation fused into the adjoint passes (complex64 only).  With
// ``norms`` set, a pass scales phi and lambda by sqrt(target / norm) as it loads
// them; ``norms`` holds [4][stride] values: current |phi|^2, lambda target,
// phi target, current |lambda|^2.  With ``partials`` set, the fused-phase pass
// (PH = 2) sums |phi|^2 and |lambda|^2 of the values it stores, per block, in
// FP64-equivalent arithmetic, to partials[b][x] and partials[b][kRnCol + x].
struct RenormFuse {
  const double* norms = nullptr;
  int stride = 0;
  double* partials = nullptr;
};
constexpr int kRnCol = 2432;

// The pass with every register round in shared memory, a staged load before
// and a staged store after; used for the fused-phase adjoint pass (PH = 2).
// PH = 2: after the mixer uncompute, each amplitude contributes
// C(x) Im(conj(lambda) phi) to the phase gradient (partials_g), and both
// vectors are multiplied by conj(T_b[C(x)]) as they are stored, which saves
// a full pass per layer.
template <class TR, bool ADJ, int C, int PH>
__device__ __forceinline__ void mixer_fast_body_staged(typename TR::V* __restrict__ phi,
                                                         typename TR::V* __restrict__ lam, uint64_t N, int s_bits,
                                                         const typename TR::RX* __restrict__ rx,
                                                         double* __restrict__ partials, int part_stride, unsigned* flag,
                                                         const uint8_t* __restrict__ cut,
                                                         const typename TR::PH* __restrict__ tables, int tsize,
                                                         double* __restrict__ partials_g, int per_graph,
                                                         const RenormFuse rn) {
  using W = typename TR::W;
  using PHT = typename TR::PH;
  constexpr bool kRn = ADJ && TR::kBlockSum;  // fused renormalisation: complex64 adjoint passes
  __shared__ PHT st[PH ? kEdgeChunk + 1 : 1];
  __shared__ float rn_f[2];
  bool scale_in = false;
  float f_phi = 1.f, f_lam = 1.f;
  if constexpr (kRn) {
    if (rn.norms) {
      if (threadIdx.x == 0) {
        const unsigned b = blockIdx.y;
        const double np = rn.norms[b], tl = rn.norms[rn.stride + b];
        const double tp = rn.norms[2 * rn.stride + b], nl = rn.norms[3 * rn.stride + b];
        rn_f[0] = (float)(np > 0.0 ? sqrt(tp / np) : 1.0);
        rn_f[1] = (float)(nl > 0.0 ? sqrt(tl / nl) : 1.0);
      }
      __syncthreads();
      scale_in = true;
      f_phi = rn_f[0];
      f_lam = rn_f[1];
    }
  }
  if (PH) {
    cut += (uint64_t)(blockIdx.y / (unsigned)per_graph) * N;  // state b uses graph b / per_graph
    for (int i = threadIdx.x; i < tsize; i += blockDim.x) {
      const PHT tt = tables[(uint64_t)blockIdx.y * tsize + i];
      st[i] = PH == 2 ? TR::conj(tt) : tt;
    }
    __syncthreads();
  }
  constexpr int K = TR::kTileBits;
  constexpr int M = K - C;
  constexpr unsigned T = 1u << K;
  constexpr unsigned PER = T / kThreads;  // elements per thread in the load/store phases
  extern __shared__ __align__(16) unsigned char smem_raw[];
  W* sp = reinterpret_cast<W*>(smem_raw);
  W* sl = sp + T;
  const unsigned b = blockIdx.y;
  typename TR::V* P = phi + (uint64_t)b * N;
  typename TR::V* L = ADJ ? lam + (uint64_t)b * N : nullptr;
  const typename TR::RX k = ADJ ? TR::rx_inv(rx[b]) : rx[b];
  const uint64_t tiles = N >> K;
  const unsigned tid = threadIdx.x;
  // element l = tid + kThreads * i sits at (l >> C) << s | (l & (2^C - 1)) inside the tile
  // footprint; for C <= 8 that is off0 + i * step (kThreads = 2^8 carries no bit into the row).
  const int s = C == 0 ? 0 : s_bits;
  const uint64_t off0 = C == 0 ? tid : ((uint64_t)(tid >> C) << s) | (tid & ((1u << C) - 1u));
  const uint64_t step = C == 0 ? kThreads : ((uint64_t)(kThreads >> (C <= 8 ? C : 8)) << s);
  const unsigned sw0 = swz<TR>(tid);
  const int mid = s - C;
  unsigned bad = 0;
  dfx::Acc acc, accg;
  // fused renormalisation: this thread's running |phi|^2 and |lambda|^2, kept in
  // shared memory between tiles so that they hold no registers across the rounds
  __shared__ dfx::Acc rn_acc[kRn && PH == 2 ? 2 * kThreads : 1];
  const bool norm_out = kRn && PH == 2 && rn.partials != nullptr;
  if constexpr (kRn && PH == 2) {
    rn_acc[tid] = dfx::Acc();
    rn_acc[kThreads + tid] = dfx::Acc();
  }
  for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const uint64_t tbase = C == 0 ? (t << K) : (((t >> mid) << (s + M)) | ((t & ((1ull << mid) - 1ull)) << C));
#pragma unroll
    for (unsigned i = 0; i < PER; ++i) {
      const unsigned l = tid + kThreads * i;
      const uint64_t x = C <= 8 ? tbase + off0 + step * i : tbase + (((uint64_t)(l >> C)) << s) + (l & ((1u << C) - 1u));
      const unsigned idx = sw0 ^ swz<TR>(kThreads * i);
      if (PH == 1) {
        sp[idx] = TR::mul(st[cut[x]], TR::load(P[x], bad));
      } else {
        W w = TR::load(P[x], bad);
        if constexpr (kRn) {
          if (scale_in) w = qops::scale_int(w, f_phi);
        }
        sp[idx] = w;
      }
      if (ADJ) {
        W w = TR::load(L[x], bad);
        if constexpr (kRn) {
          if (scale_in) w = qops::scale_int(w, f_lam);
        }
        sl[idx] = w;
      }
    }
    __syncthreads();
    mixer_rounds<TR, ADJ, C, C>(sp, sl, k, acc);
    float gsum = 0.f;
    dfx::Acc acc_np, acc_nl;
    if constexpr (kRn && PH == 2) {
      if (norm_out) {
        acc_np = rn_acc[tid];
        acc_nl = rn_acc[kThreads + tid];
      }
    }
#pragma unroll
    for (unsigned i = 0; i < PER; ++i) {
      const unsigned l = tid + kThreads * i;
      const uint64_t x = C <= 8 ? tbase + off0 + step * i : tbase + (((uint64_t)(l >> C)) << s) + (l & ((1u << C) - 1u));
      const unsigned idx = sw0 ^ swz<TR>(kThreads * i);
      if (PH == 2) {
        const int c = cut[x];
        const W xv = sp[idx], yv = sl[idx];
        const float cf = (float)c;
        if constexpr (TR::kBlockSum) {
          gsum = fmaf(cf, qops::im_conj_mul_fma(yv, xv, 0.f), gsum);
        } else {
          float pp, ee;
          qops::im_conj_mul(yv, xv, pp, ee);
          const float qq = cf * pp;
          accg.add(qq, fmaf(cf, pp, -qq) + cf * ee);
        }
        const W xo = TR::mul(st[c], xv), yo = TR::mul(st[c], yv);
        if constexpr (kRn) {
          if (norm_out) {
            float pp, ee;
            qops::abs2(xo, pp, ee);
            acc_np.add(pp, ee);
            qops::abs2(yo, pp, ee);
            acc_nl.add(pp, ee);
          }
        }
        P[x] = TR::store(xo);
        L[x] = TR::store(yo);
      } else {
        P[x] = TR::store(sp[idx]);
        if (ADJ) L[x] = TR::store(sl[idx]);
      }
    }
    if (PH == 2 && TR::kBlockSum) accg.add(gsum, 0.f);
    if constexpr (kRn && PH == 2) {
      if (norm_out) {
        rn_acc[tid] = acc_np;
        rn_acc[kThreads + tid] = acc_nl;
      }
    }
    __syncthreads();
  }
  if (bad) atomicOr(flag, 1u);
  if (ADJ) block_partial(acc.value(), partials + (uint64_t)b * part_stride + blockIdx.x);
  if (PH == 2) block_partial(accg.value(), partials_g + (uint64_t)b * part_stride + blockIdx.x);
  if constexpr (kRn && PH == 2) {
    if (norm_out) {
      block_partial(rn_acc[tid].value(), rn.partials + (uint64_t)b * part_stride + blockIdx.x);
      block_partial(rn_acc[kThreads + tid].value(), rn.partials + (uint64_t)b * part_stride + kRnCol + blockIdx.x);
    }
  }
}


// A mixer pass of a full tile shape, forward or adjoint.  PH = 1 (forward, low
// pass): the layer's cost phase T_b[C(x)] is applied to each amplitude as the
// tile is loaded, which saves a full pass per layer.  (PH = 2, the adjoint
// pass with the fused phase epilogue, is mixer_fast_body_staged.)
template <class TR, bool ADJ, int C, int PH>
__device__ __forceinline__ void mixer_fast_body(typename TR::V* __restrict__ phi,
                                                         typename TR::V* __restrict__ lam, uint64_t N, int s_bits,
                                                         const typename TR::RX* __restrict__ rx,
                                                         double* __restrict__ partials, int part_stride, unsigned* flag,
                                                         const uint8_t* __restrict__ cut,
                                                         const typename TR::PH* __restrict__ tables, int tsize,
                                                         double* __restrict__ partials_g, int per_graph,
                                                         const RenormFuse rn) {
  using W = typename TR::W;
  using PHT = typename TR::PH;
  constexpr bool kRn = ADJ && TR::kBlockSum;  // fused renormalisation: complex64 adjoint passes
  __shared__ PHT st[PH ? kEdgeChunk + 1 : 1];
  __shared__ float rn_f[2];
  bool scale_in = false;
  float f_phi = 1.f, f_lam = 1.f;
  if constexpr (kRn) {
    if (rn.norms) {
      if (threadIdx.x == 0) {
        const unsigned b = blockIdx.y;
        const double np = rn.norms[b], tl = rn.norms[rn.stride + b];
        const double tp = rn.norms[2 * rn.stride + b], nl = rn.norms[3 * rn.stride + b];
        rn_f[0] = (float)(np > 0.0 ? sqrt(tp / np) : 1.0);
        rn_f[1] = (float)(nl > 0.0 ? sqrt(tl / nl) : 1.0);
      }
      __syncthreads();
      scale_in = true;
      f_phi = rn_f[0];
      f_lam = rn_f[1];
    }
  }
  if (PH) {
    cut += (uint64_t)(blockIdx.y / (unsigned)per_graph) * N;  // state b uses graph b / per_graph
    for (int i = threadIdx.x; i < tsize; i += blockDim.x) {
      const PHT tt = tables[(uint64_t)blockIdx.y * tsize + i];
      st[i] = PH == 2 ? TR::conj(tt) : tt;
    }
    __syncthreads();
  }
  constexpr int K = TR::kTileBits;
  constexpr int M = K - C;
  constexpr unsigned T = 1u << K;
  constexpr unsigned PER = T / kThreads;  // elements per thread in a staged load or store
  extern __shared__ __align__(16) unsigned char smem_raw[];
  W* sp = reinterpret_cast<W*>(smem_raw);
  W* sl = sp + T;
  const unsigned b = blockIdx.y;
  typename TR::V* P = phi + (uint64_t)b * N;
  typename TR::V* L = ADJ ? lam + (uint64_t)b * N : nullptr;
  const typename TR::RX k = ADJ ? TR::rx_inv(rx[b]) : rx[b];
  const uint64_t tiles = N >> K;
  const unsigned tid = threadIdx.x;
  const int s = C == 0 ? 0 : s_bits;
  const int mid = s - C;
  // staged element l = tid + kThreads * i sits at fast_x(l); for C <= 8 that is
  // tbase + off0 + i * step (kThreads = 2^8 carries no bit into the row)
  const uint64_t off0 = C == 0 ? tid : ((uint64_t)(tid >> C) << s) | (tid & ((1u << C) - 1u));
  const uint64_t step = C == 0 ? kThreads : ((uint64_t)(kThreads >> (C <= 8 ? C : 8)) << s);
  // Register rounds of the pass: NR rounds of up to kRegBits gate bits.  The
  // last round, from bit POSL, writes its results straight to HBM, and high
  // passes (C > 0) also load their first round straight from HBM (a warp's
  // register blocks cover whole 2^C-amplitude rows, so the loads stay
  // coalesced); the low pass stages its tile through coalesced loads first.
  // That halves the shared-memory sweeps of a tile: the passes ran 10-13%
  // faster than with every round in shared memory.  The fused-phase adjoint
  // pass (PH = 2) runs mixer_fast_body_staged instead: with its epilogue in
  // the last round it ran up to 45% slower.
  static_assert(PH != 2, "fused-phase adjoint passes use mixer_fast_body_staged");
  constexpr int R = TR::kRegBits;
  constexpr int NR = (M + R - 1) / R;
  constexpr int POSL = C + R * (NR - 1);
  constexpr int GBL = K - POSL;
  constexpr int GB0 = M < R ? M : R;
  constexpr bool kDirect = C > 0;
  unsigned bad = 0;
  dfx::Acc acc;
  // one register block of 2^G amplitudes (gate bits from POS) to HBM
  auto store_block = [&](const W* a, const W* y, unsigned base, uint64_t tbase, auto pos_c, auto gb_c) {
    constexpr int POS = decltype(pos_c)::value;
    constexpr int G = decltype(gb_c)::value;
#pragma unroll
    for (int j = 0; j < (1 << G); ++j) {
      const uint64_t x = fast_x<C>(tbase, base | ((unsigned)j << POS), s);
      P[x] = TR::store(a[j]);
      if (ADJ) L[x] = TR::store(y[j]);
    }
  };
  // load one amplitude of each vector from HBM, with the fused phase (PH = 1)
  // or renormalisation factors applied
  auto load_amp = [&](uint64_t x, W& av, W& yv) {
    if (PH == 1) {
      av = TR::mul(st[cut[x]], TR::load(P[x], bad));
    } else {
      av = TR::load(P[x], bad);
      if constexpr (kRn) {
        if (scale_in) av = qops::scale_int(av, f_phi);
      }
    }
    if (ADJ) {
      yv = TR::load(L[x], bad);
      if constexpr (kRn) {
        if (scale_in) yv = qops::scale_int(yv, f_lam);
      }
    }
  };
  for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const uint64_t tbase = C == 0 ? (t << K) : (((t >> mid) << (s + M)) | ((t & ((1ull << mid) - 1ull)) << C));
    if constexpr (!kDirect) {
      // staged load: element l = tid + kThreads * i, coalesced across the warp
#pragma unroll
      for (unsigned i = 0; i < PER; ++i) {
        const unsigned l = tid + kThreads * i;
        const unsigned idx = swz<TR>(l);
        W av, yv;
        load_amp(C <= 8 ? tbase + off0 + step * i : fast_x<C>(tbase, l, s), av, yv);
        sp[idx] = av;
        if (ADJ) sl[idx] = yv;
      }
      __syncthreads();
      mixer_rounds_to<TR, ADJ, C, C, POSL>(sp, sl, k, acc);
    } else {
      constexpr unsigned NSUB0 = 1u << (K - GB0);
      for (unsigned sb = tid; sb < NSUB0; sb += kThreads) {
        const unsigned base = block_base<C, GB0>(sb);
        W a[1 << GB0];
        W y[ADJ ? (1 << GB0) : 1];
#pragma unroll
        for (int j = 0; j < (1 << GB0); ++j) {
          W yv;
          load_amp(fast_x<C>(tbase, base | ((unsigned)j << C), s), a[j], yv);
          if (ADJ) y[ADJ ? j : 0] = yv;
        }
        round_in_regs<TR, ADJ, GB0>(a, y, k, acc);
        if constexpr (NR == 1) {
          store_block(a, y, base, tbase, std::integral_constant<int, C>(), std::integral_constant<int, GB0>());
        } else {
          const unsigned sbase = swz<TR>(base);
#pragma unroll
          for (int j = 0; j < (1 << GB0); ++j) {
            const unsigned idx = sbase ^ swz<TR>((unsigned)j << C);
            sp[idx] = a[j];
            if (ADJ) sl[idx] = y[ADJ ? j : 0];
          }
        }
      }
      if constexpr (NR > 1) {
        __syncthreads();
        mixer_rounds_to<TR, ADJ, C, C + GB0, POSL>(sp, sl, k, acc);
      }
    }
    if constexpr (!kDirect || NR > 1) {
      // last round: shared memory -> registers -> HBM
      constexpr unsigned NSUBL = 1u << (K - GBL);
      for (unsigned sb = tid; sb < NSUBL; sb += kThreads) {
        const unsigned base = block_base<POSL, GBL>(sb);
        const unsigned sbase = swz<TR>(base);
        W a[1 << GBL];
        W y[ADJ ? (1 << GBL) : 1];
#pragma unroll
        for (int j = 0; j < (1 << GBL); ++j) {
          const unsigned idx = sbase ^ swz<TR>((unsigned)j << POSL);
          a[j] = sp[idx];
          if (ADJ) y[ADJ ? j : 0] = sl[idx];
        }
        round_in_regs<TR, ADJ, GBL>(a, y, k, acc);
        store_block(a, y, base, tbase, std::integral_constant<int, POSL>(), std::integral_constant<int, GBL>());
      }
      __syncthreads();  // the next tile reuses shared memory
    }
  }
  if (bad) atomicOr(flag, 1u);
  if (ADJ) block_partial(acc.value(), partials + (uint64_t)b * part_stride + blockIdx.x);
}

// The shape-specialised pass kernels.  The adjoint ones are held to 128
// registers (two 256-thread blocks per SM); the forward ones are left to the
// compiler's default, which keeps them near 80-100.
#define IQS_MIXER_FAST_PARAMS                                                                                    \
  typename TR::V *__restrict__ phi, typename TR::V *__restrict__ lam, uint64_t N, int s_bits,                    \
      const typename TR::RX *__restrict__ rx, double *__restrict__ partials, int part_stride, unsigned *flag,    \
      const uint8_t *__restrict__ cut, const typename TR::PH *__restrict__ tables, int tsize,                    \
      double *__restrict__ partials_g, int per_graph, const RenormFuse rn
#define IQS_MIXER_FAST_ARGS \
  phi, lam, N, s_bits, rx, partials, part_stride, flag, cut, tables, tsize, partials_g, per_graph, rn
template <class TR, int C, int PH>
__global__ void __launch_bounds__(kThreads) k_mixer_fast_fwd(IQS_MIXER_FAST_PARAMS) {
  mixer_fast_body<TR, false, C, PH>(IQS_MIXER_FAST_ARGS);
}
template <class TR, int C, int PH>
__global__ void __launch_bounds__(kThreads, 2) k_mixer_fast_adj(IQS_MIXER_FAST_PARAMS) {
  if constexpr (PH == 2)
    mixer_fast_body_staged<TR, true, C, PH>(IQS_MIXER_FAST_ARGS);
  else
    mixer_fast_body<TR, true, C, PH>(IQS_MIXER_FAST_ARGS);
}
#undef IQS_MIXER_FAST_PARAMS
#undef IQS_MIXER_FAST_ARGS

template <class TR, bool ADJ, int C, int PH>
constexpr auto k_mixer_fast() {
  if constexpr (ADJ)
    return k_mixer_fast_adj<TR, C, PH>;
  else
    return k_mixer_fast_fwd<TR, C, PH>;
}

// Tiles of the chained schedule that hold a layer boundary or the turnaround,
// with the load and store scheme of mixer_fast_body (a high pass loads its
// first round straight from HBM, the low pass stages its tile; the last round
// writes straight to HBM):
//   MODE kMgMerged: layer A's RX^dagger on the tile's bits (gradient sums to
//     out.pA), layer A's adjoint phase (its gradient term C Im(conj(lambda)
//     phi) to out.pG, then conj(T[C]) on both vectors), layer B's RX^dagger on
//     the same bits (out.pB); phi and lambda stored.  complex64 may rescale on
//     load and sum the stored norms (fused renormalisation, out.rn).
//   MODE kMgLast: layer A's RX^dagger and the phase-gradient term only;
//     nothing is stored (the last adjoint segment).
//   MODE kMgTurn: phi only is loaded; layer A's RX on the tile's bits, then
//     the turnaround (E to out.pE, |phi|^2 to out.pN, |lambda|^2 to out.pL,
//     lambda = C phi), then RX^dagger of the same layer on both vectors (out.pB);
//     only lambda is stored: phi equals the tile's input up to rounding.
enum { kMgMerged = 0, kMgLast = 1, kMgTurn = 2 };

struct MergedOut {
  double* pA = nullptr;
  double* pB = nullptr;
  double* pG = nullptr;
  double* pE = nullptr;
  double* pN = nullptr;
  double* pL = nullptr;
  double* pRnP = nullptr;  // |phi|^2 and |lambda|^2 of the stored values (fused renormalisation), or NULL
  double* pRnL = nullptr;
  RenormFuse rn;           // rn.norms: rescale on load
};

template <class TR, int C, int MODE>
__global__ void __launch_bounds__(kThreads, 2)
    k_mixer_merged(typename TR::V* __restrict__ phi, typename TR::V* __restrict__ lam, uint64_t N, int s_bits,
                   const typename TR::RX* __restrict__ rxA, const typename TR::RX* __restrict__ rxB,
                   int part_stride, unsigned* flag, const uint8_t* __restrict__ cut,
                   const typename TR::PH* __restrict__ tables, int tsize, int per_graph, const MergedOut out) {
  using W = typename TR::W;
  using PHT = typename TR::PH;
  constexpr bool kRn = MODE == kMgMerged && TR::kBlockSum;
  constexpr bool ADJA = MODE != kMgTurn;  // layer A's rounds work on both vectors
  __shared__ PHT st[MODE == kMgTurn ? 1 : kEdgeChunk + 1];
  __shared__ float rn_f[2];
  cut += (uint64_t)(blockIdx.y / (unsigned)per_graph) * N;  // state b uses graph b / per_graph
  if constexpr (MODE != kMgTurn)
    for (int i = threadIdx.x; i < tsize; i += blockDim.x) st[i] = TR::conj(tables[(uint64_t)blockIdx.y * tsize + i]);
  bool scale_in = false;
  if constexpr (kRn) {
    if (out.rn.norms) {
      if (threadIdx.x == 0) {
        const unsigned b = blockIdx.y;
        const double np = out.rn.norms[b], tl = out.rn.norms[out.rn.stride + b];
        const double tp = out.rn.norms[2 * out.rn.stride + b], nl = out.rn.norms[3 * out.rn.stride + b];
        rn_f[0] = (float)(np > 0.0 ? sqrt(tp / np) : 1.0);
        rn_f[1] = (float)(nl > 0.0 ? sqrt(tl / nl) : 1.0);
      }
      scale_in = true;
    }
  }
  __syncthreads();
  const float f_phi = kRn && scale_in ? rn_f[0] : 1.f, f_lam = kRn && scale_in ? rn_f[1] : 1.f;
  const bool norm_out = kRn && out.pRnP != nullptr;
  constexpr int K = TR::kTileBits;
  constexpr int M = K - C;
  constexpr unsigned T = 1u << K;
  constexpr unsigned PER = T / kThreads;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  W* sp = reinterpret_cast<W*>(smem_raw);
  W* sl = sp + T;
  const unsigned b = blockIdx.y;
  typename TR::V* P = phi + (uint64_t)b * N;
  typename TR::V* L = lam + (uint64_t)b * N;
  const typename TR::RX kA = ADJA ? TR::rx_inv(rxA[b]) : rxA[b];
  const typename TR::RX kB = MODE == kMgTurn ? TR::rx_inv(rxA[b]) : (MODE == kMgMerged ? TR::rx_inv(rxB[b]) : kA);
  const uint64_t tiles = N >> K;
  const unsigned tid = threadIdx.x;
  const int s = C == 0 ? 0 : s_bits;
  const int mid = s - C;
  const uint64_t off0 = C == 0 ? tid : ((uint64_t)(tid >> C) << s) | (tid & ((1u << C) - 1u));
  const uint64_t step = C == 0 ? kThreads : ((uint64_t)(kThreads >> (C <= 8 ? C : 8)) << s);
  constexpr int R = TR::kRegBits;
  constexpr int NR = (M + R - 1) / R;
  constexpr int POSL = C + R * (NR - 1);
  constexpr int GBL = K - POSL;
  constexpr int GB0 = M < R ? M : R;
  constexpr bool kDirect = C > 0;
  unsigned bad = 0;
  dfx::Acc accA, accB, accg, acce, accn, accl, rnp, rnl;
  auto load_amp = [&](uint64_t x, W& av, W& yv) {
    av = TR::load(P[x], bad);
    if constexpr (kRn) {
      if (scale_in) av = qops::scale_int(av, f_phi);
    }
    if constexpr (ADJA) {
      yv = TR::load(L[x], bad);
      if constexpr (kRn) {
        if (scale_in) yv = qops::scale_int(yv, f_lam);
      }
    }
  };
  for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const uint64_t tbase = C == 0 ? (t << K) : (((t >> mid) << (s + M)) | ((t & ((1ull << mid) - 1ull)) << C));
    // layer A: every round, the first one from HBM (high pass) or from a staged tile (low pass)
    if constexpr (!kDirect) {
#pragma unroll
      for (unsigned i = 0; i < PER; ++i) {
        const unsigned l = tid + kThreads * i;
        W av, yv;
        load_amp(C <= 8 ? tbase + off0 + step * i : fast_x<C>(tbase, l, s), av, yv);
        sp[swz<TR>(l)] = av;
        if (ADJA) sl[swz<TR>(l)] = yv;
      }
      __syncthreads();
      mixer_rounds_to<TR, ADJA, C, C, K>(sp, sl, kA, accA);
    } else {
      constexpr unsigned NSUB0 = 1u << (K - GB0);
      for (unsigned sb = tid; sb < NSUB0; sb += kThreads) {
        const unsigned base = block_base<C, GB0>(sb);
        W a[1 << GB0], y[ADJA ? (1 << GB0) : 1];
#pragma unroll
        for (int j = 0; j < (1 << GB0); ++j) {
          W yv;
          load_amp(fast_x<C>(tbase, base | ((unsigned)j << C), s), a[j], yv);
          if (ADJA) y[ADJA ? j : 0] = yv;
        }
        round_in_regs<TR, ADJA, GB0>(a, y, kA, accA);
        const unsigned sbase = swz<TR>(base);
#pragma unroll
        for (int j = 0; j < (1 << GB0); ++j) {
          const unsigned idx = sbase ^ swz<TR>((unsigned)j << C);
          sp[idx] = a[j];
          if (ADJA) sl[idx] = y[ADJA ? j : 0];
        }
      }
      __syncthreads();
      mixer_rounds_to<TR, ADJA, C, C + GB0, K>(sp, sl, kA, accA);
    }
    // the element-wise step between the two layers
    {
      float gsum = 0.f;
#pragma unroll
      for (unsigned i = 0; i < PER; ++i) {
        const unsigned l = tid + kThreads * i;
        const uint64_t x = C <= 8 ? tbase + off0 + step * i : fast_x<C>(tbase, l, s);
        const unsigned idx = swz<TR>(l);
        const int c = cut[x];
        const float cf = (float)c;
        const W xv = sp[idx];
        if constexpr (MODE == kMgTurn) {
          float pp, ee;
          qops::abs2(xv, pp, ee);
          accn.add(pp, ee);
          const float q = cf * pp;
          acce.add(q, fmaf(cf, pp, -q) + cf * ee);
          const float c2 = cf * cf;  // <= 255^2: exact
          const float q2 = c2 * pp;
          accl.add(q2, fmaf(c2, pp, -q2) + c2 * ee);
          sl[idx] = qops::scale_int(xv, cf);
        } else {
          const W yv = sl[idx];
          if constexpr (TR::kBlockSum) {
            gsum = fmaf(cf, qops::im_conj_mul_fma(yv, xv, 0.f), gsum);
          } else {
            float pp, ee;
            qops::im_conj_mul(yv, xv, pp, ee);
            const float qq = cf * pp;
            accg.add(qq, fmaf(cf, pp, -qq) + cf * ee);
          }
          if constexpr (MODE == kMgMerged) {
            sp[idx] = TR::mul(st[c], xv);
            sl[idx] = TR::mul(st[c], yv);
          }
        }
      }
      if (MODE != kMgTurn && TR::kBlockSum) accg.add(gsum, 0.f);
    }
    if constexpr (MODE != kMgLast) {
      __syncthreads();
      // layer B: rounds in shared memory, the last one straight to HBM
      mixer_rounds_to<TR, true, C, C, POSL>(sp, sl, kB, accB);
      constexpr unsigned NSUBL = 1u << (K - GBL);
      for (unsigned sb = tid; sb < NSUBL; sb += kThreads) {
        const unsigned base = block_base<POSL, GBL>(sb);
        const unsigned sbase = swz<TR>(base);
        W a[1 << GBL], y[1 << GBL];
#pragma unroll
        for (int j = 0; j < (1 << GBL); ++j) {
          const unsigned idx = sbase ^ swz<TR>((unsigned)j << POSL);
          a[j] = sp[idx];
          y[j] = sl[idx];
        }
        round_in_regs<TR, true, GBL>(a, y, kB, accB);
#pragma unroll
        for (int j = 0; j < (1 << GBL); ++j) {
          const uint64_t x = fast_x<C>(tbase, base | ((unsigned)j << POSL), s);
          if constexpr (MODE == kMgMerged) {
            if constexpr (kRn) {
              if (norm_out) {
                float pp, ee;
                qops::abs2(a[j], pp, ee);
                rnp.add(pp, ee);
                qops::abs2(y[j], pp, ee);
                rnl.add(pp, ee);
              }
            }
            P[x] = TR::store(a[j]);
          }
          L[x] = TR::store(y[j]);
        }
      }
    }
    __syncthreads();  // the next tile reuses shared memory
  }
  if (bad) atomicOr(flag, 1u);
  const uint64_t row = (uint64_t)b * part_stride + blockIdx.x;
  if (MODE != kMgTurn) block_partial(accA.value(), out.pA + row);
  if (MODE != kMgLast) block_partial(accB.value(), out.pB + row);
  if (MODE != kMgTurn) block_partial(accg.value(), out.pG + row);
  if (MODE == kMgTurn) {
    block_partial(acce.value(), out.pE + row);
    block_partial(accn.value(), out.pN + row);
    block_partial(accl.value(), out.pL + row);
  }
  if constexpr (kRn) {
    if (norm_out) {
      block_partial(rnp.value(), out.pRnP + row);
      block_partial(rnl.value(), out.pRnL + row);
    }
  }
}

// ---------------------------------------------------------------- chained segments
// A second schedule of the same evaluation (forward, energy and lambda, adjoint
// by uncompute) that moves each vector through HBM fewer times.  All RX
// factors of a mixer commute and the cost phase is diagonal, so the mixer of
// layer l may visit its passes (tile geometries g_0..g_{m-1}) in either order:
// even layers go 0..m-1, odd layers m-1..0.  The last pass of layer l and the
// first pass of layer l+1 then share a geometry, and the phase between them is
// an element-wise step, so the three run in ONE tile residency: RX_l on the
// tile's bits, phase_{l+1}, RX_{l+1} on the same bits.  The evaluation becomes
// one list of operations (phases, RX on one geometry, the turnaround that forms
// the energy and lambda = C phi, and the mirrored adjoint operations), cut into
// segments of consecutive operations on one geometry; each segment is one
// launch of k_seg.
//   - The first segment starts from |+>^n generated in registers (no fill, no load).
//   - The turnaround segment runs RX_{p-1} on its bits, forms E, |phi|^2,
//     lambda = C phi and |lambda|^2, then the adjoint RX^dagger_{p-1} on the
//     same bits; phi then equals the segment's input (up to rounding), so only
//     lambda is stored.
//   - The last adjoint segment stores nothing: only its gradient terms are needed.
// For m passes per mixer and depth p, one evaluation with gradient moves
// 3 p (m - 1) + 1 vector read-write pairs, against 3 p m + 2 for one pass
// sequence per layer (for m = 3, p = 4: 101 GB instead of 159 GB at 28 qubits).
enum : uint8_t { kOpRX = 0, kOpPhase = 1, kOpTurn = 2, kOpEnergy = 3 };
constexpr int kMaxSegOps = 2 * kMaxP + 3;  // a one-pass plan holds every operation in one segment

struct SegOp {
  uint8_t kind;
  uint8_t layer;
  uint8_t red;   // first per-thread accumulator slot of the op's sums (kSegTileSums: unused)
  uint8_t pad;
  uint16_t col;  // first partial column block (units of the launch's grid width) of the op's sums
};
constexpr uint16_t kNoCol = 0xffffu;  // an op without sums (forward RX and phase)
// Per-thread double-float accumulators of a segment's sums, kept in shared
// memory across the block's tiles and reduced once at the end (an FP64 block
// reduction per op and tile would run on the slow FP64 pipe).  A segment with
// more sums than slots (one tile pass per mixer at depth >= 3, where every
// block holds a single tile) reduces each op's sums over the block per tile.
constexpr int kSegRed = 8;

enum : uint32_t {
  kSegGen = 1u,        // phi = |+>^n, not loaded
  kSegAdjIn = 2u,      // the segment starts in the adjoint part: lambda is loaded too
  kSegStorePhi = 4u,
  kSegStoreLam = 8u,
  kSegRnScale = 16u,   // rescale phi and lambda on load (fused renormalisation)
  kSegRnSum = 32u,     // sum |phi|^2 and |lambda|^2 of the stored values
  kSegTileSums = 64u,  // per-tile block reductions instead of the accumulator slots
};

struct SegParams {
  int nops;
  int bmax;    // per-layer row stride of rx and tables
  int tsize;   // phase-table entries per state
  int per_graph;
  uint32_t flags;
  int rn_col;  // column blocks of the stored norms (|phi|^2, |lambda|^2 at rn_col + 1)
  int rn_red;  // accumulator slots of the stored norms
  int rn_stride;  // norms: [4][rn_stride] = current |phi|^2, lambda target, phi target, current |lambda|^2
  float amp;      // 2^(-n/2) (complex64 start value; complex128 uses amp64)
  double amp64;
  SegOp ops[kMaxSegOps];
};

// FP64 sums of one value per thread over the block, added to slot[0..NV) in a
// fixed order (thread 0).
template <int NV>
__device__ __forceinline__ void block_accumulate(const double (&v)[NV], double* slot, double (*red)[kThreads / 32]) {
  double w[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    w[k] = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w[k] += __shfl_xor_sync(0xffffffffu, w[k], o);
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) red[k][threadIdx.x >> 5] = w[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = 0.0;
      for (int q = 0; q < kThreads / 32; ++q) s += red[k][q];
      slot[k] += s;
    }
  }
  __syncthreads();
}

template <class V>
__device__ __forceinline__ V scale_v(V v, double f) {
  using S = decltype(v.x);
  v.x = (S)(v.x * (S)f);
  v.y = (S)(v.y * (S)f);
  return v;
}

// One segment on tiles of C row bits and K - C gate bits (the full-tile pass
// shapes of k_mixer_fast).  ANYADJ: the segment may hold the turnaround or
// start in the adjoint part (two vectors in shared memory); forward-only
// segments use the lighter instantiation.
template <class TR, int C, bool ANYADJ>
__global__ void __launch_bounds__(kThreads, 2)
    k_seg(typename TR::V* __restrict__ phi, typename TR::V* __restrict__ lam, uint64_t N, int s_bits,
          const typename TR::RX* __restrict__ rx, const typename TR::PH* __restrict__ tables,
          const uint8_t* __restrict__ cut, double* __restrict__ partials, int part_stride,
          const double* __restrict__ norms, unsigned* flag, const __grid_constant__ SegParams P) {
  using V = typename TR::V;
  using W = typename TR::W;
  using PHT = typename TR::PH;
  constexpr int K = TR::kTileBits;
  constexpr int M = K - C;
  constexpr unsigned T = 1u << K;
  constexpr unsigned PER = T / kThreads;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  W* sp = reinterpret_cast<W*>(smem_raw);
  W* sl = sp + T;
  __shared__ uint8_t cs[T];                       // cut counts of the tile's elements
  __shared__ PHT st[kEdgeChunk + 1];              // phase table of the current phase op
  __shared__ double slot[3 * kMaxSegOps + 2];     // per-op sums over this block's tiles (kSegTileSums)
  __shared__ double red[3][kThreads / 32];
  __shared__ dfx::Acc tacc[kSegRed][kThreads];    // per-thread sums over this block's tiles
  __shared__ double rn_f[2];
  const unsigned tid = threadIdx.x;
  const unsigned b = blockIdx.y;
  const bool tile_sums = (P.flags & kSegTileSums) != 0;
  for (int i = tid; i < 3 * P.nops + 2; i += kThreads) slot[i] = 0.0;
#pragma unroll
  for (int r = 0; r < kSegRed; ++r) tacc[r][tid] = dfx::Acc();
  // add this thread's sums of one op on the current tile
  auto put = [&](const SegOp& op, int o, int nv, const dfx::Acc* a) {
    if (tile_sums) {
      double v[3] = {0.0, 0.0, 0.0};
      for (int k = 0; k < nv; ++k) v[k] = a[k].value();
      block_accumulate<3>(v, &slot[3 * o], red);
    } else {
      for (int k = 0; k < nv; ++k) tacc[op.red + k][tid].add(a[k].h, a[k].l);
    }
  };
  const uint8_t* cutb = cut + (uint64_t)(b / (unsigned)P.per_graph) * N;
  V* Pv = phi + (uint64_t)b * N;
  V* Lv = ANYADJ ? lam + (uint64_t)b * N : nullptr;
  bool need_cut = false;
  for (int o = 0; o < P.nops; ++o) need_cut |= P.ops[o].kind != kOpRX;
  const bool gen = (P.flags & kSegGen) != 0;
  const bool adj_in = ANYADJ && (P.flags & kSegAdjIn) != 0;
  const bool st_phi = (P.flags & kSegStorePhi) != 0;
  const bool st_lam = ANYADJ && (P.flags & kSegStoreLam) != 0;
  const bool rn_scale = (P.flags & kSegRnScale) != 0;
  const bool rn_sum = (P.flags & kSegRnSum) != 0;
  if (rn_scale && tid == 0) {
    const double np = norms[b], tl = norms[P.rn_stride + b];
    const double tp = norms[2 * P.rn_stride + b], nl = norms[3 * P.rn_stride + b];
    rn_f[0] = np > 0.0 ? sqrt(tp / np) : 1.0;
    rn_f[1] = nl > 0.0 ? sqrt(tl / nl) : 1.0;
  }
  __syncthreads();
  unsigned bad = 0;
  V v0;
  v0.x = (decltype(v0.x))(sizeof(v0.x) == 8 ? P.amp64 : (double)P.amp);
  v0.y = 0;
  const W w0 = TR::load(v0, bad);
  const double f_phi = rn_scale ? rn_f[0] : 1.0, f_lam = rn_scale ? rn_f[1] : 1.0;
  const uint64_t tiles = N >> K;
  const int s = C == 0 ? 0 : s_bits;
  const int mid = s - C;
  const uint64_t off0 = C == 0 ? tid : ((uint64_t)(tid >> C) << s) | (tid & ((1u << C) - 1u));
  const uint64_t step = C == 0 ? kThreads : ((uint64_t)(kThreads >> (C <= 8 ? C : 8)) << s);
  const unsigned sw0 = swz<TR>(tid);
  auto gx_of = [&](uint64_t tbase, unsigned i) -> uint64_t {
    return C <= 8 ? tbase + off0 + step * i : fast_x<C>(tbase, tid + kThreads * i, s);
  };
  for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const uint64_t tbase = C == 0 ? (t << K) : (((t >> mid) << (s + M)) | ((t & ((1ull << mid) - 1ull)) << C));
    // load (coalesced: element l = tid + kThreads i)
#pragma unroll
    for (unsigned i = 0; i < PER; ++i) {
      const unsigned l = tid + kThreads * i;
      const uint64_t x = gx_of(tbase, i);
      const unsigned idx = sw0 ^ swz<TR>(kThreads * i);
      if (gen) {
        sp[idx] = w0;
      } else {
        V v = Pv[x];
        if (rn_scale) v = scale_v(v, f_phi);
        sp[idx] = TR::load(v, bad);
      }
      if constexpr (ANYADJ) {
        if (adj_in) {
          V v = Lv[x];
          if (rn_scale) v = scale_v(v, f_lam);
          sl[idx] = TR::load(v, bad);
        }
      }
      if (need_cut) cs[l] = cutb[x];
    }
    __syncthreads();
    bool adj = adj_in;
    for (int o = 0; o < P.nops; ++o) {
      const SegOp op = P.ops[o];
      if (op.kind == kOpRX) {
        const typename TR::RX k = rx[(uint64_t)op.layer * P.bmax + b];
        dfx::Acc acc;
        if constexpr (ANYADJ) {
          if (adj) {
            mixer_rounds<TR, true, C, C>(sp, sl, TR::rx_inv(k), acc);
            put(op, o, 1, &acc);
            continue;
          }
        }
        mixer_rounds<TR, false, C, C>(sp, sl, k, acc);
      } else if (op.kind == kOpPhase) {
        const PHT* tb = tables + ((uint64_t)op.layer * P.bmax + b) * P.tsize;
        for (int i = tid; i < P.tsize; i += kThreads) st[i] = adj ? TR::conj(tb[i]) : tb[i];
        __syncthreads();
        if (ANYADJ && adj) {
          float gsum = 0.f;
          dfx::Acc accg;
#pragma unroll
          for (unsigned i = 0; i < PER; ++i) {
            const unsigned l = tid + kThreads * i;
            const unsigned idx = sw0 ^ swz<TR>(kThreads * i);
            const int c = cs[l];
            const W xv = sp[idx], yv = sl[idx];
            const float cf = (float)c;
            if constexpr (TR::kBlockSum) {
              gsum = fmaf(cf, qops::im_conj_mul_fma(yv, xv, 0.f), gsum);
            } else {
              float pp, ee;
              qops::im_conj_mul(yv, xv, pp, ee);
              const float qq = cf * pp;
              accg.add(qq, fmaf(cf, pp, -qq) + cf * ee);
            }
            sp[idx] = TR::mul(st[c], xv);
            sl[idx] = TR::mul(st[c], yv);
          }
          if (TR::kBlockSum) accg.add(gsum, 0.f);
          put(op, o, 1, &accg);
          __syncthreads();  // element writes before the next op
        } else {
#pragma unroll
          for (unsigned i = 0; i < PER; ++i) {
            const unsigned l = tid + kThreads * i;
            const unsigned idx = sw0 ^ swz<TR>(kThreads * i);
            sp[idx] = TR::mul(st[cs[l]], sp[idx]);
          }
          __syncthreads();
        }
      } else {  // kOpTurn / kOpEnergy: E = sum C |phi|^2, |phi|^2, and (turnaround) lambda = C phi, |lambda|^2
        dfx::Acc acce, accn, accl;
        const bool turn = ANYADJ && op.kind == kOpTurn;
#pragma unroll
        for (unsigned i = 0; i < PER; ++i) {
          const unsigned l = tid + kThreads * i;
          const unsigned idx = sw0 ^ swz<TR>(kThreads * i);
          const float cf = (float)cs[l];
          const W xv = sp[idx];
          float p, e;
          qops::abs2(xv, p, e);
          accn.add(p, e);
          const float q = cf * p;
          acce.add(q, fmaf(cf, p, -q) + cf * e);
          if constexpr (ANYADJ) {
            if (turn) {
              const float c2 = cf * cf;  // <= 255^2: exact
              const float q2 = c2 * p;
              accl.add(q2, fmaf(c2, p, -q2) + c2 * e);
              sl[idx] = qops::scale_int(xv, cf);
            }
          }
        }
        const dfx::Acc a3[3] = {acce, accn, accl};
        put(op, o, turn ? 3 : 2, a3);
        __syncthreads();  // lambda writes before the next op
        if (turn) adj = true;
      }
    }
    // store
    dfx::Acc an, al;
#pragma unroll
    for (unsigned i = 0; i < PER; ++i) {
      const uint64_t x = gx_of(tbase, i);
      const unsigned idx = sw0 ^ swz<TR>(kThreads * i);
      if (st_phi) {
        const W w = sp[idx];
        if (rn_sum) {
          float p, e;
          qops::abs2(w, p, e);
          an.add(p, e);
        }
        Pv[x] = TR::store(w);
      }
      if constexpr (ANYADJ) {
        if (st_lam) {
          const W w = sl[idx];
          if (rn_sum) {
            float p, e;
            qops::abs2(w, p, e);
            al.add(p, e);
          }
          Lv[x] = TR::store(w);
        }
      }
    }
    if (rn_sum) {
      if (tile_sums) {
        const double v[2] = {an.value(), al.value()};
        block_accumulate<2>(v, &slot[3 * P.nops], red);
      } else {
        tacc[P.rn_red][tid].add(an.h, an.l);
        tacc[P.rn_red + 1][tid].add(al.h, al.l);
      }
    }
    __syncthreads();  // the next tile reuses shared memory
  }
  if (bad) atomicOr(flag, 1u);
  // this block's sums to its column of each op's partial blocks
  const uint64_t row = (uint64_t)b * part_stride + blockIdx.x;
  const uint64_t w = gridDim.x;
  if (tile_sums) {
    if (tid == 0) {
      for (int o = 0; o < P.nops; ++o) {
        const SegOp op = P.ops[o];
        if (op.col == kNoCol) continue;
        const int nv = (op.kind == kOpTurn) ? 3 : (op.kind == kOpEnergy ? 2 : 1);
        for (int k = 0; k < nv; ++k) partials[row + ((uint64_t)op.col + k) * w] = slot[3 * o + k];
      }
      if (rn_sum) {
        partials[row + (uint64_t)P.rn_col * w] = slot[3 * P.nops];
        partials[row + ((uint64_t)P.rn_col + 1) * w] = slot[3 * P.nops + 1];
      }
    }
  } else {
    for (int o = 0; o < P.nops; ++o) {
      const SegOp op = P.ops[o];
      if (op.col == kNoCol) continue;
      const int nv = (op.kind == kOpTurn) ? 3 : (op.kind == kOpEnergy ? 2 : 1);
      for (int k = 0; k < nv; ++k)
        block_partial(tacc[op.red + k][tid].value(), partials + row + ((uint64_t)op.col + k) * w);
    }
    if (rn_sum) {
      block_partial(tacc[P.rn_red][tid].value(), partials + row + (uint64_t)P.rn_col * w);
      block_partial(tacc[P.rn_red + 1][tid].value(), partials + row + ((uint64_t)P.rn_col + 1) * w);
    }
  }
}

// ---------------------------------------------------------------- TMA-staged mixer pass
// The same pass with its tiles moved by the Tensor Memory Accelerator: one
// thread issues cp.async.bulk.tensor loads (completion counted on an
// mbarrier) and stores (bulk groups); two tile buffers per vector let the next
// tile stream in while the current one is computed.  The tensor maps use the
// hardware 128-byte swizzle, which the register rounds index directly
// (kTmaSwizzle).  x coordinates are always 0, so every copy starts on a
// 128-byte row.
template <class TR>
struct TmaTraits : TR {
  static constexpr bool kTmaSwizzle = true;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void tma_load(void* dst, const CUtensorMap* map, int rank, const int* c, uint64_t* bar) {
  if (rank == 3)
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(map), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(smem_u32(bar))
        : "memory");
  else
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], "
        "[%7];" ::"r"(smem_u32(dst)), "l"(map), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(c[4]),
        "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_store(const CUtensorMap* map, int rank, const int* c, const void* src) {
  if (rank == 3)
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(map),
                 "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(smem_u32(src))
                 : "memory");
  else
    asm volatile("cp.async.bulk.tensor.5d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4, %5}], [%6];" ::"l"(map),
                 "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(c[4]), "r"(smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

constexpr uint32_t kMbarSpinLimit = 1u << 26;  // try_wait rounds before a wait is declared failed

// Forward-only modes of the chained schedule:
//   PH = 3: layer A's RX on the tile's bits, then layer B's cost phase on
//           every element, then layer B's RX (rx2) on the same bits;
//   PH = 4: RX, then the energy sums of the stored tile (sum C |phi|^2 to
//           partials, |phi|^2 to partials_g): the last forward tile of an
//           energy-only evaluation;
//   PH = 5: the first tile of an evaluation: |+>^n (amplitude amp0) times the
//           first cost phase is generated in shared memory, nothing is loaded.
__device__ __forceinline__ void bulk_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }

template <class TR, bool ADJ, int C, int PH>
__global__ void __launch_bounds__(kThreads) k_mixer_tma(const __grid_constant__ CUtensorMap tm_phi,
                                                        const __grid_constant__ CUtensorMap tm_lam, uint64_t N,
                                                        int s_bits, int hi_bits, const typename TR::RX* __restrict__ rx,
                                                        double* __restrict__ partials, int part_stride, unsigned* flag,
                                                        const uint8_t* __restrict__ cut,
                                                        const typename TR::PH* __restrict__ tables, int tsize,
                                                        double* __restrict__ partials_g, unsigned* err, int per_graph,
                                                        const typename TR::RX* __restrict__ rx2, double amp0) {
  static_assert(PH < 3 || !ADJ, "merged, energy and generating tiles of the TMA kernel are forward only");
  constexpr bool GEN = PH == 5;
  if (PH) cut += (uint64_t)(blockIdx.y / (unsigned)per_graph) * N;  // state b uses graph b / per_graph
  using TT = TmaTraits<TR>;
  using V = typename TR::V;
  using W = typename TR::W;
  using PHT = typename TR::PH;
  constexpr int K = TR::kTileBits;
  constexpr int M = K - C;
  constexpr unsigned T = 1u << K;
  constexpr unsigned PER = T / kThreads;
  constexpr unsigned TILE = T * sizeof(V);
  constexpr int NV = ADJ ? 2 : 1;
  constexpr bool CONVERT = !std::is_same<V, W>::value;  // complex128: split in place after the load
  constexpr int RANK = C == 0 ? 3 : 5;
  extern __shared__ __align__(16) unsigned char smem_dyn[];
  // the 128-byte TMA swizzle needs 1024-byte aligned tiles (1 KiB of slack is allocated)
  unsigned char* smem_raw = smem_dyn + ((1024u - (smem_u32(smem_dyn) & 1023u)) & 1023u);
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ PHT st[PH ? kEdgeChunk + 1 : 1];
  const unsigned tid = threadIdx.x;
  const unsigned b = blockIdx.y;
  if (PH && PH != 4) {
    for (int i = tid; i < tsize; i += blockDim.x) {
      const PHT tt = tables[(uint64_t)b * tsize + i];
      st[i] = PH == 2 ? TR::conj(tt) : tt;
    }
  }
  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  const typename TR::RX k = ADJ ? TR::rx_inv(rx[b]) : rx[b];
  const uint64_t tiles = N >> K;
  const int s = C == 0 ? 0 : s_bits;
  const int mid = s - C;
  auto vbuf = [&](int buf, int vec) { return smem_raw + (size_t)(buf * NV + vec) * TILE; };
  auto coords = [&](uint64_t t, int* c) {
    if (C == 0) {
      c[0] = 0; c[1] = 0; c[2] = (int)(b * tiles + t);
    } else {
      c[0] = 0; c[1] = 0; c[2] = (int)(t & ((1ull << mid) - 1ull)); c[3] = 0;
      c[4] = (int)((t >> mid) + ((uint64_t)b << hi_bits));
    }
  };
  auto issue = [&](uint64_t t, int buf) {
    int c[5];
    coords(t, c);
    mbar_expect_tx(&mbar[buf], TILE * NV);
    tma_load(vbuf(buf, 0), &tm_phi, RANK, c, &mbar[buf]);
    if (ADJ) tma_load(vbuf(buf, 1), &tm_lam, RANK, c, &mbar[buf]);
  };
  unsigned phase0 = 0, phase1 = 0;
  unsigned bad = 0;
  dfx::Acc acc, accg;
  V v0;
  v0.x = (decltype(v0.x))amp0;
  v0.y = 0;
  const W w0 = TR::load(v0, bad);
  uint64_t t = blockIdx.x;
  if (!GEN && t < tiles && tid == 0) issue(t, 0);
  for (int it = 0; t < tiles; ++it, t += gridDim.x) {
    const int buf = it & 1;
    const uint64_t tn = t + gridDim.x;
    W* sp = reinterpret_cast<W*>(vbuf(buf, 0));
    W* sl = ADJ ? reinterpret_cast<W*>(vbuf(buf, 1)) : nullptr;
    const uint64_t tbase = C == 0 ? (t << K) : (((t >> mid) << (s + M)) | ((t & ((1ull << mid) - 1ull)) << C));
    if constexpr (GEN) {
      if (tid == 0) bulk_wait_read1();  // the store from this buffer two tiles ago has read its shared memory
      __syncthreads();
#pragma unroll
      for (unsigned i = 0; i < PER; ++i) {
        const unsigned l = tid + kThreads * i;
        const uint64_t x = tbase + (((uint64_t)(l >> C)) << s) + (l & ((1u << C) - 1u));
        sp[swz<TT>(l)] = TR::mul(st[cut[x]], w0);
      }
      __syncthreads();
    } else {
      if (tid == 0 && tn < tiles) {
        bulk_wait_read0();  // the other buffer's previous store has read its shared memory
        fence_proxy_async();
        issue(tn, buf ^ 1);
      }
      unsigned& ph = buf ? phase1 : phase0;
      bool ok = false;
      for (uint32_t spin = 0; spin < kMbarSpinLimit; ++spin)
        if (mbar_try_wait(&mbar[buf], ph)) { ok = true; break; }
      ph ^= 1u;
      if (__syncthreads_or(!ok)) {  // a tile never arrived: report and leave
        if (tid == 0) atomicOr(err, 1u);
        break;
      }
    }
    if (!GEN && (CONVERT || PH == 1)) {
#pragma unroll
      for (unsigned i = 0; i < PER; ++i) {
        const unsigned l = tid + kThreads * i;
        const unsigned idx = swz<TT>(l);
        W w = TR::load(reinterpret_cast<const V*>(sp)[idx], bad);
        if (PH == 1) {
          const uint64_t x = tbase + (((uint64_t)(l >> C)) << s) + (l & ((1u << C) - 1u));
          w = TR::mul(st[cut[x]], w);
        }
        sp[idx] = w;
        if (ADJ && CONVERT) sl[idx] = TR::load(reinterpret_cast<const V*>(sl)[idx], bad);
      }
      __syncthreads();
    }
    mixer_rounds<TT, ADJ, C, C>(sp, sl, k, acc);
    if constexpr (PH == 3) {
#pragma unroll
      for (unsigned i = 0; i < PER; ++i) {
        const unsigned l = tid + kThreads * i;
        const unsigned idx = swz<TT>(l);
        const uint64_t x = tbase + (((uint64_t)(l >> C)) << s) + (l & ((1u << C) - 1u));
        sp[idx] = TR::mul(st[cut[x]], sp[idx]);
      }
      __syncthreads();
      mixer_rounds<TT, ADJ, C, C>(sp, sl, rx2[b], acc);
    }
    if (CONVERT || PH == 2 || PH == 4) {
      float gsum = 0.f;
#pragma unroll
      for (unsigned i = 0; i < PER; ++i) {
        const unsigned l = tid + kThreads * i;
        const unsigned idx = swz<TT>(l);
        W xv = sp[idx];
        W yv = ADJ ? sl[idx] : xv;
        if (PH == 4) {
          const uint64_t x = tbase + (((uint64_t)(l >> C)) << s) + (l & ((1u << C) - 1u));
          const float cf = (float)cut[x];
          float pp, ee;
          qops::abs2(xv, pp, ee);
          accg.add(pp, ee);  // |phi|^2
          const float q = cf * pp;
          acc.add(q, fmaf(cf, pp, -q) + cf * ee);  // C |phi|^2 (forward RX rounds add nothing to acc)
        }
        if (PH == 2) {
          const uint64_t x = tbase + (((uint64_t)(l >> C)) << s) + (l & ((1u << C) - 1u));
          const int c = cut[x];
          const float cf = (float)c;
          if constexpr (TR::kBlockSum) {
            gsum = fmaf(cf, qops::im_conj_mul_fma(yv, xv, 0.f), gsum);
          } else {
            float pp, ee;
            qops::im_conj_mul(yv, xv, pp, ee);
            const float qq = cf * pp;
            accg.add(qq, fmaf(cf, pp, -qq) + cf * ee);
          }
          xv = TR::mul(st[c], xv);
          yv = TR::mul(st[c], yv);
        }
        reinterpret_cast<V*>(sp)[idx] = TR::store(xv);
        if (ADJ) reinterpret_cast<V*>(sl)[idx] = TR::store(yv);
      }
      if (PH == 2 && TR::kBlockSum) accg.add(gsum, 0.f);
    }
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      int c[5];
      coords(t, c);
      tma_store(&tm_phi, RANK, c, vbuf(buf, 0));
      if (ADJ) tma_store(&tm_lam, RANK, c, vbuf(buf, 1));
      bulk_commit();
    }
  }
  if (tid == 0) bulk_wait0();
  __syncthreads();
  if (bad) atomicOr(flag, 1u);
  if (ADJ || PH == 4) block_partial(acc.value(), partials + (uint64_t)b * part_stride + blockIdx.x);
  if (PH == 2 || PH == 4) block_partial(accg.value(), partials_g + (uint64_t)b * part_stride + blockIdx.x);
}

// Cost phase: psi_x <- T_b[C(x)] psi_x.  When ADJ: accumulate Im conj(lambda) C phi
// first, then multiply both vectors by conj(T_b[C(x)]).
template <class TR, bool ADJ>
__global__ void __launch_bounds__(kThreads) k_phase(typename TR::V* __restrict__ phi, typename TR::V* __restrict__ lam,
                                                    uint64_t N, const uint8_t* __restrict__ cut,
                                                    const typename TR::PH* __restrict__ tables, int tsize,
                                                    double* __restrict__ partials, int part_stride, unsigned* flag,
                                                    int per_graph) {
  using PH = typename TR::PH;
  using W = typename TR::W;
  __shared__ PH st[kEdgeChunk + 1];
  const unsigned b = blockIdx.y;
  cut += (uint64_t)(b / (unsigned)per_graph) * N;
  for (int i = threadIdx.x; i < tsize; i += blockDim.x) {
    const PH t = tables[(uint64_t)b * tsize + i];
    st[i] = ADJ ? TR::conj(t) : t;
  }
  __syncthreads();
  typename TR::V* P = phi + (uint64_t)b * N;
  typename TR::V* L = ADJ ? lam + (uint64_t)b * N : nullptr;
  unsigned bad = 0;
  dfx::Acc acc;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x) {
    const int c = cut[i];
    W x = TR::load(P[i], bad);
    if (ADJ) {
      W y = TR::load(L[i], bad);
      float p, e;
      qops::im_conj_mul(y, x, p, e);
      const float cf = (float)c;
      const float q = cf * p;
      acc.add(q, fmaf(cf, p, -q) + cf * e);
      L[i] = TR::store(TR::mul(st[c], y));
    }
    P[i] = TR::store(TR::mul(st[c], x));
  }
  if (bad) atomicOr(flag, 1u);
  if (ADJ) block_partial(acc.value(), partials + (uint64_t)b * part_stride + blockIdx.x);
}

// Energy sum C |phi|^2 and squared norm sum |phi|^2 (partials at [blockIdx.x]
// and [gridDim.x + blockIdx.x]), and lambda = C phi when lam != nullptr.
template <class TR>
__global__ void __launch_bounds__(kThreads) k_energy_lambda(const typename TR::V* __restrict__ phi,
                                                            typename TR::V* __restrict__ lam, uint64_t N,
                                                            const uint8_t* __restrict__ cut,
                                                            double* __restrict__ partials, int part_stride,
                                                            unsigned* flag, int per_graph) {
  const unsigned b = blockIdx.y;
  cut += (uint64_t)(b / (unsigned)per_graph) * N;
  const typename TR::V* P = phi + (uint64_t)b * N;
  typename TR::V* L = lam ? lam + (uint64_t)b * N : nullptr;
  unsigned bad = 0;
  dfx::Acc acc, accn;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x) {
    const float cf = (float)cut[i];
    const typename TR::W x = TR::load(P[i], bad);
    float p, e;
    qops::abs2(x, p, e);
    accn.add(p, e);
    const float q = cf * p;
    acc.add(q, fmaf(cf, p, -q) + cf * e);
    if (L) L[i] = TR::store(qops::scale_int(x, cf));
  }
  if (bad) atomicOr(flag, 1u);
  block_partial(acc.value(), partials + (uint64_t)b * part_stride + blockIdx.x);
  block_partial(accn.value(), partials + (uint64_t)b * part_stride + gridDim.x + blockIdx.x);
}

// results[b][0..count) /= norm[b]: energies and gradients become Rayleigh
// quotients of the computed state, which removes the norm drift that rounded
// (not exactly unitary) gate coefficients leave in complex64.
__global__ void k_divide_results(double* __restrict__ results, int stride, int count, const double* __restrict__ norm) {
  const unsigned b = blockIdx.x;
  const double nb = norm[b];
  for (int j = threadIdx.x; j < count; j += blockDim.x) results[(uint64_t)b * stride + j] /= nb;
}

// Squared norm of each state (for renormalisation).
template <class TR>
__global__ void __launch_bounds__(kThreads) k_norm_batch(const typename TR::V* __restrict__ a, uint64_t N,
                                                         double* __restrict__ partials, int part_stride,
                                                         unsigned* flag) {
  const unsigned b = blockIdx.y;
  const typename TR::V* P = a + (uint64_t)b * N;
  unsigned bad = 0;
  dfx::Acc acc;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x) {
    float p, e;
    qops::abs2(TR::load(P[i], bad), p, e);
    acc.add(p, e);
  }
  if (bad) atomicOr(flag, 1u);
  block_partial(acc.value(), partials + (uint64_t)b * part_stride + blockIdx.x);
}

// out[b * out_stride + slot] = scale * sum_{j < count} partials[b * part_stride + j]
__global__ void k_finalize_batch(const double* __restrict__ partials, int count, int part_stride, double scale,
                                 double* __restrict__ out, int out_stride, int slot) {
  const unsigned b = blockIdx.x;
  double s = 0.0;
  for (int j = threadIdx.x; j < count; j += blockDim.x) s += partials[(uint64_t)b * part_stride + j];
  __shared__ double red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    out[(uint64_t)b * out_stride + slot] = scale * t;
  }
}

// a_b <- a_b * sqrt(target_b / norm_b)   (target == nullptr: target 1).  The
// factor is formed once per block in FP64 and rounded to the storage precision,
// so complex64 states are scaled on the FP32 pipe (one rounding of the factor,
// one of the product: the same order as storing an FP64-scaled value).
template <class V>
__global__ void k_rescale(V* __restrict__ a, uint64_t N, const double* __restrict__ norm, const double* __restrict__ target) {
  using S = decltype(V::x);
  __shared__ S fs;
  const unsigned b = blockIdx.y;
  if (threadIdx.x == 0) {
    const double nb = norm[b];
    fs = (S)(nb > 0.0 ? sqrt((target ? target[b] : 1.0) / nb) : 1.0);
  }
  __syncthreads();
  const S f = fs;
  V* P = a + (uint64_t)b * N;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x) {
    V v = P[i];
    v.x *= f;
    v.y *= f;
    P[i] = v;
  }
}

}  // namespace
}  // namespace iqs

// ================================================================ host engine
struct iqs_qaoa {
  int n = 0, dtype = IQS_C64, bmax = 0, n_edges = 0;
  int engine = 0;     // 0 auto (= tiled), 1 tiled passes, 2 cluster-resident (energies only, complex64)
  int clogc = -1;     // cluster size 2^clogc of the cluster-resident forward (-1: not available)
  int cclusters = 0;  // co-resident clusters of that kernel
  int n_graphs = 1;          // cut tables, one per graph ([n_graphs][N] bytes)
  int per_graph = 1 << 30;   // state b uses graph b / per_graph
  uint64_t N = 0;
  cudaStream_t stream = nullptr;
  int renorm_every = 0;
  void* phi = nullptr;
  void* lam = nullptr;
  uint8_t* cut = nullptr;
  void* rx = nullptr;          // [kMaxP][bmax] RX coefficients
  void* tables = nullptr;      // [kMaxP][bmax][n_edges + 1] phase factors
  double* partials = nullptr;  // [bmax][part_stride]
  double* results = nullptr;   // [bmax][1 + 2 kMaxP]
  double* norms = nullptr;     // [4][bmax]: current norm, lambda target, phi norm after the forward pass,
                               // current lambda norm (fused renormalisation)
  unsigned* flag = nullptr;
  unsigned char* host_params = nullptr;  // pinned staging of rx + tables
  double* host_results = nullptr;        // pinned
  size_t rx_bytes = 0, table_bytes = 0;
  std::vector<iqs::Geo> passes;
  std::map<std::tuple<int, int, int, int>, std::pair<cudaGraphExec_t, int>> graphs;  // (B, p, grad, renorm) -> graph, kernels
  bool use_graphs = true;
  bool own_stream = false;
  // tile-shape choice (autotuner): high-pass row bits (-1: default) and grid multiplier
  int row_bits = -1;
  int grid_mult = 1;
  // TMA-staged mixer passes: 0 off, 1 forward passes, 2 forward and adjoint passes.
  // Forward staging is the default: it measured 5-6% faster than register-loaded
  // tiles at 16-28 qubits, while staged adjoint passes (128 KB, one block per SM)
  // measured slower.  Passes whose tensor maps could not be built load directly.
  int tma_mode = 1;
  std::vector<CUtensorMap> tm_phi, tm_lam;  // one per mixer pass (valid when tma_ok)
  bool tma_ok = false;
  unsigned* tma_err = nullptr;              // device word: a TMA wait gave up
  // Pass schedule: 0 chained segments (default where every pass is a full tile),
  // 1 one pass sequence per layer with separate energy and lambda passes.
  int schedule = 0;
  size_t partials_cap = 0;  // doubles allocated at partials
};

namespace iqs {

// pool_cluster.cu: the cluster-resident forward pass (energies only, complex64)
int qaoa_cluster_setup(int n, int* logc);
cudaError_t launch_qaoa_cluster(int logc, int clusters, const uint8_t* cut, uint64_t N, int per_graph,
                                const float2* rx, const float2* tables, int tsize, int bmax, int n, int p, int batch,
                                float2* phi, double* results, int rstride, cudaStream_t s);

namespace {

// The cluster-resident forward only on request: measured against the tiled
// passes it ties up to 14 qubits and loses at 16 and 18 (issue-bound at 16
// warps per SM, while the batched tiled passes mostly hit L2).
bool use_cluster(const iqs_qaoa* q) { return q->engine == 2 && q->clogc >= 0 && q->cclusters > 0; }

// Partial slots per state: mixer passes x blocks (<= 4 x 2432), then the fused
// phase-gradient partials at kGammaCol, then the fused renormalisation's norm
// partials (|phi|^2 at kNormCol, |lambda|^2 at kNormCol + kRnCol).
constexpr int kGammaCol = 2432 * 4;
constexpr int kNormCol = 2432 * 5;
int part_stride_for(const iqs_qaoa* q) { return 2432 * 7; }

int blocks_per_state(const iqs_qaoa* q, int B) {
  const uint64_t by_size = std::max<uint64_t>(1, q->N / 4096);
  const int by_batch = std::max(1, q->grid_mult * 2432 / std::max(B, 1));
  return (int)std::min<uint64_t>(by_size, (uint64_t)std::min(by_batch, 2432));
}

// Mixer passes for n qubits: a low pass over the first min(n, K) qubits
// (contiguous tile), then the remaining qubits spread evenly over high passes
// of at most K - row_bits gate bits each; every high pass fills its tile to
// 2^K amplitudes with K - m contiguous row bits.
std::vector<Geo> plan_mixer(int n, int tile_bits, int row_bits) {
  std::vector<Geo> out;
  const int m0 = std::min(n, tile_bits);
  out.push_back(Geo{0, 0, m0});
  const int rem = n - m0;
  if (rem > 0) {
    const int maxm = tile_bits - row_bits;
    const int np = (rem + maxm - 1) / maxm;
    int q0 = m0;
    for (int i = 0; i < np; ++i) {
      const int mm = rem / np + (i < rem % np ? 1 : 0);
      out.push_back(Geo{tile_bits - mm, q0, mm});
      q0 += mm;
    }
  }
  return out;
}

void replan(iqs_qaoa* q);

template <class TR>
size_t tile_smem(const Geo& g, int nvec) {
  return (size_t)nvec * ((size_t)1 << (g.c + g.m)) * sizeof(typename TR::W);
}

// Optional fused cost phase of a mixer pass (see k_mixer_fast).
template <class TR>
struct PhaseFuse {
  int mode = 0;  // 0 none, 1 forward on load, 2 adjoint on store
  const uint8_t* cut = nullptr;
  const typename TR::PH* tables = nullptr;
  int tsize = 0;
  double* partials_g = nullptr;
  int per_graph = 1 << 30;  // state b uses cut table b / per_graph
  RenormFuse rn;            // fused renormalisation (adjoint, complex64, shape-specialised passes)
  // mode 3 (chained schedule): RX of layer A, the phase, RX of layer B (rx2) in one tile;
  // adjoint: layer B's gradient sums go to partials_b2
  const typename TR::RX* rx2 = nullptr;
  double* partials_b2 = nullptr;
  double amp0 = 0.0;  // mode 5: amplitude of |+>^n
};

template <class TR, bool ADJ, int C>
void launch_fast(dim3 grid, size_t smem, cudaStream_t s, typename TR::V* phi, typename TR::V* lam, uint64_t N, int sb,
                 const typename TR::RX* rx, double* partials, int ps, unsigned* flag, const PhaseFuse<TR>& f) {
  if (!ADJ && f.mode == 1)
    k_mixer_fast<TR, ADJ, C, (ADJ ? 0 : 1)>()<<<grid, kThreads, smem, s>>>(phi, lam, N, sb, rx, partials, ps, flag,
                                                                          f.cut, f.tables, f.tsize, f.partials_g,
                                                                          f.per_graph, RenormFuse());
  else if (ADJ && f.mode == 2)
    k_mixer_fast<TR, ADJ, C, (ADJ ? 2 : 0)>()<<<grid, kThreads, smem, s>>>(phi, lam, N, sb, rx, partials, ps, flag,
                                                                          f.cut, f.tables, f.tsize, f.partials_g,
                                                                          f.per_graph, f.rn);
  else
    k_mixer_fast<TR, ADJ, C, 0>()<<<grid, kThreads, smem, s>>>(phi, lam, N, sb, rx, partials, ps, flag, nullptr, nullptr,
                                                             0, nullptr, 1, f.rn);
}

template <class TR, int C>
cudaError_t set_attr_c(int bytes) {
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(k_mixer_fast<TR, false, C, 0>(), a, bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mixer_fast<TR, true, C, 0>(), a, bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mixer_fast<TR, false, C, 1>(), a, bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mixer_fast<TR, true, C, 2>(), a, bytes);
  return e;
}

template <class TR, int... Cs>
cudaError_t set_attr_all(int bytes, std::integer_sequence<int, Cs...>) {
  cudaError_t e = cudaSuccess;
  ((e = (e == cudaSuccess ? set_attr_c<TR, Cs + TR::kRowBits>(bytes) : e)), ...);
  return e;
}

template <class TR>
cudaError_t set_smem_attrs() {
  const int bytes = 2 * (1 << TR::kTileBits) * (int)sizeof(typename TR::W);
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(k_mixer<TR, false>, a, bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mixer<TR, true>, a, bytes);
  if (e == cudaSuccess) e = set_attr_c<TR, 0>(bytes);
  if (e == cudaSuccess) e = set_attr_all<TR>(bytes, std::make_integer_sequence<int, TR::kTileBits - TR::kRowBits>{});
  return e;
}

template <class TR, bool ADJ, int... Cs>
bool dispatch_fast(int c, dim3 grid, size_t smem, cudaStream_t s, typename TR::V* phi, typename TR::V* lam,
                   uint64_t N, int sb, const typename TR::RX* rx, double* partials, int ps, unsigned* flag,
                   const PhaseFuse<TR>& f, std::integer_sequence<int, Cs...>) {
  bool done = false;
  ((c == Cs + TR::kRowBits && !done
        ? (launch_fast<TR, ADJ, Cs + TR::kRowBits>(grid, smem, s, phi, lam, N, sb, rx, partials, ps, flag, f),
           done = true)
        : false),
   ...);
  return done;
}

// One mixer pass: a kernel specialised for the tile shape when the tile is
// full (2^kTileBits amplitudes), the generic one otherwise (tiny states).
// True when a pass runs on the shape-specialised kernels (full 2^K tile),
// which are the ones that can carry the fused cost phase.
template <class TR>
bool fast_shape(const Geo& g) {
  return g.c + g.m == TR::kTileBits && (g.c == 0 ? g.s == 0 : g.c >= TR::kRowBits);
}

// TMA staging of one pass (tensor maps built by replan()).
struct TmaArgs {
  bool use = false;
  const CUtensorMap* phi = nullptr;
  const CUtensorMap* lam = nullptr;
  int hi_bits = 0;
  unsigned* err = nullptr;
};

template <class TR>
size_t tma_smem(bool adj) {
  return (size_t)2 * (adj ? 2 : 1) * ((size_t)1 << TR::kTileBits) * sizeof(typename TR::V) + 1024;
}

template <class TR, bool ADJ, int C, int PH>
void launch_tma1(dim3 grid, cudaStream_t s, uint64_t N, int sb, const typename TR::RX* rx, double* partials, int ps,
                 unsigned* flag, const PhaseFuse<TR>& f, const TmaArgs& ta) {
  k_mixer_tma<TR, ADJ, C, PH><<<grid, kThreads, tma_smem<TR>(ADJ), s>>>(
      *ta.phi, ADJ ? *ta.lam : *ta.phi, N, sb, ta.hi_bits, rx, partials, ps, flag, f.cut, f.tables, f.tsize,
      f.partials_g, ta.err, f.per_graph, f.rx2, f.amp0);
}

template <class TR, bool ADJ, int C>
void launch_tma_c(dim3 grid, cudaStream_t s, uint64_t N, int sb, const typename TR::RX* rx, double* partials, int ps,
                  unsigned* flag, const PhaseFuse<TR>& f, const TmaArgs& ta) {
  if (!ADJ && f.mode == 3)
    launch_tma1<TR, ADJ, C, ADJ ? 0 : 3>(grid, s, N, sb, rx, partials, ps, flag, f, ta);
  else if (!ADJ && f.mode == 4)
    launch_tma1<TR, ADJ, C, ADJ ? 0 : 4>(grid, s, N, sb, rx, partials, ps, flag, f, ta);
  else if (!ADJ && f.mode == 5)
    launch_tma1<TR, ADJ, C, ADJ ? 0 : 5>(grid, s, N, sb, rx, partials, ps, flag, f, ta);
  else if (!ADJ && f.mode == 1 && C == 0)
    launch_tma1<TR, ADJ, C, (!ADJ && C == 0) ? 1 : 0>(grid, s, N, sb, rx, partials, ps, flag, f, ta);
  else if (ADJ && f.mode == 2)
    launch_tma1<TR, ADJ, C, ADJ ? 2 : 0>(grid, s, N, sb, rx, partials, ps, flag, f, ta);
  else
    launch_tma1<TR, ADJ, C, 0>(grid, s, N, sb, rx, partials, ps, flag, f, ta);
}

template <class TR, bool ADJ, int... Cs>
void dispatch_tma(int c, dim3 grid, cudaStream_t s, uint64_t N, int sb, const typename TR::RX* rx, double* partials,
                  int ps, unsigned* flag, const PhaseFuse<TR>& f, const TmaArgs& ta,
                  std::integer_sequence<int, Cs...>) {
  bool done = false;
  ((c == Cs + TR::kRowBits && !done
        ? (launch_tma_c<TR, ADJ, Cs + TR::kRowBits>(grid, s, N, sb, rx, partials, ps, flag, f, ta), done = true)
        : false),
   ...);
}

template <class TR, bool ADJ, int... Cs>
cudaError_t set_tma_attrs_c(std::integer_sequence<int, Cs...>) {
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  const int bytes = (int)tma_smem<TR>(ADJ);
  cudaError_t e = cudaSuccess;
  ((e = e == cudaSuccess ? cudaFuncSetAttribute(k_mixer_tma<TR, ADJ, Cs + TR::kRowBits, 0>, a, bytes) : e), ...);
  if (ADJ) ((e = e == cudaSuccess ? cudaFuncSetAttribute(k_mixer_tma<TR, ADJ, Cs + TR::kRowBits, ADJ ? 2 : 0>, a, bytes) : e), ...);
  if (!ADJ) ((e = e == cudaSuccess ? cudaFuncSetAttribute(k_mixer_tma<TR, ADJ, Cs + TR::kRowBits, ADJ ? 0 : 3>, a, bytes) : e), ...);
  if (!ADJ) ((e = e == cudaSuccess ? cudaFuncSetAttribute(k_mixer_tma<TR, ADJ, Cs + TR::kRowBits, ADJ ? 0 : 4>, a, bytes) : e), ...);
  if (!ADJ) ((e = e == cudaSuccess ? cudaFuncSetAttribute(k_mixer_tma<TR, ADJ, Cs + TR::kRowBits, ADJ ? 0 : 5>, a, bytes) : e), ...);
  return e;
}

template <class TR>
cudaError_t set_tma_attrs() {
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(k_mixer_tma<TR, false, 0, 0>, a, (int)tma_smem<TR>(false));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mixer_tma<TR, false, 0, 1>, a, (int)tma_smem<TR>(false));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mixer_tma<TR, false, 0, 3>, a, (int)tma_smem<TR>(false));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mixer_tma<TR, false, 0, 4>, a, (int)tma_smem<TR>(false));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mixer_tma<TR, false, 0, 5>, a, (int)tma_smem<TR>(false));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mixer_tma<TR, true, 0, 0>, a, (int)tma_smem<TR>(true));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mixer_tma<TR, true, 0, 2>, a, (int)tma_smem<TR>(true));
  const auto seq = std::make_integer_sequence<int, TR::kTileBits - TR::kRowBits>{};
  if (e == cudaSuccess) e = set_tma_attrs_c<TR, false>(seq);
  if (e == cudaSuccess) e = set_tma_attrs_c<TR, true>(seq);
  return e;
}

// One mixer pass: TMA-staged when requested and possible, else the kernel
// specialised for the tile shape when the tile is full (2^kTileBits
// amplitudes), else the generic one (tiny states).
template <class TR, bool ADJ>
void launch_mixer(const Geo& g, dim3 grid, cudaStream_t s, typename TR::V* phi, typename TR::V* lam, uint64_t N,
                  const typename TR::RX* rx, double* partials, int ps, unsigned* flag,
                  const PhaseFuse<TR>& f = PhaseFuse<TR>(), const TmaArgs& ta = TmaArgs()) {
  if (ta.use && fast_shape<TR>(g)) {
    if (g.c == 0)
      launch_tma_c<TR, ADJ, 0>(grid, s, N, 0, rx, partials, ps, flag, f, ta);
    else
      dispatch_tma<TR, ADJ>(g.c, grid, s, N, g.s, rx, partials, ps, flag, f, ta,
                            std::make_integer_sequence<int, TR::kTileBits - TR::kRowBits>{});
    return;
  }
  const size_t smem = tile_smem<TR>(g, ADJ ? 2 : 1);
  if (g.c + g.m == TR::kTileBits && g.c == 0 && g.s == 0) {
    launch_fast<TR, ADJ, 0>(grid, smem, s, phi, lam, N, 0, rx, partials, ps, flag, f);
    return;
  }
  if (g.c + g.m == TR::kTileBits &&
      dispatch_fast<TR, ADJ>(g.c, grid, smem, s, phi, lam, N, g.s, rx, partials, ps, flag, f,
                             std::make_integer_sequence<int, TR::kTileBits - TR::kRowBits>{}))
    return;
  k_mixer<TR, ADJ><<<grid, kThreads, smem, s>>>(phi, lam, N, g, rx, partials, ps, flag);
}

// Enqueue one full evaluation (forward, energy, optional backward) for B states and depth p.
template <class TR>
cudaError_t enqueue(iqs_qaoa* q, int B, int p, bool grad, int* n_launches) {
  using V = typename TR::V;
  using RX = typename TR::RX;
  using PH = typename TR::PH;
  const uint64_t N = q->N;
  cudaStream_t s = q->stream;
  V* phi = (V*)q->phi;
  V* lam = (V*)q->lam;
  const RX* rx = (const RX*)q->rx;
  const PH* tab = (const PH*)q->tables;
  const int tsize = q->n_edges + 1;
  const int out_stride = 1 + 2 * kMaxP;
  const int PB = blocks_per_state(q, B);
  const int ps = part_stride_for(q);
  int launches = 0;
  if constexpr (std::is_same<TR, T64>::value) {
    if (!grad && use_cluster(q)) {  // every state resident in a thread-block cluster for all p layers
      *n_launches = 1;
      return launch_qaoa_cluster(q->clogc, q->cclusters, q->cut, N, q->per_graph, (const float2*)q->rx,
                                 (const float2*)q->tables, tsize, q->bmax, q->n, p, B, (float2*)q->phi, q->results,
                                 out_stride, s);
    }
  }
  const double amp = std::pow(2.0, -q->n / 2.0);
  V v0;
  v0.x = (decltype(v0.x))amp;
  v0.y = 0;
  k_fill_uniform<V><<<grid_for(N * B, 1, 16), kThreads, 0, s>>>(phi, N * B, v0);
  ++launches;
  const dim3 g_stream(PB, B);
  const bool fuse_in = fast_shape<TR>(q->passes.front());
  const bool fuse_out = fast_shape<TR>(q->passes.back());
  for (int l = 0; l < p; ++l) {
    const typename TR::PH* tab_l = tab + (uint64_t)l * q->bmax * tsize;
    if (!fuse_in) {
      k_phase<TR, false><<<g_stream, kThreads, 0, s>>>(phi, nullptr, N, q->cut, tab_l, tsize, nullptr, 0, q->flag,
                                                       q->per_graph);
      ++launches;
    }
    for (size_t i = 0; i < q->passes.size(); ++i) {
      const Geo& g = q->passes[i];
      const uint64_t tiles = N >> (g.c + g.m);
      const dim3 grid((unsigned)std::min<uint64_t>(tiles, (uint64_t)PB), B);
      PhaseFuse<TR> f;
      if (i == 0 && fuse_in) {
        f.mode = 1;
        f.cut = q->cut;
        f.per_graph = q->per_graph;
        f.tables = tab_l;
        f.tsize = tsize;
      }
      TmaArgs ta;
      ta.use = q->tma_ok && q->tma_mode >= 1;
      ta.phi = &q->tm_phi[i];
      ta.lam = &q->tm_lam[i];
      ta.hi_bits = q->n - g.s - g.m;
      ta.err = q->tma_err;
      launch_mixer<TR, false>(g, grid, s, phi, nullptr, N, rx + (uint64_t)l * q->bmax, nullptr, 0, q->flag, f, ta);
      ++launches;
    }
  }
  double* phi_norm = q->norms + 2 * q->bmax;  // |phi|^2 after the forward pass
  k_energy_lambda<TR><<<g_stream, kThreads, 0, s>>>(phi, grad ? lam : nullptr, N, q->cut, q->partials, ps, q->flag,
                                                    q->per_graph);
  k_finalize_batch<<<B, kThreads, 0, s>>>(q->partials, PB, ps, 1.0, q->results, out_stride, 0);
  k_finalize_batch<<<B, kThreads, 0, s>>>(q->partials + PB, PB, ps, 1.0, phi_norm, 1, 0);
  launches += 3;
  if (grad) {
    const int R = q->renorm_every;
    if (R > 0) {  // record |lambda|^2 as the target of later rescaling
      k_norm_batch<TR><<<g_stream, kThreads, 0, s>>>(lam, N, q->partials, ps, q->flag);
      k_finalize_batch<<<B, kThreads, 0, s>>>(q->partials, PB, ps, 1.0, q->norms + q->bmax, 1, 0);
      launches += 2;
    }
    double* partials_g = q->partials + kGammaCol;  // phase-gradient partials of the fused last pass
    // complex64 on the shape-specialised adjoint passes: the last pass of a layer
    // sums the norms of what it stores and the next layer's first pass rescales
    // on load, instead of separate norm and rescale passes over both vectors
    const bool adj_tma = q->tma_ok && q->tma_mode >= 2;
    const bool fuse_rn = std::is_same<TR, T64>::value && R > 0 && fuse_out && fuse_in && !adj_tma;
    bool scale_pending = false;
    for (int l = p - 1; l >= 0; --l) {
      const typename TR::PH* tab_l = tab + (uint64_t)l * q->bmax * tsize;
      const bool renorm_after = R > 0 && l > 0 && ((p - l) % R) == 0;
      int col = 0;
      unsigned last_gx = 0;
      for (size_t i = 0; i < q->passes.size(); ++i) {
        const Geo& g = q->passes[i];
        const uint64_t tiles = N >> (g.c + g.m);
        const unsigned gx = (unsigned)std::min<uint64_t>(tiles, (uint64_t)PB);
        const dim3 grid(gx, B);
        PhaseFuse<TR> f;
        if (i + 1 == q->passes.size() && fuse_out) {
          f.mode = 2;
          f.cut = q->cut;
          f.per_graph = q->per_graph;
          f.tables = tab_l;
          f.tsize = tsize;
          f.partials_g = partials_g;
          if (fuse_rn && renorm_after) f.rn.partials = q->partials + kNormCol;
        }
        if (i == 0 && scale_pending) {
          f.rn.norms = q->norms;
          f.rn.stride = q->bmax;
          scale_pending = false;
        }
        TmaArgs ta;
        ta.use = adj_tma;
        ta.phi = &q->tm_phi[i];
        ta.lam = &q->tm_lam[i];
        ta.hi_bits = q->n - g.s - g.m;
        ta.err = q->tma_err;
        launch_mixer<TR, true>(g, grid, s, phi, lam, N, rx + (uint64_t)l * q->bmax, q->partials + col, ps, q->flag, f,
                               ta);
        col += gx;
        last_gx = gx;
        ++launches;
      }
      k_finalize_batch<<<B, kThreads, 0, s>>>(q->partials, col, ps, 2.0, q->results, out_stride, 1 + p + l);
      ++launches;
      if (fuse_out) {
        k_finalize_batch<<<B, kThreads, 0, s>>>(partials_g, (int)last_gx, ps, 2.0, q->results, out_stride, 1 + l);
        ++launches;
      } else {
        k_phase<TR, true><<<g_stream, kThreads, 0, s>>>(phi, lam, N, q->cut, tab_l, tsize, q->partials, ps, q->flag,
                                                        q->per_graph);
        k_finalize_batch<<<B, kThreads, 0, s>>>(q->partials, PB, ps, 2.0, q->results, out_stride, 1 + l);
        launches += 2;
      }
      if (renorm_after && fuse_rn) {
        k_finalize_batch<<<B, kThreads, 0, s>>>(q->partials + kNormCol, (int)last_gx, ps, 1.0, q->norms, 1, 0);
        k_finalize_batch<<<B, kThreads, 0, s>>>(q->partials + kNormCol + kRnCol, (int)last_gx, ps, 1.0,
                                                q->norms + 3 * q->bmax, 1, 0);
        launches += 2;
        scale_pending = true;
      } else if (renorm_after) {
        k_norm_batch<TR><<<g_stream, kThreads, 0, s>>>(phi, N, q->partials, ps, q->flag);
        k_finalize_batch<<<B, kThreads, 0, s>>>(q->partials, PB, ps, 1.0, q->norms, 1, 0);
        k_rescale<V><<<g_stream, kThreads, 0, s>>>(phi, N, q->norms, phi_norm);
        k_norm_batch<TR><<<g_stream, kThreads, 0, s>>>(lam, N, q->partials, ps, q->flag);
        k_finalize_batch<<<B, kThreads, 0, s>>>(q->partials, PB, ps, 1.0, q->norms, 1, 0);
        k_rescale<V><<<g_stream, kThreads, 0, s>>>(lam, N, q->norms, q->norms + q->bmax);
        launches += 6;
      }
    }
  }
  k_divide_results<<<B, 32, 0, s>>>(q->results, out_stride, grad ? 1 + 2 * p : 1, phi_norm);
  ++launches;
  *n_launches = launches;
  return cudaGetLastError();
}

// ---------------------------------------------------------------- chained-segment schedule (host)
struct HostOp {
  uint8_t kind;
  int layer;
  int geo;  // mixer pass index (RX only)
  int sub;  // position of the pass within its layer (RX only)
};

struct HostSeg {
  int geo = -1;
  bool adj_in = false;
  bool has_turn = false;
  std::vector<HostOp> ops;
};

// The evaluation as one operation list cut into segments of one geometry each
// (see k_seg).  Layer l visits passes 0..m-1 when l is even, m-1..0 when odd.
std::vector<HostSeg> chain_segments(int m, int p, bool grad) {
  std::vector<HostOp> fwd;
  for (int l = 0; l < p; ++l) {
    fwd.push_back(HostOp{kOpPhase, l, -1, 0});
    for (int j = 0; j < m; ++j) fwd.push_back(HostOp{kOpRX, l, (l % 2 == 0) ? j : m - 1 - j, j});
  }
  std::vector<HostOp> ops = fwd;
  ops.push_back(HostOp{grad ? kOpTurn : kOpEnergy, p - 1, -1, 0});
  if (grad)
    for (int i = (int)fwd.size() - 1; i >= 0; --i) ops.push_back(fwd[i]);
  std::vector<HostSeg> segs;
  bool adj = false;
  for (const HostOp& o : ops) {
    if (segs.empty() || (o.kind == kOpRX && segs.back().geo >= 0 && segs.back().geo != o.geo)) {
      segs.push_back(HostSeg());
      segs.back().adj_in = adj;
    }
    if (o.kind == kOpRX && segs.back().geo < 0) segs.back().geo = o.geo;
    segs.back().ops.push_back(o);
    if (o.kind == kOpTurn) {
      adj = true;
      segs.back().has_turn = true;
    }
  }
  return segs;
}

// Partial column blocks per state: beta sums of layer l, pass j at l m + j;
// gamma sums of layer l at p m + l; energy, |phi|^2, |lambda|^2 at p (m + 1)
// + 0..2; the stored norms of the renormalisation at p (m + 1) + 3, 4.
inline int chain_cols(int m, int p) { return p * (m + 1) + 5; }

bool chain_available(const iqs_qaoa* q) {
  if (q->passes.empty()) return false;
  for (const Geo& g : q->passes) {
    const bool ok = q->dtype == IQS_C128 ? fast_shape<T128>(g) : fast_shape<T64>(g);
    if (!ok) return false;
  }
  return true;
}

template <class TR, int MODE, int C>
void launch_merged1(dim3 grid, size_t smem, cudaStream_t s, typename TR::V* phi, typename TR::V* lam, uint64_t N,
                    int sb, const typename TR::RX* rxA, const typename TR::RX* rxB, int ps, unsigned* flag,
                    const uint8_t* cut, const typename TR::PH* tab, int tsize, int per_graph, const MergedOut& out) {
  k_mixer_merged<TR, C, MODE><<<grid, kThreads, smem, s>>>(phi, lam, N, sb, rxA, rxB, ps, flag, cut, tab, tsize,
                                                           per_graph, out);
}

template <class TR, int MODE, int... Cs>
void dispatch_merged(int c, dim3 grid, size_t smem, cudaStream_t s, typename TR::V* phi, typename TR::V* lam,
                     uint64_t N, int sb, const typename TR::RX* rxA, const typename TR::RX* rxB, int ps,
                     unsigned* flag, const uint8_t* cut, const typename TR::PH* tab, int tsize, int per_graph,
                     const MergedOut& out, std::integer_sequence<int, Cs...>) {
  if (c == 0) {
    launch_merged1<TR, MODE, 0>(grid, smem, s, phi, lam, N, sb, rxA, rxB, ps, flag, cut, tab, tsize, per_graph, out);
    return;
  }
  bool done = false;
  ((c == Cs + TR::kRowBits && !done
        ? (launch_merged1<TR, MODE, Cs + TR::kRowBits>(grid, smem, s, phi, lam, N, sb, rxA, rxB, ps, flag, cut, tab,
                                                       tsize, per_graph, out),
           done = true)
        : false),
   ...);
}

template <class TR, int MODE, int... Cs>
cudaError_t set_merged_attrs_c(int bytes, std::integer_sequence<int, Cs...>) {
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(k_mixer_merged<TR, 0, MODE>, a, bytes);
  ((e = e == cudaSuccess ? cudaFuncSetAttribute(k_mixer_merged<TR, Cs + TR::kRowBits, MODE>, a, bytes) : e), ...);
  return e;
}

template <class TR, bool ANYADJ, int C>
void launch_seg1(dim3 grid, size_t smem, cudaStream_t s, typename TR::V* phi, typename TR::V* lam, uint64_t N, int sb,
                 const typename TR::RX* rx, const typename TR::PH* tab, const uint8_t* cut, double* partials, int ps,
                 const double* norms, unsigned* flag, const SegParams& P) {
  k_seg<TR, C, ANYADJ><<<grid, kThreads, smem, s>>>(phi, lam, N, sb, rx, tab, cut, partials, ps, norms, flag, P);
}

template <class TR, bool ANYADJ, int... Cs>
void dispatch_seg(int c, dim3 grid, size_t smem, cudaStream_t s, typename TR::V* phi, typename TR::V* lam, uint64_t N,
                  int sb, const typename TR::RX* rx, const typename TR::PH* tab, const uint8_t* cut, double* partials,
                  int ps, const double* norms, unsigned* flag, const SegParams& P, std::integer_sequence<int, Cs...>) {
  if (c == 0) {
    launch_seg1<TR, ANYADJ, 0>(grid, smem, s, phi, lam, N, sb, rx, tab, cut, partials, ps, norms, flag, P);
    return;
  }
  bool done = false;
  ((c == Cs + TR::kRowBits && !done
        ? (launch_seg1<TR, ANYADJ, Cs + TR::kRowBits>(grid, smem, s, phi, lam, N, sb, rx, tab, cut, partials, ps,
                                                     norms, flag, P),
           done = true)
        : false),
   ...);
}

template <class TR, bool ANYADJ, int... Cs>
cudaError_t set_seg_attrs_c(int bytes, std::integer_sequence<int, Cs...>) {
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(k_seg<TR, 0, ANYADJ>, a, bytes);
  ((e = e == cudaSuccess ? cudaFuncSetAttribute(k_seg<TR, Cs + TR::kRowBits, ANYADJ>, a, bytes) : e), ...);
  return e;
}

template <class TR>
cudaError_t set_seg_attrs() {
  const auto seq = std::make_integer_sequence<int, TR::kTileBits - TR::kRowBits>{};
  const int one = (1 << TR::kTileBits) * (int)sizeof(typename TR::W);
  cudaError_t e = set_seg_attrs_c<TR, false>(one, seq);
  if (e == cudaSuccess) e = set_seg_attrs_c<TR, true>(2 * one, seq);
  if (e == cudaSuccess) e = set_merged_attrs_c<TR, kMgMerged>(2 * one, seq);
  if (e == cudaSuccess) e = set_merged_attrs_c<TR, kMgLast>(2 * one, seq);
  if (e == cudaSuccess) e = set_merged_attrs_c<TR, kMgTurn>(2 * one, seq);
  return e;
}

// Enqueue one evaluation on the chained schedule.  Segments of one RX, and
// merged [RX, phase, RX] segments, run on the tuned pass kernels (TMA-staged
// forward tiles, adjoint tiles with direct HBM rounds); the first segment,
// the turnaround, the last segment and the renormalising ones run on k_seg.
template <class TR>
cudaError_t enqueue_chain(iqs_qaoa* q, int B, int p, bool grad, int* n_launches) {
  using V = typename TR::V;
  const uint64_t N = q->N;
  cudaStream_t s = q->stream;
  V* phi = (V*)q->phi;
  V* lam = (V*)q->lam;
  const auto* rx = (const typename TR::RX*)q->rx;
  const auto* tab = (const typename TR::PH*)q->tables;
  const int m = (int)q->passes.size();
  const uint64_t tiles = N >> TR::kTileBits;
  const int gx = (int)std::min<uint64_t>(tiles, (uint64_t)blocks_per_state(q, B));
  const int ncols = chain_cols(m, p);
  const int ps = gx * ncols;
  if ((size_t)B * ps > q->partials_cap) return cudaErrorInvalidValue;
  const int out_stride = 1 + 2 * kMaxP;
  const int E0 = p * (m + 1);  // energy column block
  const int R = grad ? q->renorm_every : 0;
  double* phi_norm = q->norms + 2 * q->bmax;
  std::vector<HostSeg> segs = chain_segments(m, p, grad);
  const int S = (int)segs.size();
  // renormalisation (gradient runs, more than one segment): after the adjoint
  // phase of layer l > 0 with (p - l) % R == 0 the segment holding that phase
  // sums the norms of what it stores and the next segment rescales on load
  std::vector<int> rn_sum(S, 0);
  if (R > 0 && S > 1)
    for (int i = 0; i + 1 < S; ++i)
      if (segs[i].adj_in)  // with more than one segment, adjoint phases sit only in such segments
        for (const HostOp& o : segs[i].ops)
          if (o.kind == kOpPhase && o.layer > 0 && ((p - o.layer) % R) == 0) rn_sum[i] = 1;
  int launches = 0;
  const dim3 grid(gx, B);
  for (int i = 0; i < S; ++i) {
    const HostSeg& sg = segs[i];
    const Geo& g = q->passes[sg.geo];
    SegParams P;
    std::memset(&P, 0, sizeof(P));
    P.nops = (int)sg.ops.size();
    P.bmax = q->bmax;
    P.tsize = q->n_edges + 1;
    P.per_graph = q->per_graph;
    P.rn_stride = q->bmax;
    P.rn_col = E0 + 3;
    P.amp64 = std::pow(2.0, -q->n / 2.0);
    P.amp = (float)P.amp64;
    const bool last = i + 1 == S;
    const bool anyadj = sg.adj_in || sg.has_turn;
    uint32_t fl = 0;
    if (i == 0) fl |= kSegGen;
    if (sg.adj_in) fl |= kSegAdjIn;
    if (!grad || (!anyadj) || (sg.adj_in && !last)) fl |= kSegStorePhi;
    if (grad && anyadj && !last) fl |= kSegStoreLam;
    if (i > 0 && rn_sum[i - 1]) fl |= kSegRnScale;
    if (rn_sum[i]) fl |= kSegRnSum;
    P.flags = fl;
    bool adj = sg.adj_in;
    int nred = 0;
    for (int o = 0; o < P.nops; ++o) {
      const HostOp& h = sg.ops[o];
      SegOp so;
      so.kind = h.kind;
      so.layer = (uint8_t)h.layer;
      so.col = kNoCol;
      so.red = 0;
      so.pad = 0;
      int nv = 0;
      if (h.kind == kOpRX && adj) so.col = (uint16_t)(h.layer * m + h.sub), nv = 1;
      if (h.kind == kOpPhase && adj) so.col = (uint16_t)(p * m + h.layer), nv = 1;
      if (h.kind == kOpTurn) so.col = (uint16_t)E0, nv = 3;
      if (h.kind == kOpEnergy) so.col = (uint16_t)E0, nv = 2;
      if (h.kind == kOpTurn) adj = true;
      so.red = (uint8_t)std::min(nred, 255);
      nred += nv;
      P.ops[o] = so;
    }
    P.rn_red = nred;
    if (rn_sum[i]) nred += 2;
    if (nred > kSegRed) P.flags |= kSegTileSums;
    const size_t smem = (size_t)(anyadj ? 2 : 1) * ((size_t)1 << TR::kTileBits) * sizeof(typename TR::W);
    const auto seq = std::make_integer_sequence<int, TR::kTileBits - TR::kRowBits>{};
    const int nop = (int)sg.ops.size();
    const bool plain = (fl & (kSegGen | kSegRnScale | kSegRnSum)) == 0 && !sg.has_turn;
    const bool rn_ok = std::is_same<TR, T64>::value;  // fused renormalisation in the tuned kernels: complex64
    const bool no_gen = (fl & kSegGen) == 0;
    const bool single = nop == 1 && sg.ops[0].kind == kOpRX;
    const bool merged = nop == 3 && sg.ops[0].kind == kOpRX && sg.ops[1].kind == kOpPhase && sg.ops[2].kind == kOpRX;
    const bool turn3 = nop == 3 && sg.ops[0].kind == kOpRX && sg.ops[1].kind == kOpTurn && sg.ops[2].kind == kOpRX;
    const bool last2 = nop == 2 && sg.ops[0].kind == kOpRX && sg.ops[1].kind == kOpPhase;
    const size_t tsz = (size_t)(q->n_edges + 1);
    auto col = [&](int o) { return q->partials + (size_t)P.ops[o].col * gx; };
    TmaArgs ta;
    ta.use = q->tma_ok && q->tma_mode >= 1;
    ta.phi = &q->tm_phi[sg.geo];
    ta.lam = &q->tm_lam[sg.geo];
    ta.hi_bits = q->n - g.s - g.m;
    ta.err = q->tma_err;
    const typename TR::RX* rx0 = rx + (uint64_t)sg.ops[0].layer * q->bmax;
    const bool first2 = nop == 2 && sg.ops[0].kind == kOpPhase && sg.ops[1].kind == kOpRX;
    const bool energy2 = nop == 2 && sg.ops[0].kind == kOpRX && sg.ops[1].kind == kOpEnergy;
    if (plain && single && !sg.adj_in) {
      launch_mixer<TR, false>(g, grid, s, phi, nullptr, N, rx0, nullptr, 0, q->flag, PhaseFuse<TR>(), ta);
    } else if (ta.use && first2 && (fl & ~(uint32_t)(kSegGen | kSegStorePhi)) == 0 && (fl & kSegGen)) {
      PhaseFuse<TR> f;
      f.mode = 5;
      f.cut = q->cut;
      f.per_graph = q->per_graph;
      f.tables = tab + (uint64_t)sg.ops[0].layer * q->bmax * tsz;
      f.tsize = (int)tsz;
      f.amp0 = P.amp64;
      launch_mixer<TR, false>(g, grid, s, phi, nullptr, N, rx + (uint64_t)sg.ops[1].layer * q->bmax, nullptr, 0,
                              q->flag, f, ta);
    } else if (ta.use && energy2 && fl == kSegStorePhi) {
      PhaseFuse<TR> f;
      f.mode = 4;
      f.cut = q->cut;
      f.per_graph = q->per_graph;
      f.partials_g = q->partials + (size_t)(E0 + 1) * gx;
      launch_mixer<TR, false>(g, grid, s, phi, nullptr, N, rx0, q->partials + (size_t)E0 * gx, ps, q->flag, f, ta);
    } else if (single && sg.adj_in && !last && no_gen && (fl & kSegRnSum) == 0 &&
               ((fl & kSegRnScale) == 0 || rn_ok)) {
      PhaseFuse<TR> f;
      if (fl & kSegRnScale) {
        f.rn.norms = q->norms;
        f.rn.stride = q->bmax;
      }
      TmaArgs tadj = ta;
      tadj.use = q->tma_ok && q->tma_mode >= 2 && (fl & kSegRnScale) == 0;
      launch_mixer<TR, true>(g, grid, s, phi, lam, N, rx0, col(0), ps, q->flag, f, tadj);
    } else if (plain && merged && !sg.adj_in && ta.use) {
      PhaseFuse<TR> f;
      f.mode = 3;
      f.cut = q->cut;
      f.per_graph = q->per_graph;
      f.tables = tab + (uint64_t)sg.ops[1].layer * q->bmax * tsz;
      f.tsize = (int)tsz;
      f.rx2 = rx + (uint64_t)sg.ops[2].layer * q->bmax;
      launch_mixer<TR, false>(g, grid, s, phi, nullptr, N, rx0, nullptr, 0, q->flag, f, ta);
    } else if (merged && sg.adj_in && !last && no_gen && ((fl & (kSegRnScale | kSegRnSum)) == 0 || rn_ok)) {
      MergedOut mo;
      mo.pA = col(0);
      mo.pG = col(1);
      mo.pB = col(2);
      if (fl & kSegRnScale) {
        mo.rn.norms = q->norms;
        mo.rn.stride = q->bmax;
      }
      if (fl & kSegRnSum) {
        mo.pRnP = q->partials + (size_t)(E0 + 3) * gx;
        mo.pRnL = q->partials + (size_t)(E0 + 4) * gx;
      }
      dispatch_merged<TR, kMgMerged>(g.c, grid, smem, s, phi, lam, N, g.s, rx0,
                                     rx + (uint64_t)sg.ops[2].layer * q->bmax, ps, q->flag, q->cut,
                                     tab + (uint64_t)sg.ops[0].layer * q->bmax * tsz, (int)tsz, q->per_graph, mo, seq);
    } else if (last2 && sg.adj_in && last && no_gen && (fl & (kSegRnScale | kSegRnSum)) == 0) {
      MergedOut mo;
      mo.pA = col(0);
      mo.pG = col(1);
      dispatch_merged<TR, kMgLast>(g.c, grid, smem, s, phi, lam, N, g.s, rx0, rx0, ps, q->flag, q->cut,
                                   tab + (uint64_t)sg.ops[0].layer * q->bmax * tsz, (int)tsz, q->per_graph, mo, seq);
    } else if (turn3 && !sg.adj_in && !last && no_gen && (fl & (kSegRnScale | kSegRnSum)) == 0) {
      MergedOut mo;
      mo.pB = col(2);
      mo.pE = q->partials + (size_t)E0 * gx;
      mo.pN = q->partials + (size_t)(E0 + 1) * gx;
      mo.pL = q->partials + (size_t)(E0 + 2) * gx;
      dispatch_merged<TR, kMgTurn>(g.c, grid, smem, s, phi, lam, N, g.s, rx0, rx0, ps, q->flag, q->cut, tab,
                                   (int)tsz, q->per_graph, mo, seq);
    } else if (anyadj) {
      dispatch_seg<TR, true>(g.c, grid, smem, s, phi, lam, N, g.s, rx, tab, q->cut, q->partials, ps, q->norms,
                             q->flag, P, seq);
    } else {
      dispatch_seg<TR, false>(g.c, grid, smem, s, phi, lam, N, g.s, rx, tab, q->cut, q->partials, ps, q->norms,
                              q->flag, P, seq);
    }
    ++launches;
    if (sg.has_turn || (!grad && last)) {
      k_finalize_batch<<<B, kThreads, 0, s>>>(q->partials + (size_t)E0 * gx, gx, ps, 1.0, q->results, out_stride, 0);
      k_finalize_batch<<<B, kThreads, 0, s>>>(q->partials + (size_t)(E0 + 1) * gx, gx, ps, 1.0, phi_norm, 1, 0);
      launches += 2;
      if (sg.has_turn && R > 0) {  // |lambda|^2 at the turnaround: the target of later rescaling
        k_finalize_batch<<<B, kThreads, 0, s>>>(q->partials + (size_t)(E0 + 2) * gx, gx, ps, 1.0,
                                                q->norms + q->bmax, 1, 0);
        ++launches;
      }
    }
    if (rn_sum[i]) {
      k_finalize_batch<<<B, kThreads, 0, s>>>(q->partials + (size_t)(E0 + 3) * gx, gx, ps, 1.0, q->norms, 1, 0);
      k_finalize_batch<<<B, kThreads, 0, s>>>(q->partials + (size_t)(E0 + 4) * gx, gx, ps, 1.0,
                                              q->norms + 3 * q->bmax, 1, 0);
      launches += 2;
    }
  }
  if (grad) {
    for (int l = 0; l < p; ++l) {
      k_finalize_batch<<<B, kThreads, 0, s>>>(q->partials + (size_t)(l * m) * gx, m * gx, ps, 2.0, q->results,
                                              out_stride, 1 + p + l);
      k_finalize_batch<<<B, kThreads, 0, s>>>(q->partials + (size_t)(p * m + l) * gx, gx, ps, 2.0, q->results,
                                              out_stride, 1 + l);
      launches += 2;
    }
  }
  k_divide_results<<<B, 32, 0, s>>>(q->results, out_stride, grad ? 1 + 2 * p : 1, phi_norm);
  ++launches;
  *n_launches = launches;
  return cudaGetLastError();
}

// The chained schedule where it applies (every pass a full tile, partial sums
// allocated, not the cluster-resident energy engine), else one pass sequence per layer.
cudaError_t enqueue_any(iqs_qaoa* q, int B, int p, bool grad, int* n_launches) {
  const bool chain = q->schedule == 0 && chain_available(q) && !(!grad && use_cluster(q)) &&
                     (size_t)B * (size_t)std::min<uint64_t>(q->N >> (q->dtype == IQS_C128 ? T128::kTileBits
                                                                                         : T64::kTileBits),
                                                             (uint64_t)blocks_per_state(q, B)) *
                             chain_cols((int)q->passes.size(), p) <=
                         q->partials_cap;
  if (chain)
    return q->dtype == IQS_C128 ? enqueue_chain<T128>(q, B, p, grad, n_launches)
                                : enqueue_chain<T64>(q, B, p, grad, n_launches);
  return q->dtype == IQS_C128 ? enqueue<T128>(q, B, p, grad, n_launches) : enqueue<T64>(q, B, p, grad, n_launches);
}

// Device-side parameter tables (iqs_qaoa_run_async): the same FP64-built RX
// coefficients and exp(-i gamma k) tables as fill_params_c64/c128, from
// parameter arrays in device memory ([batch][p] each).  One thread per
// (layer, state, table entry); entry tsize holds the RX coefficients.
__device__ __forceinline__ void put_params(float2* rx, float2* tab, uint64_t i_rx, uint64_t i_tab, double be,
                                           double ga, int k, bool do_rx) {
  if (do_rx) rx[i_rx] = make_float2((float)cos(be), (float)sin(be));
  else tab[i_tab] = make_float2((float)cos(ga * k), (float)-sin(ga * k));
}
__device__ __forceinline__ void put_params(qops::RXc* rx, qops::Ph* tab, uint64_t i_rx, uint64_t i_tab, double be,
                                           double ga, int k, bool do_rx) {
  if (do_rx) {
    qops::RXc r;
    r.c = dfx::make_coef(cos(be));
    r.s = dfx::make_coef(sin(be));
    r.ns = dfx::make_coef(-sin(be));
    rx[i_rx] = r;
  } else {
    const double tr = cos(ga * k), ti = -sin(ga * k);
    qops::Ph t;
    t.tr = dfx::make_coef(tr);
    t.ti = dfx::make_coef(ti);
    t.nti = dfx::make_coef(-ti);
    tab[i_tab] = t;
  }
}

template <class TR>
__global__ void k_qaoa_params(const double* __restrict__ gam, const double* __restrict__ bet, int B, int p, int bmax,
                              int tsize, typename TR::RX* __restrict__ rx, typename TR::PH* __restrict__ tab) {
  const uint64_t total = (uint64_t)p * B * (tsize + 1);
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total; i += (uint64_t)gridDim.x * blockDim.x) {
    const int k = (int)(i % (tsize + 1));
    const uint64_t lb = i / (tsize + 1);
    const int b = (int)(lb % B), l = (int)(lb / B);
    const double be = bet[(uint64_t)b * p + l], ga = gam[(uint64_t)b * p + l];
    put_params(rx, tab, (uint64_t)l * bmax + b, ((uint64_t)l * bmax + b) * tsize + k, be, ga, k, k == tsize);
  }
}

// results[b][0 | 1 + l | 1 + p + l] -> energies[b], grad_gammas[b][l], grad_betas[b][l] (device arrays).
__global__ void k_scatter_results(const double* __restrict__ results, int stride, int B, int p,
                                  double* __restrict__ E, double* __restrict__ dg, double* __restrict__ db) {
  const int per = dg ? 1 + 2 * p : 1;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B * per; i += gridDim.x * blockDim.x) {
    const int b = i / per, j = i % per;
    const double v = results[(uint64_t)b * stride + j];
    if (j == 0) E[b] = v;
    else if (j <= p) dg[(uint64_t)b * p + j - 1] = v;
    else db[(uint64_t)b * p + j - 1 - p] = v;
  }
}

// Host-side parameters: RX(2 beta) coefficients and exp(-i gamma k) tables, FP64-built.
void fill_params_c64(iqs_qaoa* q, int B, int p, const double* gam, const double* bet) {
  float2* rx = (float2*)q->host_params;
  float2* tab = (float2*)(q->host_params + q->rx_bytes);
  const int tsize = q->n_edges + 1;
  for (int l = 0; l < p; ++l)
    for (int b = 0; b < B; ++b) {
      const double be = bet[(uint64_t)b * p + l], ga = gam[(uint64_t)b * p + l];
      rx[(uint64_t)l * q->bmax + b] = make_float2((float)std::cos(be), (float)std::sin(be));
      for (int k = 0; k < tsize; ++k)
        tab[((uint64_t)l * q->bmax + b) * tsize + k] = make_float2((float)std::cos(ga * k), (float)-std::sin(ga * k));
    }
}

void fill_params_c128(iqs_qaoa* q, int B, int p, const double* gam, const double* bet) {
  qops::RXc* rx = (qops::RXc*)q->host_params;
  qops::Ph* tab = (qops::Ph*)(q->host_params + q->rx_bytes);
  const int tsize = q->n_edges + 1;
  for (int l = 0; l < p; ++l)
    for (int b = 0; b < B; ++b) {
      const double be = bet[(uint64_t)b * p + l], ga = gam[(uint64_t)b * p + l];
      qops::RXc& r = rx[(uint64_t)l * q->bmax + b];
      r.c = dfx::make_coef(std::cos(be));
      r.s = dfx::make_coef(std::sin(be));
      r.ns = dfx::make_coef(-std::sin(be));
      for (int k = 0; k < tsize; ++k) {
        qops::Ph& t = tab[((uint64_t)l * q->bmax + b) * tsize + k];
        const double tr = std::cos(ga * k), ti = -std::sin(ga * k);
        t.tr = dfx::make_coef(tr);
        t.ti = dfx::make_coef(ti);
        t.nti = dfx::make_coef(-ti);
      }
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn tensor_map_encoder() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult res;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &res) ==
            cudaSuccess &&
        res == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(ptr);
    cudaGetLastError();
  });
  return fn;
}

// Tensor map of one mixer pass over ``bmax`` states of 2^n amplitudes at ``base``
// (8-byte units: a complex128 amplitude is two).  Low pass: [row, rows, tiles x B];
// high pass: [row, row blocks, mid bits, gate bits, high bits x B], box = one tile.
bool make_tile_map(CUtensorMap* m, void* base, const Geo& g, int n, int bmax, int amp_bytes, int K, int r0) {
  EncodeTiledFn enc = tensor_map_encoder();
  if (enc == nullptr) return false;
  const cuuint64_t eb = (cuuint64_t)amp_bytes, upa = (cuuint64_t)amp_bytes / 8;
  const cuuint32_t es[5] = {1, 1, 1, 1, 1};
  if (g.c == 0) {
    const cuuint64_t dims[3] = {(1ull << r0) * upa, 1ull << (K - r0), ((1ull << n) >> K) * (cuuint64_t)bmax};
    const cuuint64_t strides[2] = {(1ull << r0) * eb, (1ull << K) * eb};
    const cuuint32_t box[3] = {(cuuint32_t)((1u << r0) * upa), 1u << (K - r0), 1u};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  }
  const cuuint64_t dims[5] = {(1ull << r0) * upa, 1ull << (g.c - r0), 1ull << (g.s - g.c), 1ull << g.m,
                              (1ull << (n - g.s - g.m)) * (cuuint64_t)bmax};
  const cuuint64_t strides[4] = {(1ull << r0) * eb, (1ull << g.c) * eb, (1ull << g.s) * eb,
                                 (1ull << (g.s + g.m)) * eb};
  const cuuint32_t box[5] = {(cuuint32_t)((1u << r0) * upa), 1u << (g.c - r0), 1u, 1u << g.m, 1u};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 5, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void replan(iqs_qaoa* q) {
  const int K = q->dtype == IQS_C128 ? T128::kTileBits : T64::kTileBits;
  const int rows0 = q->dtype == IQS_C128 ? T128::kRowBits : T64::kRowBits;
  const int rows = q->row_bits < 0 ? rows0 : std::max(rows0, std::min(K - 1, q->row_bits));
  q->passes = plan_mixer(q->n, K, rows);
  for (auto& kv : q->graphs) cudaGraphExecDestroy(kv.second.first);
  q->graphs.clear();
  // the chained schedule's partial sums: B x blocks per state <= max(bmax, 4 x 2432) rows
  // of chain_cols(m, p) column blocks (a failed growth leaves that schedule unavailable)
  const size_t need = (size_t)std::max(q->bmax, 4 * 2432) * chain_cols((int)q->passes.size(), kMaxP);
  if (need > q->partials_cap) {
    double* grown = nullptr;
    if (cudaMalloc(&grown, sizeof(double) * need) == cudaSuccess) {
      cudaFree(q->partials);
      q->partials = grown;
      q->partials_cap = need;
    } else {
      cudaGetLastError();
    }
  }
  // tensor maps for the TMA-staged passes (full tiles only)
  const int amp = q->dtype == IQS_C128 ? 16 : 8;
  q->tm_phi.assign(q->passes.size(), CUtensorMap{});
  q->tm_lam.assign(q->passes.size(), CUtensorMap{});
  q->tma_ok = tensor_map_encoder() != nullptr;
  for (size_t i = 0; i < q->passes.size() && q->tma_ok; ++i) {
    const Geo& g = q->passes[i];
    if (g.c + g.m != K || (g.c != 0 && g.c < rows0)) {
      q->tma_ok = false;
      break;
    }
    q->tma_ok = make_tile_map(&q->tm_phi[i], q->phi, g, q->n, q->bmax, amp, K, rows0) &&
                make_tile_map(&q->tm_lam[i], q->lam, g, q->n, q->bmax, amp, K, rows0);
  }
}

const char* dtype_name(int dtype) { return dtype == IQS_C128 ? "c128" : "c64"; }

// Tile-shape choices persisted by the autotuner:
// lines "qaoa <dtype> <n> <batch_max> <row_bits> <grid_mult> <tma_mode> <schedule>"
// (a line without the schedule field means the chained schedule).
void load_tuning(iqs_qaoa* q) {
  const char* path = std::getenv("IQS_AUTOTUNE_CACHE");
  if (path == nullptr) return;
  FILE* f = std::fopen(path, "r");
  if (f == nullptr) return;
  char line[256];
  while (std::fgets(line, sizeof(line), f)) {
    char kind[16], dt[8];
    int n, bm, rows, mult, tma, sched = 0;
    const int got = std::sscanf(line, "%15s %7s %d %d %d %d %d %d", kind, dt, &n, &bm, &rows, &mult, &tma, &sched);
    if (got >= 7 && std::strcmp(kind, "qaoa") == 0 && std::strcmp(dt, dtype_name(q->dtype)) == 0 && n == q->n &&
        bm == q->bmax && mult >= 1 && mult <= 4 && tma >= 0 && tma <= 2 && sched >= 0 && sched <= 1) {
      q->row_bits = rows;
      q->grid_mult = mult;  // the last matching line wins
      q->tma_mode = tma;
      q->schedule = sched;
    }
  }
  std::fclose(f);
}

void save_tuning(const iqs_qaoa* q) {
  const char* path = std::getenv("IQS_AUTOTUNE_CACHE");
  if (path == nullptr) return;
  FILE* f = std::fopen(path, "a");
  if (f == nullptr) return;
  std::fprintf(f, "qaoa %s %d %d %d %d %d %d\n", dtype_name(q->dtype), q->n, q->bmax, q->row_bits, q->grid_mult,
               q->tma_mode, q->schedule);
  std::fclose(f);
}

void free_qaoa(iqs_qaoa* q) {
  for (auto& kv : q->graphs) cudaGraphExecDestroy(kv.second.first);
  if (q->own_stream && q->stream) cudaStreamDestroy(q->stream);
  cudaFree(q->phi);
  cudaFree(q->lam);
  cudaFree(q->cut);
  cudaFree(q->rx);
  cudaFree(q->tables);
  cudaFree(q->partials);
  cudaFree(q->results);
  cudaFree(q->norms);
  cudaFree(q->flag);
  cudaFree(q->tma_err);
  if (q->host_params) cudaFreeHost(q->host_params);
  if (q->host_results) cudaFreeHost(q->host_results);
  delete q;
}

// One evaluation of the workspace's current parameter tables on its stream:
// the captured CUDA graph of this (batch, p, gradient, renormalisation) shape,
// captured on first use, or a direct enqueue.  Counts the kernels launched.
cudaError_t launch_evaluation(iqs_qaoa* q, int batch, int p, bool grad) {
  cudaStream_t s = q->stream;
  cudaError_t e = cudaSuccess;
  const auto key = std::make_tuple(batch, p, grad ? 1 : 0, q->renorm_every);
  int kernels = 0;
  if (q->use_graphs) {
    auto it = q->graphs.find(key);
    if (it == q->graphs.end()) {
      cudaGraph_t graph = nullptr;
      e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        const cudaError_t ee = enqueue_any(q, batch, p, grad, &kernels);
        e = cudaStreamEndCapture(s, &graph);
        if (ee != cudaSuccess) e = ee;
      }
      cudaGraphExec_t exec = nullptr;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (e != cudaSuccess) return e;
      it = q->graphs.emplace(key, std::make_pair(exec, kernels)).first;
    }
    kernels = it->second.second;
    e = cudaGraphLaunch(it->second.first, s);
  } else {
    e = enqueue_any(q, batch, p, grad, &kernels);
  }
  if (e == cudaSuccess) note_launches(kernels);
  return e;
}

}  // namespace
}  // namespace iqs

extern "C" {

iqs_status iqs_qaoa_run_async(iqs_qaoa* q, int batch, int p, const double* d_gammas, const double* d_betas,
                              double* d_energies, double* d_grad_gammas, double* d_grad_betas) {
  using namespace iqs;
  if (q == nullptr) return report(IQS_EINVAL, "handle is NULL");
  if (batch < 1 || batch > q->bmax) return report(IQS_EINVAL, "batch %d outside [1, %d]", batch, q->bmax);
  if (p < 1 || p > kMaxP) return report(IQS_EINVAL, "depth p = %d outside [1, %d]", p, kMaxP);
  if (!d_gammas || !d_betas || !d_energies) return report(IQS_EINVAL, "gammas, betas and energies must not be NULL");
  const bool grad = d_grad_gammas != nullptr || d_grad_betas != nullptr;
  if (grad && (!d_grad_gammas || !d_grad_betas)) return report(IQS_EINVAL, "give both gradient outputs or neither");
  if (fault_now(2)) return report(IQS_ECUDA, "iqs_qaoa_run_async: injected launch failure");
  cudaStream_t s = q->stream;
  const int tsize = q->n_edges + 1;
  const uint64_t work = (uint64_t)p * batch * (tsize + 1);
  if (q->dtype == IQS_C128)
    k_qaoa_params<T128><<<grid_for(work, 1, 4), kThreads, 0, s>>>(d_gammas, d_betas, batch, p, q->bmax, tsize,
                                                                  (qops::RXc*)q->rx, (qops::Ph*)q->tables);
  else
    k_qaoa_params<T64><<<grid_for(work, 1, 4), kThreads, 0, s>>>(d_gammas, d_betas, batch, p, q->bmax, tsize,
                                                                 (float2*)q->rx, (float2*)q->tables);
  cudaError_t e = launched(1);
  if (e == cudaSuccess) e = launch_evaluation(q, batch, p, grad);
  if (e == cudaSuccess) {
    const int stride = 1 + 2 * kMaxP;
    k_scatter_results<<<grid_for((uint64_t)batch * (1 + 2 * p), 1, 4), kThreads, 0, s>>>(
        q->results, stride, batch, p, d_energies, grad ? d_grad_gammas : nullptr, grad ? d_grad_betas : nullptr);
    e = launched(1);
  }
  if (e != cudaSuccess) return report(IQS_ECUDA, "QAOA asynchronous launch: %s", cudaGetErrorString(e));
  return IQS_OK;
}

iqs_status iqs_qaoa_synchronize(iqs_qaoa* q) {
  using namespace iqs;
  if (q == nullptr) return report(IQS_EINVAL, "handle is NULL");
  unsigned w[2] = {0, 0};
  cudaError_t e = cudaStreamSynchronize(q->stream);
  if (e == cudaSuccess) e = cudaMemcpy(&w[0], q->flag, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&w[1], q->tma_err, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return report(IQS_ECUDA, "QAOA synchronize: %s", cudaGetErrorString(e));
  if (w[1]) {
    cudaMemset(q->tma_err, 0, sizeof(unsigned));
    return report(IQS_ETIMEOUT, "a TMA tile load did not complete within its wait limit; results are invalid");
  }
  if (w[0]) {
    cudaMemset(q->flag, 0, sizeof(unsigned));
    return report(IQS_ERANGE, "an amplitude outside the emulated-FP64 range was met");
  }
  return IQS_OK;
}

iqs_status iqs_qaoa_create(int n, int dtype, int batch_max, int n_edges, const int32_t* edges, void* stream,
                           iqs_qaoa** out) {
  return iqs_qaoa_create_multi(n, dtype, 1, batch_max, n_edges, edges, stream, out);
}

iqs_status iqs_qaoa_create_multi(int n, int dtype, int n_graphs, int per_graph, int n_edges, const int32_t* edges,
                                 void* stream, iqs_qaoa** out) {
  using namespace iqs;
  if (out == nullptr) return report(IQS_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 2 || n > IQS_MAX_QUBITS) return report(IQS_EINVAL, "number of qubits %d outside [2, %d]", n, IQS_MAX_QUBITS);
  if (dtype != IQS_C64 && dtype != IQS_C128) return report(IQS_EINVAL, "dtype must be IQS_C64 or IQS_C128");
  if (n_graphs < 1 || per_graph < 1 || (int64_t)n_graphs * per_graph > 65535)
    return report(IQS_EINVAL, "n_graphs %d x per_graph %d outside [1, 65535]", n_graphs, per_graph);
  const int batch_max = n_graphs * per_graph;
  if (n_edges < 1 || n_edges > kEdgeChunk || edges == nullptr)
    return report(IQS_EINVAL, "n_edges %d outside [1, %d] or edges NULL", n_edges, kEdgeChunk);
  for (int e = 0; e < n_graphs * n_edges; ++e) {
    const int u = edges[2 * e], v = edges[2 * e + 1];
    if (u < 0 || u >= n || v < 0 || v >= n || u == v)
      return report(IQS_EINVAL, "edge %d of graph %d = (%d, %d) invalid for %d qubits", e % n_edges, e / n_edges, u,
                    v, n);
  }
  if (fault_now(1)) return report(IQS_ENOMEM, "injected allocation failure");
  iqs_qaoa* q = new (std::nothrow) iqs_qaoa();
  if (q == nullptr) return report(IQS_ENOMEM, "host allocation failed");
  q->n = n;
  q->dtype = dtype;
  q->bmax = batch_max;
  q->n_edges = n_edges;
  q->n_graphs = n_graphs;
  q->per_graph = n_graphs == 1 ? (1 << 30) : per_graph;
  q->N = 1ull << n;
  q->stream = (cudaStream_t)stream;
  if (q->stream == nullptr) {  // graphs cannot be captured on the legacy stream: use a blocking stream of our own
    if (cudaStreamCreate(&q->stream) != cudaSuccess) {
      cudaGetLastError();
      delete q;
      return report(IQS_ECUDA, "cannot create a stream");
    }
    q->own_stream = true;
  }
  const size_t amp = dtype == IQS_C128 ? 16 : 8;
  const size_t tsize = (size_t)n_edges + 1;
  q->rx_bytes = (size_t)kMaxP * batch_max * (dtype == IQS_C128 ? sizeof(qops::RXc) : sizeof(float2));
  q->rx_bytes = (q->rx_bytes + 255) & ~(size_t)255;
  q->table_bytes = (size_t)kMaxP * batch_max * tsize * (dtype == IQS_C128 ? sizeof(qops::Ph) : sizeof(float2));
  const int ps = part_stride_for(q);
  bool ok = cudaMalloc(&q->phi, amp * q->N * batch_max) == cudaSuccess &&
            cudaMalloc(&q->lam, amp * q->N * batch_max) == cudaSuccess &&
            cudaMalloc(&q->cut, q->N * (size_t)n_graphs) == cudaSuccess && cudaMalloc(&q->rx, q->rx_bytes) == cudaSuccess &&
            cudaMalloc(&q->tables, q->table_bytes) == cudaSuccess &&
            cudaMalloc(&q->partials, sizeof(double) * (size_t)ps * batch_max) == cudaSuccess &&
            ((q->partials_cap = (size_t)ps * batch_max), true) &&
            cudaMalloc(&q->results, sizeof(double) * (size_t)batch_max * (1 + 2 * kMaxP)) == cudaSuccess &&
            cudaMalloc(&q->norms, sizeof(double) * 4 * (size_t)batch_max) == cudaSuccess &&
            cudaMalloc(&q->flag, sizeof(unsigned)) == cudaSuccess &&
            cudaMalloc(&q->tma_err, sizeof(unsigned)) == cudaSuccess &&
            cudaMallocHost(&q->host_params, q->rx_bytes + q->table_bytes) == cudaSuccess &&
            cudaMallocHost(&q->host_results, sizeof(double) * ((size_t)batch_max * (1 + 2 * kMaxP) + 1)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_qaoa(q);
    return report(IQS_ENOMEM, "cannot allocate the QAOA workspace (%d states of %d qubits)", batch_max, n);
  }
  cudaError_t e = cudaSuccess;
  for (int gi = 0; gi < n_graphs && e == cudaSuccess; ++gi) {
    EdgesU8 E;
    E.m = n_edges;
    const int32_t* eg = edges + (size_t)2 * n_edges * gi;
    for (int k = 0; k < n_edges; ++k) {
      E.u[k] = (uint8_t)eg[2 * k];
      E.v[k] = (uint8_t)eg[2 * k + 1];
    }
    uint8_t* cg = q->cut + q->N * (size_t)gi;
    if (n <= 32)
      k_cut_table<uint32_t><<<grid_for(q->N, 1, 16), kThreads, 0, q->stream>>>(cg, q->N, E);
    else
      k_cut_table<uint64_t><<<grid_for(q->N, 1, 16), kThreads, 0, q->stream>>>(cg, q->N, E);
    e = cudaGetLastError();
    if (e == cudaSuccess) note_launches(1);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(q->flag, 0, sizeof(unsigned), q->stream);
  if (e == cudaSuccess) e = dtype == IQS_C128 ? set_smem_attrs<T128>() : set_smem_attrs<T64>();
  if (e == cudaSuccess) e = dtype == IQS_C128 ? set_tma_attrs<T128>() : set_tma_attrs<T64>();
  if (e == cudaSuccess) e = dtype == IQS_C128 ? set_seg_attrs<T128>() : set_seg_attrs<T64>();
  if (e == cudaSuccess) e = cudaMemsetAsync(q->tma_err, 0, sizeof(unsigned), q->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(q->stream);
  if (e != cudaSuccess) {
    free_qaoa(q);
    return report(IQS_ECUDA, "QAOA set-up: %s", cudaGetErrorString(e));
  }
  load_tuning(q);
  replan(q);
  if (dtype == IQS_C64) q->cclusters = qaoa_cluster_setup(n, &q->clogc);
  *out = q;
  return IQS_OK;
}

iqs_status iqs_qaoa_info(const iqs_qaoa* q, int* n, int* dtype, int* n_graphs, int* per_graph, int* n_edges) {
  if (q == nullptr) return iqs::report(IQS_EINVAL, "handle is NULL");
  if (n) *n = q->n;
  if (dtype) *dtype = q->dtype;
  if (n_graphs) *n_graphs = q->n_graphs;
  if (per_graph) *per_graph = q->n_graphs == 1 ? q->bmax : q->per_graph;
  if (n_edges) *n_edges = q->n_edges;
  return IQS_OK;
}

iqs_status iqs_qaoa_max_cut(iqs_qaoa* q, double* out) {
  using namespace iqs;
  if (q == nullptr || out == nullptr) return report(IQS_EINVAL, "handle or out is NULL");
  unsigned* d = nullptr;
  if (cudaMallocAsync(&d, sizeof(unsigned) * q->n_graphs, q->stream) != cudaSuccess) {
    cudaGetLastError();
    return report(IQS_ENOMEM, "cannot allocate %d words", q->n_graphs);
  }
  std::vector<unsigned> h(q->n_graphs);
  cudaError_t e = cudaMemsetAsync(d, 0, sizeof(unsigned) * q->n_graphs, q->stream);
  if (e == cudaSuccess) {
    const dim3 grid((unsigned)std::min<uint64_t>(std::max<uint64_t>(1, q->N / (kThreads * 8)), 2 * kSMs), q->n_graphs);
    k_cut_max<<<grid, kThreads, 0, q->stream>>>(q->cut, q->N, d);
    e = cudaGetLastError();
    if (e == cudaSuccess) note_launches(1);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d, sizeof(unsigned) * q->n_graphs, cudaMemcpyDeviceToHost, q->stream);
  cudaFreeAsync(d, q->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(q->stream);
  if (e != cudaSuccess) return report(IQS_ECUDA, "max cut: %s", cudaGetErrorString(e));
  for (int g = 0; g < q->n_graphs; ++g) out[g] = (double)h[g];
  return IQS_OK;
}

iqs_status iqs_qaoa_destroy(iqs_qaoa* q) {
  if (q == nullptr) return IQS_OK;
  cudaStreamSynchronize(q->stream);
  iqs::free_qaoa(q);
  return IQS_OK;
}

iqs_status iqs_qaoa_set_options(iqs_qaoa* q, int renorm_every, int use_graphs) {
  if (q == nullptr) return iqs::report(IQS_EINVAL, "handle is NULL");
  if (renorm_every < 0) return iqs::report(IQS_EINVAL, "renorm_every must be >= 0");
  q->renorm_every = renorm_every;
  q->use_graphs = use_graphs != 0;
  return IQS_OK;
}

iqs_status iqs_qaoa_set_engine(iqs_qaoa* q, int engine) {
  using namespace iqs;
  if (q == nullptr) return report(IQS_EINVAL, "handle is NULL");
  if (engine < 0 || engine > 2) return report(IQS_EINVAL, "engine must be 0 (auto), 1 (tiled) or 2 (cluster)");
  if (engine == 2 && !(q->clogc >= 0 && q->cclusters > 0))
    return report(IQS_EINVAL, "the cluster-resident forward takes complex64 states of 8..18 qubits on this device");
  if (engine != q->engine) {  // captured graphs embed the engine's kernels
    cudaStreamSynchronize(q->stream);
    for (auto& kv : q->graphs) cudaGraphExecDestroy(kv.second.first);
    q->graphs.clear();
  }
  q->engine = engine;
  return IQS_OK;
}

iqs_status iqs_qaoa_run(iqs_qaoa* q, int batch, int p, const double* gammas, const double* betas, double* energies,
                        double* grad_gammas, double* grad_betas) {
  using namespace iqs;
  if (q == nullptr) return report(IQS_EINVAL, "handle is NULL");
  if (batch < 1 || batch > q->bmax) return report(IQS_EINVAL, "batch %d outside [1, %d]", batch, q->bmax);
  if (p < 1 || p > kMaxP) return report(IQS_EINVAL, "depth p = %d outside [1, %d]", p, kMaxP);
  if (!gammas || !betas || !energies) return report(IQS_EINVAL, "gammas, betas and energies must not be NULL");
  const bool grad = grad_gammas != nullptr || grad_betas != nullptr;
  if (grad && (!grad_gammas || !grad_betas)) return report(IQS_EINVAL, "give both gradient outputs or neither");
  for (int i = 0; i < batch * p; ++i)
    if (!std::isfinite(gammas[i]) || !std::isfinite(betas[i])) return report(IQS_EINVAL, "non-finite parameter");
  if (fault_now(2)) return report(IQS_ECUDA, "iqs_qaoa_run: injected launch failure");
  if (q->dtype == IQS_C128) fill_params_c128(q, batch, p, gammas, betas);
  else fill_params_c64(q, batch, p, gammas, betas);
  cudaStream_t s = q->stream;
  const size_t rx_elem = q->dtype == IQS_C128 ? sizeof(qops::RXc) : sizeof(float2);
  const size_t ph_elem = q->dtype == IQS_C128 ? sizeof(qops::Ph) : sizeof(float2);
  cudaError_t e = cudaMemcpyAsync(q->rx, q->host_params, (size_t)p * q->bmax * rx_elem, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(q->tables, q->host_params + q->rx_bytes, (size_t)p * q->bmax * (q->n_edges + 1) * ph_elem,
                        cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return report(IQS_ECUDA, "parameter upload: %s", cudaGetErrorString(e));
  e = launch_evaluation(q, batch, p, grad);
  if (e != cudaSuccess) return report(IQS_ECUDA, "QAOA launch: %s", cudaGetErrorString(e));
  const int stride = 1 + 2 * kMaxP;
  e = cudaMemcpyAsync(q->host_results, q->results, sizeof(double) * (size_t)batch * stride, cudaMemcpyDeviceToHost, s);
  unsigned f = 0, terr = 0;
  double* flag_slot = q->host_results + (size_t)q->bmax * stride;
  if (e == cudaSuccess) e = cudaMemcpyAsync(flag_slot, q->flag, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(reinterpret_cast<unsigned*>(flag_slot) + 1, q->tma_err, sizeof(unsigned),
                        cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return report(IQS_ECUDA, "QAOA results: %s", cudaGetErrorString(e));
  std::memcpy(&f, flag_slot, sizeof(unsigned));
  std::memcpy(&terr, reinterpret_cast<unsigned*>(flag_slot) + 1, sizeof(unsigned));
  if (terr) {
    cudaMemsetAsync(q->tma_err, 0, sizeof(unsigned), s);
    return report(IQS_ETIMEOUT, "a TMA tile load did not complete within its wait limit; results are invalid");
  }
  for (int b = 0; b < batch; ++b) {
    const double* r = q->host_results + (size_t)b * stride;
    energies[b] = r[0];
    if (grad)
      for (int l = 0; l < p; ++l) {
        grad_gammas[(size_t)b * p + l] = r[1 + l];
        grad_betas[(size_t)b * p + l] = r[1 + p + l];
      }
  }
  if (f) {
    cudaMemsetAsync(q->flag, 0, sizeof(unsigned), s);
    return report(IQS_ERANGE, "an amplitude outside the emulated-FP64 range was met");
  }
  return IQS_OK;
}

iqs_status iqs_qaoa_autotune(iqs_qaoa* q, int batch, int p, double* best_ms) {
  using namespace iqs;
  if (q == nullptr) return report(IQS_EINVAL, "handle is NULL");
  if (batch < 1 || batch > q->bmax || p < 1 || p > kMaxP) return report(IQS_EINVAL, "bad batch or depth");
  std::vector<double> g((size_t)batch * p, 0.3), b((size_t)batch * p, 0.2), E(batch), dg((size_t)batch * p),
      db((size_t)batch * p);
  const int rows0 = q->dtype == IQS_C128 ? T128::kRowBits : T64::kRowBits;
  const bool graphs = q->use_graphs;
  q->use_graphs = false;
  double best = 1e300;
  int best_rows = rows0, best_mult = 1;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return report(IQS_ECUDA, "autotune events");
  iqs_status st = IQS_OK;
  auto time_one = [&](float* ms) -> iqs_status {
    replan(q);
    iqs_status r = iqs_qaoa_run(q, batch, p, g.data(), b.data(), E.data(), dg.data(), db.data());  // warm
    if (r != IQS_OK) return r;
    cudaEventRecord(e0, q->stream);
    r = iqs_qaoa_run(q, batch, p, g.data(), b.data(), E.data(), dg.data(), db.data());
    cudaEventRecord(e1, q->stream);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(ms, e0, e1);
    return r;
  };
  // 1) pass schedule and TMA staging at the default shape: the chained schedule
  //    (forward tiles TMA-staged when available) against the per-layer schedule
  //    with staging off / forward / forward + adjoint
  int best_tma = 0, best_sched = 0;
  q->row_bits = rows0;
  q->grid_mult = 1;
  const int sched0 = q->schedule;
  for (int sched = 0; sched <= 1 && st == IQS_OK; ++sched) {
    q->schedule = sched;
    if (sched == 0 && !chain_available(q)) continue;
    for (int tma = sched == 0 ? 1 : 0; tma <= (sched == 0 ? 1 : 2) && st == IQS_OK; ++tma) {
      q->tma_mode = tma;
      float ms = 0.f;
      st = time_one(&ms);
      if (st == IQS_OK && ms < best) {
        best = ms;
        best_tma = tma;
        best_sched = sched;
      }
      if (!q->tma_ok) break;  // no tensor maps here: staging unavailable
    }
  }
  (void)sched0;
  q->schedule = best_sched;
  q->tma_mode = best_tma;
  // 2) high-pass row width and grid size with that staging
  for (int rows = rows0; rows <= rows0 + 2 && st == IQS_OK; ++rows) {
    for (int mult = 1; mult <= 2 && st == IQS_OK; ++mult) {
      if (rows == rows0 && mult == 1) continue;  // measured above
      q->row_bits = rows;
      q->grid_mult = mult;
      float ms = 0.f;
      st = time_one(&ms);
      if (st == IQS_OK && ms < best) {
        best = ms;
        best_rows = rows;
        best_mult = mult;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  q->row_bits = best_rows;
  q->grid_mult = best_mult;
  replan(q);
  q->use_graphs = graphs;
  if (st != IQS_OK) return st;
  save_tuning(q);
  if (best_ms) *best_ms = best;
  return IQS_OK;
}

iqs_status iqs_qaoa_set_schedule(iqs_qaoa* q, int schedule) {
  if (q == nullptr) return iqs::report(IQS_EINVAL, "handle is NULL");
  if (schedule < 0 || schedule > 1) return iqs::report(IQS_EINVAL, "schedule must be 0 or 1");
  q->schedule = schedule;
  iqs::replan(q);
  return IQS_OK;
}

iqs_status iqs_qaoa_get_schedule(const iqs_qaoa* q, int* schedule, int* chained_available) {
  if (q == nullptr) return iqs::report(IQS_EINVAL, "handle is NULL");
  if (schedule) *schedule = q->schedule;
  if (chained_available) *chained_available = iqs::chain_available(q) ? 1 : 0;
  return IQS_OK;
}

iqs_status iqs_qaoa_set_tma(iqs_qaoa* q, int mode) {
  if (q == nullptr) return iqs::report(IQS_EINVAL, "handle is NULL");
  if (mode < 0 || mode > 2) return iqs::report(IQS_EINVAL, "TMA mode must be 0, 1 or 2");
  q->tma_mode = mode;
  iqs::replan(q);
  return IQS_OK;
}

iqs_status iqs_qaoa_get_tma(const iqs_qaoa* q, int* mode, int* available) {
  if (q == nullptr) return iqs::report(IQS_EINVAL, "handle is NULL");
  if (mode) *mode = q->tma_mode;
  if (available) *available = q->tma_ok ? 1 : 0;
  return IQS_OK;
}

iqs_status iqs_qaoa_tuning(const iqs_qaoa* q, int* row_bits, int* grid_mult) {
  if (q == nullptr) return iqs::report(IQS_EINVAL, "handle is NULL");
  const int rows0 = q->dtype == IQS_C128 ? iqs::T128::kRowBits : iqs::T64::kRowBits;
  if (row_bits) *row_bits = q->row_bits < 0 ? rows0 : q->row_bits;
  if (grid_mult) *grid_mult = q->grid_mult;
  return IQS_OK;
}

iqs_status iqs_qaoa_download_state(iqs_qaoa* q, int index, void* host, size_t bytes) {
  using namespace iqs;
  if (q == nullptr || host == nullptr) return report(IQS_EINVAL, "NULL argument");
  const size_t amp = q->dtype == IQS_C128 ? 16 : 8;
  if (index < 0 || index >= q->bmax || bytes != amp * q->N) return report(IQS_EINVAL, "bad index or size");
  cudaError_t e = cudaMemcpyAsync(host, (const char*)q->phi + amp * q->N * index, bytes, cudaMemcpyDeviceToHost, q->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(q->stream);
  if (e != cudaSuccess) return report(IQS_ECUDA, "download: %s", cudaGetErrorString(e));
  return IQS_OK;
}

}  // extern "C"
