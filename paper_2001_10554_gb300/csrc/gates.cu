// One-qubit and controlled one-qubit gates (Section 2, "Distributed
// implementation": the pair update alpha'_{..0_q..} = U00 alpha_{..0_q..} +
// U01 alpha_{..1_q..}, alpha'_{..1_q..} = U10 alpha_{..0_q..} + U11 alpha_{..1_q..}).
//
// Every kernel streams the state once: each thread takes pair indices k in a
// grid-stride loop, inserts the zero bit(s) in registers to get i0, reads the
// two amplitudes, applies U and writes them back in place.  Variants:
//   complex64   FP32 math; 128-bit loads of two consecutive amplitudes when
//               the lowest touched bit is >= 1, or of the whole pair when the
//               target is bit 0.
//   complex128  double-float emulation (df64.cuh) or native FP64.
//   monomial    matrices with entries in {0, +-1, +-i} and one nonzero per row
//               and column (X, Y, Z, S, CNOT, CZ ...): exact swaps and sign
//               flips, no rounding; a diagonal with U00 = 1 touches only the
//               |1>-half of the pairs.
#include "common.cuh"
#include "df64.cuh"
#include "internal.h"

namespace iqs {
namespace {

// ---------------------------------------------------------------- index maps
// One-qubit gate: pair k -> (insert_zero(k, q), + 2^q).
struct Map1 {
  int q;
  uint64_t off;
  __device__ __forceinline__ uint64_t i0(uint64_t k) const { return insert_zero(k, q); }
};
// Controlled gate: pair k -> (insert two zeros at lo < hi, then set the control bit), + 2^t.
struct Map2 {
  int lo, hi;
  uint64_t cbit, off;
  __device__ __forceinline__ uint64_t i0(uint64_t k) const { return insert_two_zeros(k, lo, hi) | cbit; }
};

// ---------------------------------------------------------------- complex64
struct GateF32 {
  float r[4], i[4];
};

__device__ __forceinline__ void apply_f32(const GateF32& u, float2 x0, float2 x1, float2& y0, float2& y1) {
  y0.x = u.r[0] * x0.x - u.i[0] * x0.y + u.r[1] * x1.x - u.i[1] * x1.y;
  y0.y = u.r[0] * x0.y + u.i[0] * x0.x + u.r[1] * x1.y + u.i[1] * x1.x;
  y1.x = u.r[2] * x0.x - u.i[2] * x0.y + u.r[3] * x1.x - u.i[3] * x1.y;
  y1.y = u.r[2] * x0.y + u.i[2] * x0.x + u.r[3] * x1.y + u.i[3] * x1.x;
}

// Two consecutive pairs per thread (lowest touched bit >= 1): pairs 2j and
// 2j+1 sit at i0, i0+1 and i1, i1+1 -> one float4 from each half.
template <class Map>
__global__ void __launch_bounds__(kThreads) k_c64_vec2(float2* __restrict__ a, uint64_t n_pairs2, Map m, GateF32 u) {
  for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < n_pairs2; j += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i0 = m.i0(2 * j);
    float4* p0 = reinterpret_cast<float4*>(a + i0);
    float4* p1 = reinterpret_cast<float4*>(a + i0 + m.off);
    const float4 v0 = *p0, v1 = *p1;
    float2 y00, y01, y10, y11;
    apply_f32(u, make_float2(v0.x, v0.y), make_float2(v1.x, v1.y), y00, y01);
    apply_f32(u, make_float2(v0.z, v0.w), make_float2(v1.z, v1.w), y10, y11);
    *p0 = make_float4(y00.x, y00.y, y10.x, y10.y);
    *p1 = make_float4(y01.x, y01.y, y11.x, y11.y);
  }
}

// Pair contiguous (target bit 0, control bit >= 1 or none): one float4 = (alpha_i0, alpha_i0+1).
template <class Map>
__global__ void __launch_bounds__(kThreads) k_c64_pairvec(float2* __restrict__ a, uint64_t n_pairs, Map m, GateF32 u) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < n_pairs; k += (uint64_t)gridDim.x * blockDim.x) {
    float4* p = reinterpret_cast<float4*>(a + m.i0(k));
    const float4 v = *p;
    float2 y0, y1;
    apply_f32(u, make_float2(v.x, v.y), make_float2(v.z, v.w), y0, y1);
    *p = make_float4(y0.x, y0.y, y1.x, y1.y);
  }
}

// General scalar form (control on bit 0).
template <class Map>
__global__ void __launch_bounds__(kThreads) k_c64_scalar(float2* __restrict__ a, uint64_t n_pairs, Map m, GateF32 u) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < n_pairs; k += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i0 = m.i0(k);
    const float2 x0 = a[i0], x1 = a[i0 + m.off];
    float2 y0, y1;
    apply_f32(u, x0, x1, y0, y1);
    a[i0] = y0;
    a[i0 + m.off] = y1;
  }
}

// ---------------------------------------------------------------- complex128, emulated
// Coefficients per output component (rows: out0.re, out0.im, out1.re,
// out1.im), each over the terms (x0.re, x0.im, x1.re, x1.im).
struct GateDF {
  dfx::Coef c[16];
};

template <class Map>
__global__ void __launch_bounds__(kThreads) k_c128_df(double2* __restrict__ a, uint64_t n_pairs, Map m, GateDF g,
                                                       unsigned* __restrict__ flag) {
  unsigned bad = 0;
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < n_pairs; k += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i0 = m.i0(k), i1 = i0 + m.off;
    const double2 x0 = a[i0], x1 = a[i1];
    float xh[4], xl[4];
    dfx::split(x0.x, xh[0], xl[0], bad);
    dfx::split(x0.y, xh[1], xl[1], bad);
    dfx::split(x1.x, xh[2], xl[2], bad);
    dfx::split(x1.y, xh[3], xl[3], bad);
    double y[4];
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      float p, e;
      dfx::dot<4>(&g.c[4 * o], xh, xl, p, e);
      y[o] = dfx::join(p, e);
    }
    a[i0] = make_double2(y[0], y[1]);
    a[i1] = make_double2(y[2], y[3]);
  }
  if (bad) atomicOr(flag, 1u);
}

// ---------------------------------------------------------------- complex128, native FP64
struct GateF64 {
  double r[4], i[4];
};

template <class Map>
__global__ void __launch_bounds__(kThreads) k_c128_native(double2* __restrict__ a, uint64_t n_pairs, Map m, GateF64 u) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < n_pairs; k += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i0 = m.i0(k), i1 = i0 + m.off;
    const double2 x0 = a[i0], x1 = a[i1];
    double2 y0, y1;
    y0.x = u.r[0] * x0.x - u.i[0] * x0.y + u.r[1] * x1.x - u.i[1] * x1.y;
    y0.y = u.r[0] * x0.y + u.i[0] * x0.x + u.r[1] * x1.y + u.i[1] * x1.x;
    y1.x = u.r[2] * x0.x - u.i[2] * x0.y + u.r[3] * x1.x - u.i[3] * x1.y;
    y1.y = u.r[2] * x0.y + u.i[2] * x0.x + u.r[3] * x1.y + u.i[3] * x1.x;
    a[i0] = y0;
    a[i1] = y1;
  }
}

// ---------------------------------------------------------------- monomial (exact)
template <class V, class Map>
__global__ void __launch_bounds__(kThreads) k_mono(V* __restrict__ a, uint64_t n_pairs, Map m, int perm, int k0, int k1,
                                                   int only1) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < n_pairs; k += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i0 = m.i0(k), i1 = i0 + m.off;
    if (only1) {
      a[i1] = mul_ipow(a[i1], k1);
      continue;
    }
    const V x0 = a[i0], x1 = a[i1];
    a[i0] = mul_ipow(perm ? x1 : x0, k0);
    a[i1] = mul_ipow(perm ? x0 : x1, k1);
  }
}

// ---------------------------------------------------------------- host helpers
GateF32 to_f32(const Mat2& u) {
  GateF32 g;
  for (int k = 0; k < 4; ++k) {
    g.r[k] = (float)u.re[k];
    g.i[k] = (float)u.im[k];
  }
  return g;
}

GateF64 to_f64(const Mat2& u) {
  GateF64 g;
  for (int k = 0; k < 4; ++k) {
    g.r[k] = u.re[k];
    g.i[k] = u.im[k];
  }
  return g;
}

GateDF to_df(const Mat2& u) {
  // out_row.re = Ur0.re x0.re - Ur0.im x0.im + Ur1.re x1.re - Ur1.im x1.im
  // out_row.im = Ur0.im x0.re + Ur0.re x0.im + Ur1.im x1.re + Ur1.re x1.im
  GateDF g;
  for (int row = 0; row < 2; ++row) {
    const int a = 2 * row, b = 2 * row + 1;
    const double re[4] = {u.re[a], -u.im[a], u.re[b], -u.im[b]};
    const double im[4] = {u.im[a], u.re[a], u.im[b], u.re[b]};
    for (int k = 0; k < 4; ++k) {
      g.c[8 * row + k] = dfx::make_coef(re[k]);
      g.c[8 * row + 4 + k] = dfx::make_coef(im[k]);
    }
  }
  return g;
}

int unit_power(double re, double im) {  // i^k == re + i im -> k, or -1
  if (re == 1.0 && im == 0.0) return 0;
  if (re == 0.0 && im == 1.0) return 1;
  if (re == -1.0 && im == 0.0) return 2;
  if (re == 0.0 && im == -1.0) return 3;
  return -1;
}

template <class Map>
cudaError_t dispatch(iqs_reg* r, uint64_t n_pairs, const Map& m, int lowest_bit, bool target_is_bit0,
                     const Mat2& u) {
  Mono mono;
  if (as_monomial(u, &mono)) {
    const bool diag = !mono.perm;
    if (diag && mono.k[0] == 0 && mono.k[1] == 0) return cudaSuccess;  // identity
    const int only1 = (diag && mono.k[0] == 0) ? 1 : 0;
    const unsigned grid = grid_for(n_pairs, 1, 32);
    if (r->dtype == IQS_C64)
      k_mono<float2, Map><<<grid, kThreads, 0, r->stream>>>((float2*)r->data, n_pairs, m, mono.perm, mono.k[0],
                                                            mono.k[1], only1);
    else
      k_mono<double2, Map><<<grid, kThreads, 0, r->stream>>>((double2*)r->data, n_pairs, m, mono.perm, mono.k[0],
                                                             mono.k[1], only1);
    return launched(1);
  }
  if (r->dtype == IQS_C64) {
    const GateF32 g = to_f32(u);
    if (lowest_bit >= 1 && n_pairs >= 2) {
      const uint64_t n2 = n_pairs / 2;
      k_c64_vec2<Map><<<grid_for(n2, 1, 32), kThreads, 0, r->stream>>>((float2*)r->data, n2, m, g);
    } else if (target_is_bit0) {
      k_c64_pairvec<Map><<<grid_for(n_pairs, 1, 32), kThreads, 0, r->stream>>>((float2*)r->data, n_pairs, m, g);
    } else {
      k_c64_scalar<Map><<<grid_for(n_pairs, 1, 32), kThreads, 0, r->stream>>>((float2*)r->data, n_pairs, m, g);
    }
    return launched(1);
  }
  if (use_emulated(r)) {
    k_c128_df<Map><<<grid_for(n_pairs, 1, 32), kThreads, 0, r->stream>>>((double2*)r->data, n_pairs, m, to_df(u),
                                                                          r->flag);
  } else {
    k_c128_native<Map><<<grid_for(n_pairs, 1, 32), kThreads, 0, r->stream>>>((double2*)r->data, n_pairs, m,
                                                                              to_f64(u));
  }
  return launched(1);
}

}  // namespace

bool as_monomial(const Mat2& u, Mono* m) {
  int k[4];
  bool zero[4];
  for (int e = 0; e < 4; ++e) {
    zero[e] = (u.re[e] == 0.0 && u.im[e] == 0.0);
    k[e] = unit_power(u.re[e], u.im[e]);
    if (!zero[e] && k[e] < 0) return false;
  }
  if (zero[1] && zero[2] && !zero[0] && !zero[3]) {
    m->perm = false;
    m->k[0] = k[0];
    m->k[1] = k[3];
    return true;
  }
  if (zero[0] && zero[3] && !zero[1] && !zero[2]) {
    m->perm = true;
    m->k[0] = k[1];
    m->k[1] = k[2];
    return true;
  }
  return false;
}

cudaError_t launch_1q(iqs_reg* r, int q, const Mat2& u) {
  const uint64_t n_pairs = num_amps(r) >> 1;
  Map1 m{q, 1ull << q};
  return dispatch(r, n_pairs, m, q, q == 0, u);
}

cudaError_t launch_c1q(iqs_reg* r, int c, int t, const Mat2& u) {
  const uint64_t n_pairs = num_amps(r) >> 2;
  const int lo = c < t ? c : t, hi = c < t ? t : c;
  Map2 m{lo, hi, 1ull << c, 1ull << t};
  return dispatch(r, n_pairs, m, lo, t == 0, u);
}

}  // namespace iqs
