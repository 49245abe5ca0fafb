// Double-float arithmetic for complex128 states on the FP32 pipe.
//
// GB300 (sm_103a) executes FP64 FMA, add and FP32<->FP64 conversion at about
// 2 operations per clock per SM, 1/64 of its FP32 rate; a native FP64
// one-qubit gate on a 2^30-amplitude state therefore reaches only ~30% of the
// HBM bandwidth.  These helpers keep the data in IEEE FP64 in memory but do
// the arithmetic with FP32 FMAs and integer bit operations only:
//
//   split : double x -> (h, l52) with x ~= h + l52 * 2^-52, h = x truncated to
//           24 significant bits, l52 the next bits (rounded to 24) scaled by
//           2^52 so that it stays a normal float.  Pure integer ops + one I2F.
//   dot   : sum_k c_k x_k of K real terms with error-free products
//           (FMA residuals) and TwoSum accumulation of the leading parts; the
//           small parts (residuals, cross products) go to a second float.
//   join  : (p + e) -> double with integer ops and one F2I, no FP64 ops.
//
// Range: inputs with |x| < 2^-80 are flushed to zero (absolute error below
// 1e-24); inputs with |x| >= 2^64, Inf or NaN raise the ``bad`` flag, which
// the caller turns into IQS_ERANGE.  Relative error per gate output is about
// 2^-45 of the largest input of the pair.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace iqs {
namespace dfx {

// One real coefficient c = h + l (h = fl32(c)); h52 = h * 2^-52 multiplies
// the 2^52-scaled low parts produced by split().
struct Coef {
  float h, l, h52;
};

__host__ __device__ inline Coef make_coef(double c) {
  Coef r;
  r.h = (float)c;
  r.l = (float)(c - (double)r.h);
  r.h52 = (float)((double)r.h * 0x1p-52);
  return r;
}

// Exponent window accepted without flushing: biased FP64 exponent E in
// [kEmin, kEmax) <=> 2^-80 <= |x| < 2^64.
constexpr unsigned kEmin = 943u;
constexpr unsigned kEmax = 1087u;

__device__ __forceinline__ void split(double x, float& h, float& l52, unsigned& bad) {
  const unsigned lo = (unsigned)__double2loint(x);
  const unsigned hi = (unsigned)__double2hiint(x);
  // (hi:lo) << 3 puts the top 23 fraction bits at bits 0..22 and the low 8
  // exponent bits at 23..30; adding 128 << 23 rebiases the exponent from
  // 1023 to 127 modulo 256, exact inside the accepted window.
  const unsigned t = __funnelshift_l(lo, hi, 3) + 0x40000000u;
  unsigned hb = (t & 0x7fffffffu) | (hi & 0x80000000u);
  const unsigned e = hi & 0x7ff00000u;
  hb = (e - (kEmin << 20)) < ((kEmax - kEmin) << 20) ? hb : 0u;
  bad |= (e >= (kEmax << 20)) ? 1u : 0u;
  h = __uint_as_float(hb);
  // remainder: low 29 fraction bits times 2^(E-1075) = (that integer) * 2^(E-1023) * 2^-52
  l52 = __uint2float_rn(lo & 0x1fffffffu) * __uint_as_float(hb & 0xff800000u);
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& err) {
  s = a + b;
  const float bb = s - a;
  err = (a - (s - bb)) + (b - bb);
}

// p + e ~= sum_{k<K} c_k * x_k  with x_k = xh_k + xl_k * 2^-52.
template <int K>
__device__ __forceinline__ void dot(const Coef* c, const float* xh, const float* xl, float& p, float& e) {
  p = c[0].h * xh[0];
  e = fmaf(c[0].h, xh[0], -p);
  e = fmaf(c[0].h52, xl[0], e);
  e = fmaf(c[0].l, xh[0], e);
#pragma unroll
  for (int k = 1; k < K; ++k) {
    const float q = c[k].h * xh[k];
    const float eq = fmaf(c[k].h, xh[k], -q);
    float s, t;
    two_sum(p, q, s, t);
    p = s;
    e += eq + t;
    e = fmaf(c[k].h52, xl[k], e);
    e = fmaf(c[k].l, xh[k], e);
  }
}

// Round the unevaluated sum p + e to the nearest-ish double using integer
// operations: h = fl(p + e) converts exactly by re-biasing its exponent, and
// the rest l = (p + e) - h is added as an integer number of ulps of the
// double binade that the result lands in (RZ(h + l) finds that binade even
// when h is a power of two and l is negative).
__device__ __forceinline__ double join(float p, float e) {
  const float h = p + e;
  const float l = e - (h - p);
  const unsigned hb = __float_as_uint(h);
  const unsigned rb = __float_as_uint(__fadd_rz(h, l));
  unsigned dhi = (((hb & 0x7fffffffu) >> 3) + (896u << 20)) | (hb & 0x80000000u);
  dhi = (hb << 1) ? dhi : (hb & 0x80000000u);
  const unsigned dlo = hb << 29;
  const unsigned er = max(rb & 0x7f800000u, 52u << 23);
  const unsigned sb = ((306u << 23) - er) | (hb & 0x80000000u);
  const int k = __float2int_rn(l * __uint_as_float(sb));
  unsigned long long bits = ((unsigned long long)dhi << 32) | dlo;
  bits += (unsigned long long)(long long)k;
  return __longlong_as_double((long long)bits);
}

// Error-free square: x*x = p + e exactly (x a float).
__device__ __forceinline__ void sqr(float x, float& p, float& e) {
  p = x * x;
  e = fmaf(x, x, -p);
}

// A double-float accumulator (h + l); add() takes an unevaluated pair.  After
// the error-free TwoSum of the leading parts the pair is renormalised
// (Fast2Sum: |l| stays below half an ulp of h), so each add loses at most
// about 2^-48 of the running sum however many terms one thread accumulates;
// without it the low word grows with the term count and its own rounding
// then drops the small residuals.
struct Acc {
  float h = 0.f, l = 0.f;
  __device__ __forceinline__ void add(float p, float e) {
    float s, t;
    two_sum(h, p, s, t);
    const float lo = l + (t + e);
    h = s + lo;
    l = lo - (h - s);
  }
  // Final value; uses two FP32->FP64 conversions and one FP64 add (once per thread).
  __device__ __forceinline__ double value() const { return (double)h + (double)l; }
};

// |a|^2 of a complex128 amplitude as an unevaluated pair, via split().
__device__ __forceinline__ void abs2_c128(double re, double im, float& p, float& e, unsigned& bad) {
  float rh, rl, ih, il;
  split(re, rh, rl, bad);
  split(im, ih, il, bad);
  float p1, e1, p2, e2;
  sqr(rh, p1, e1);
  sqr(ih, p2, e2);
  // cross terms 2*h*l (l = l52 * 2^-52)
  e1 = fmaf(rh * 0x1p-51f, rl, e1);
  e2 = fmaf(ih * 0x1p-51f, il, e2);
  float t;
  two_sum(p1, p2, p, t);
  e = e1 + e2 + t;
}

// |a|^2 of a complex64 amplitude as an unevaluated pair (exact).
__device__ __forceinline__ void abs2_c64(float re, float im, float& p, float& e) {
  float p1, e1, p2, e2;
  sqr(re, p1, e1);
  sqr(im, p2, e2);
  float t;
  two_sum(p1, p2, p, t);
  e = e1 + e2 + t;
}

}  // namespace dfx
}  // namespace iqs
