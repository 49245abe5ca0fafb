// Element operations of the QAOA engine for the two storage types.
//
// complex64 (float2): FP32 arithmetic; products for reductions are exact
// (FMA residuals) and accumulate in double-float.
// complex128 (double2): values are split once into double-float form
// (df64.cuh) when a tile is loaded, every gate of the tile works on the split
// form, and the join back to IEEE FP64 happens once on store.
#pragma once

#include "df64.cuh"

namespace iqs {
namespace qops {

// ---------------------------------------------------------------- split complex128
// value = h + l * 2^-52 per component
struct S2 {
  float rh, rl, ih, il;
};

__device__ __forceinline__ S2 to_split(double2 v, unsigned& bad) {
  S2 s;
  dfx::split(v.x, s.rh, s.rl, bad);
  dfx::split(v.y, s.ih, s.il, bad);
  return s;
}

__device__ __forceinline__ double2 from_split(const S2& s) {
  return make_double2(dfx::join(s.rh, s.rl * 0x1p-52f), dfx::join(s.ih, s.il * 0x1p-52f));
}

// Unevaluated (p + e) -> split form (h, l * 2^52).
__device__ __forceinline__ void renorm(float p, float e, float& h, float& l52) {
  h = p + e;
  l52 = (e - (h - p)) * 0x1p52f;
}

// Coefficient pairs for 2-term dot products.
struct C2 {
  dfx::Coef a, b;
};

__device__ __forceinline__ void dot2s(const dfx::Coef& ca, float xh, float xl, const dfx::Coef& cb, float yh, float yl,
                                      float& h, float& l52) {
  const dfx::Coef c[2] = {ca, cb};
  const float xs[2] = {xh, yh};
  const float ls[2] = {xl, yl};
  float p, e;
  dfx::dot<2>(c, xs, ls, p, e);
  renorm(p, e, h, l52);
}

// RX(2 beta) (or its inverse with sb -> -sb) on a pair, complex64.
//   y0 = c x0 - i s x1,  y1 = -i s x0 + c x1
__device__ __forceinline__ void rx_pair(float2& x0, float2& x1, float c, float s) {
  const float2 y0 = make_float2(c * x0.x + s * x1.y, c * x0.y - s * x1.x);
  const float2 y1 = make_float2(s * x0.y + c * x1.x, -s * x0.x + c * x1.y);
  x0 = y0;
  x1 = y1;
}

// RX coefficients for the split form: c, s, -s.
struct RXc {
  dfx::Coef c, s, ns;
};

__device__ __forceinline__ void rx_pair(S2& x0, S2& x1, const RXc& k) {
  S2 y0, y1;
  dot2s(k.c, x0.rh, x0.rl, k.s, x1.ih, x1.il, y0.rh, y0.rl);   // c x0r + s x1i
  dot2s(k.c, x0.ih, x0.il, k.ns, x1.rh, x1.rl, y0.ih, y0.il);  // c x0i - s x1r
  dot2s(k.s, x0.ih, x0.il, k.c, x1.rh, x1.rl, y1.rh, y1.rl);   // s x0i + c x1r
  dot2s(k.ns, x0.rh, x0.rl, k.c, x1.ih, x1.il, y1.ih, y1.il);  // -s x0r + c x1i
  x0 = y0;
  x1 = y1;
}

// Phase factor t = (tr, ti) times x.
__device__ __forceinline__ float2 cmul(float2 t, float2 x) {
  return make_float2(t.x * x.x - t.y * x.y, t.x * x.y + t.y * x.x);
}

// Split-form phase factor: rows (tr, -ti) and (ti, tr).
struct Ph {
  dfx::Coef tr, ti, nti;
};

__device__ __forceinline__ S2 cmul(const Ph& t, const S2& x) {
  S2 y;
  dot2s(t.tr, x.rh, x.rl, t.nti, x.ih, x.il, y.rh, y.rl);
  dot2s(t.ti, x.rh, x.rl, t.tr, x.ih, x.il, y.ih, y.il);
  return y;
}

// ---------------------------------------------------------------- exact products for reductions
// a*b + c*d as an unevaluated pair (floats).
__device__ __forceinline__ void dot2_exact(float a, float b, float c, float d, float& p, float& e) {
  const float p1 = a * b, e1 = fmaf(a, b, -p1);
  const float p2 = c * d, e2 = fmaf(c, d, -p2);
  float t;
  dfx::two_sum(p1, p2, p, t);
  e = e1 + e2 + t;
}

// (xh + xl 2^-52)(yh + yl 2^-52) as an unevaluated pair.
__device__ __forceinline__ void mul_split(float xh, float xl, float yh, float yl, float& p, float& e) {
  p = xh * yh;
  e = fmaf(xh, yh, -p);
  e = fmaf(xh * 0x1p-52f, yl, e);
  e = fmaf(yh * 0x1p-52f, xl, e);
}

// Im(conj(l) * f) = lr fi - li fr
__device__ __forceinline__ void im_conj_mul(float2 l, float2 f, float& p, float& e) {
  dot2_exact(l.x, f.y, -l.y, f.x, p, e);
}
__device__ __forceinline__ void im_conj_mul(const S2& l, const S2& f, float& p, float& e) {
  float p1, e1, p2, e2, t;
  mul_split(l.rh, l.rl, f.ih, f.il, p1, e1);
  mul_split(l.ih, l.il, f.rh, f.rl, p2, e2);
  dfx::two_sum(p1, -p2, p, t);
  e = e1 - e2 + t;
}

// acc + Im(conj(l) * f) in plain FP32 (two FMAs; complex64 block sums)
__device__ __forceinline__ float im_conj_mul_fma(float2 l, float2 f, float acc) {
  return fmaf(-l.y, f.x, fmaf(l.x, f.y, acc));
}
__device__ __forceinline__ float im_conj_mul_fma(const S2&, const S2&, float acc) { return acc; }  // unused for complex128

// |x|^2
__device__ __forceinline__ void abs2(float2 x, float& p, float& e) { dfx::abs2_c64(x.x, x.y, p, e); }
__device__ __forceinline__ void abs2(const S2& x, float& p, float& e) {
  float p1, e1, p2, e2, t;
  mul_split(x.rh, x.rl, x.rh, x.rl, p1, e1);
  mul_split(x.ih, x.il, x.ih, x.il, p2, e2);
  dfx::two_sum(p1, p2, p, t);
  e = e1 + e2 + t;
}

// k * x for a small integer k (exact in float), complex64 and split form.
__device__ __forceinline__ float2 scale_int(float2 x, float k) { return make_float2(k * x.x, k * x.y); }
__device__ __forceinline__ S2 scale_int(const S2& x, float k) {
  S2 y;
  float p, e;
  p = k * x.rh; e = fmaf(k, x.rh, -p); e = fmaf(k * 0x1p-52f, x.rl, e); renorm(p, e, y.rh, y.rl);
  p = k * x.ih; e = fmaf(k, x.ih, -p); e = fmaf(k * 0x1p-52f, x.il, e); renorm(p, e, y.ih, y.il);
  return y;
}

}  // namespace qops
}  // namespace iqs
