// Packed pairs of FP32 values for the sm_100-family paired FP32 instructions
// (PTX add/sub/mul/fma .f32x2).  Each lane is an ordinary IEEE FP32 operation
// with round-to-nearest, so a packed computation gives bit for bit the results
// of the same scalar operations done lane by lane, in half the instructions.
#pragma once

#include <cuda_runtime.h>

namespace iqs {
namespace f2 {

using P = unsigned long long;  // (lo, hi) = (lane 0, lane 1)

__device__ __forceinline__ P pack(float lo, float hi) {
  P r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void unpack(P v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ P pack(float2 v) { return pack(v.x, v.y); }

__device__ __forceinline__ P add(P a, P b) {
  P d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ P sub(P a, P b) {
  P d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ P mul(P a, P b) {
  P d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
// a * b + c, one rounding per lane
__device__ __forceinline__ P fma(P a, P b, P c) {
  P d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

}  // namespace f2
}  // namespace iqs
