// Dense k-qubit gates (Section 2, "Scope and basic use": custom multi-qubit
// gates): a 2^k x 2^k matrix U acts on the amplitudes that differ only in the
// k target bits; bit j of U's row/column index is the value of qubits[j].
//
// One thread owns one group of 2^k amplitudes (the other n - k bits fixed):
// it loads the group into registers, forms every output as a dot product with
// a row of U and stores it.  The loops are unrolled completely, so every
// coefficient is a compile-time offset into the kernel's parameter block and
// enters the FMAs as a constant-bank operand (no shared-memory traffic).
// complex64 computes in FP32 (k <= 5); complex128 in the double-float
// emulation (k <= 4) or, for small states or on request, in native FP64.
// One read and one write of the state per gate.
#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "df64.cuh"
#include "internal.h"

namespace iqs {
namespace {

constexpr int kMaxK64 = 5, kMaxK128 = 4;

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

template <int K>
cudaError_t launch_k(iqs_reg* r, const int* qubits, const double* U) {
  constexpr int D = 1 << K;
  const uint64_t n_groups = num_amps(r) >> K;
  const unsigned grid = grid_for(n_groups, 1, 8);
  const Targets<K> T = make_targets<K>(qubits);
  if (r->dtype == IQS_C64) {
    if constexpr (K <= kMaxK64) {
      UF32<K> u;
      for (int i = 0; i < D * D; ++i) u.u[i] = make_float2((float)U[2 * i], (float)U[2 * i + 1]);
      k_kgate_c64<K><<<grid, kThreads, 0, r->stream>>>((float2*)r->data, n_groups, T, u);
      return launched(1);
    }
  } else if (!use_emulated(r)) {
    if constexpr (K <= kMaxK128) {
      UF64<K> u;
      for (int i = 0; i < D * D; ++i) u.u[i] = make_double2(U[2 * i], U[2 * i + 1]);
      k_kgate_c128_native<K><<<grid, kThreads, 0, r->stream>>>((double2*)r->data, n_groups, T, u);
      return launched(1);
    }
  } else {
    if constexpr (K <= kMaxK128) {
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
      k_kgate_c128_df<K><<<grid, kThreads, 0, r->stream>>>((double2*)r->data, n_groups, T, u, r->flag);
      return launched(1);
    }
  }
  return cudaErrorInvalidValue;  // unreachable: k is checked against the dtype's limit by the caller
}

}  // namespace

int max_kq(int dtype) { return dtype == IQS_C64 ? kMaxK64 : kMaxK128; }

cudaError_t launch_kq(iqs_reg* r, int k, const int* qubits, const double* U) {
  switch (k) {
    case 1: return launch_k<1>(r, qubits, U);
    case 2: return launch_k<2>(r, qubits, U);
    case 3: return launch_k<3>(r, qubits, U);
    case 4: return launch_k<4>(r, qubits, U);
    case 5: return launch_k<5>(r, qubits, U);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace iqs
