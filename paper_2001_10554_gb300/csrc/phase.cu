// State initialisation, scaling, and the QAOA cost-phase layer
// psi_x <- exp(-i gamma C(x)) psi_x (Section 2 footnote: one global diagonal
// operation per QAOA step; Section 4: C counts the cut edges).
//
// Unweighted graphs use an FP64-built table T[k] = exp(-i gamma k), k = 0..|E|,
// held in shared memory; each amplitude computes its cut count with integer
// ops and multiplies by T[C(x)].  Weighted graphs multiply the per-edge unit
// factors exp(-i gamma w_e) of the cut edges.  Edge lists longer than one
// parameter block (255 edges) are applied in chunks, since the phase of a
// sum of cut counts is the product of the phases.
#include <cmath>
#include <vector>

#include "common.cuh"
#include "cut.cuh"
#include "df64.cuh"
#include "internal.h"

namespace iqs {
namespace {

template <class V>
__global__ void k_fill(V* __restrict__ a, uint64_t n, V val) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) a[i] = val;
}

template <class V>
__global__ void k_set_one(V* a, uint64_t index, V val) { a[index] = val; }

__global__ void k_scale_c64(float2* __restrict__ a, uint64_t n, float s) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    float2 v = a[i];
    v.x *= s;
    v.y *= s;
    a[i] = v;
  }
}

// Scaling is 2 multiplies per amplitude: native FP64 keeps pace with HBM here.
__global__ void k_scale_c128(double2* __restrict__ a, uint64_t n, double s) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    double2 v = a[i];
    v.x *= s;
    v.y *= s;
    a[i] = v;
  }
}

// ---------------------------------------------------------------- unweighted, table
struct TableF32 {
  float2 t[kEdgeChunk + 1];
};
struct TableF64 {
  double2 t[kEdgeChunk + 1];
};
// Emulated complex128: per entry the coefficient rows of (T * x).re = Tr xr - Ti xi
// and (T * x).im = Ti xr + Tr xi.
struct TableDF {
  dfx::Coef re[2 * (kEdgeChunk + 1)];
  dfx::Coef im[2 * (kEdgeChunk + 1)];
};

template <class X>
__global__ void __launch_bounds__(kThreads) k_zz_c64(float2* __restrict__ a, uint64_t n_amps, EdgesU8 E, TableF32 T) {
  __shared__ float2 s_t[kEdgeChunk + 1];
  for (int i = threadIdx.x; i <= E.m; i += blockDim.x) s_t[i] = T.t[i];
  __syncthreads();
  // two amplitudes per thread (one float4)
  const uint64_t n2 = n_amps >> 1;
  for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < n2; j += (uint64_t)gridDim.x * blockDim.x) {
    const X x0 = (X)(2 * j);
    float4* p = reinterpret_cast<float4*>(a) + j;
    float4 v = *p;
    const float2 t0 = s_t[cut_count(x0, E)];
    const float2 t1 = s_t[cut_count((X)(x0 | 1), E)];
    float4 w;
    w.x = t0.x * v.x - t0.y * v.y;
    w.y = t0.x * v.y + t0.y * v.x;
    w.z = t1.x * v.z - t1.y * v.w;
    w.w = t1.x * v.w + t1.y * v.z;
    *p = w;
  }
}

template <class X>
__global__ void __launch_bounds__(kThreads) k_zz_c128_df(double2* __restrict__ a, uint64_t n_amps, EdgesU8 E,
                                                          TableDF T, unsigned* __restrict__ flag) {
  __shared__ dfx::Coef s_re[2 * (kEdgeChunk + 1)];
  __shared__ dfx::Coef s_im[2 * (kEdgeChunk + 1)];
  for (int i = threadIdx.x; i < 2 * (E.m + 1); i += blockDim.x) {
    s_re[i] = T.re[i];
    s_im[i] = T.im[i];
  }
  __syncthreads();
  unsigned bad = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n_amps; i += (uint64_t)gridDim.x * blockDim.x) {
    const int c = cut_count((X)i, E);
    const double2 v = a[i];
    float xh[2], xl[2];
    dfx::split(v.x, xh[0], xl[0], bad);
    dfx::split(v.y, xh[1], xl[1], bad);
    float p, e;
    dfx::dot<2>(&s_re[2 * c], xh, xl, p, e);
    const double yr = dfx::join(p, e);
    dfx::dot<2>(&s_im[2 * c], xh, xl, p, e);
    const double yi = dfx::join(p, e);
    a[i] = make_double2(yr, yi);
  }
  if (bad) atomicOr(flag, 1u);
}

template <class X>
__global__ void __launch_bounds__(kThreads) k_zz_c128_native(double2* __restrict__ a, uint64_t n_amps, EdgesU8 E,
                                                              TableF64 T) {
  __shared__ double2 s_t[kEdgeChunk + 1];
  for (int i = threadIdx.x; i <= E.m; i += blockDim.x) s_t[i] = T.t[i];
  __syncthreads();
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n_amps; i += (uint64_t)gridDim.x * blockDim.x) {
    const double2 t = s_t[cut_count((X)i, E)];
    const double2 v = a[i];
    a[i] = make_double2(t.x * v.x - t.y * v.y, t.x * v.y + t.y * v.x);
  }
}

// ---------------------------------------------------------------- weighted: product of per-edge factors
struct FactorsF32 {
  float2 f[kEdgeChunk + 1];
};
struct FactorsF64 {
  double2 f[kEdgeChunk + 1];
};

template <class X>
__global__ void __launch_bounds__(kThreads) k_zzw_c64(float2* __restrict__ a, uint64_t n_amps, EdgesU8 E, FactorsF32 F) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n_amps; i += (uint64_t)gridDim.x * blockDim.x) {
    const X x = (X)i;
    float2 ph = make_float2(1.f, 0.f);
    for (int e = 0; e < E.m; ++e) {
      if (((x >> E.u[e]) ^ (x >> E.v[e])) & 1) {
        const float2 f = F.f[e];
        ph = make_float2(ph.x * f.x - ph.y * f.y, ph.x * f.y + ph.y * f.x);
      }
    }
    const float2 v = a[i];
    a[i] = make_float2(ph.x * v.x - ph.y * v.y, ph.x * v.y + ph.y * v.x);
  }
}

// Weighted complex128 uses native FP64 (a secondary path; the table path is the fast one).
template <class X>
__global__ void __launch_bounds__(kThreads) k_zzw_c128(double2* __restrict__ a, uint64_t n_amps, EdgesU8 E, FactorsF64 F) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n_amps; i += (uint64_t)gridDim.x * blockDim.x) {
    const X x = (X)i;
    double2 ph = make_double2(1.0, 0.0);
    for (int e = 0; e < E.m; ++e) {
      if (((x >> E.u[e]) ^ (x >> E.v[e])) & 1) {
        const double2 f = F.f[e];
        ph = make_double2(ph.x * f.x - ph.y * f.y, ph.x * f.y + ph.y * f.x);
      }
    }
    const double2 v = a[i];
    a[i] = make_double2(ph.x * v.x - ph.y * v.y, ph.x * v.y + ph.y * v.x);
  }
}

template <class X>
cudaError_t zz_chunk(iqs_reg* r, const EdgesU8& E, const double* w, double gamma) {
  const uint64_t N = num_amps(r);
  const unsigned grid = grid_for(N, 2, 32);
  if (w == nullptr) {
    if (r->dtype == IQS_C64) {
      TableF32 T;
      for (int k = 0; k <= E.m; ++k) T.t[k] = make_float2((float)std::cos(gamma * k), (float)-std::sin(gamma * k));
      if (N >= 2)
        k_zz_c64<X><<<grid, kThreads, 0, r->stream>>>((float2*)r->data, N, E, T);
      else
        return cudaErrorInvalidValue;
    } else if (use_emulated(r)) {
      TableDF T;
      for (int k = 0; k <= E.m; ++k) {
        const double tr = std::cos(gamma * k), ti = -std::sin(gamma * k);
        T.re[2 * k] = dfx::make_coef(tr);
        T.re[2 * k + 1] = dfx::make_coef(-ti);
        T.im[2 * k] = dfx::make_coef(ti);
        T.im[2 * k + 1] = dfx::make_coef(tr);
      }
      k_zz_c128_df<X><<<grid_for(N, 1, 32), kThreads, 0, r->stream>>>((double2*)r->data, N, E, T, r->flag);
    } else {
      TableF64 T;
      for (int k = 0; k <= E.m; ++k) T.t[k] = make_double2(std::cos(gamma * k), -std::sin(gamma * k));
      k_zz_c128_native<X><<<grid_for(N, 1, 32), kThreads, 0, r->stream>>>((double2*)r->data, N, E, T);
    }
  } else {
    if (r->dtype == IQS_C64) {
      FactorsF32 F;
      for (int e = 0; e < E.m; ++e)
        F.f[e] = make_float2((float)std::cos(gamma * w[e]), (float)-std::sin(gamma * w[e]));
      k_zzw_c64<X><<<grid_for(N, 1, 32), kThreads, 0, r->stream>>>((float2*)r->data, N, E, F);
    } else {
      FactorsF64 F;
      for (int e = 0; e < E.m; ++e) F.f[e] = make_double2(std::cos(gamma * w[e]), -std::sin(gamma * w[e]));
      k_zzw_c128<X><<<grid_for(N, 1, 32), kThreads, 0, r->stream>>>((double2*)r->data, N, E, F);
    }
  }
  return launched(1);
}

}  // namespace

cudaError_t launch_init_basis(iqs_reg* r, uint64_t index) {
  cudaError_t e = cudaMemsetAsync(r->data, 0, num_amps(r) * amp_bytes(r), r->stream);
  if (e != cudaSuccess) return e;
  if (r->dtype == IQS_C64)
    k_set_one<float2><<<1, 1, 0, r->stream>>>((float2*)r->data, index, make_float2(1.f, 0.f));
  else
    k_set_one<double2><<<1, 1, 0, r->stream>>>((double2*)r->data, index, make_double2(1.0, 0.0));
  return launched(1);
}

cudaError_t launch_init_uniform(iqs_reg* r) {
  const uint64_t N = num_amps(r);
  const double v = std::pow(2.0, -r->n / 2.0);
  if (r->dtype == IQS_C64)
    k_fill<float2><<<grid_for(N, 1, 16), kThreads, 0, r->stream>>>((float2*)r->data, N, make_float2((float)v, 0.f));
  else
    k_fill<double2><<<grid_for(N, 1, 16), kThreads, 0, r->stream>>>((double2*)r->data, N, make_double2(v, 0.0));
  return launched(1);
}

cudaError_t launch_scale(iqs_reg* r, double s) {
  const uint64_t N = num_amps(r);
  if (r->dtype == IQS_C64)
    k_scale_c64<<<grid_for(N, 1, 16), kThreads, 0, r->stream>>>((float2*)r->data, N, (float)s);
  else
    k_scale_c128<<<grid_for(N, 1, 16), kThreads, 0, r->stream>>>((double2*)r->data, N, s);
  return launched(1);
}

cudaError_t launch_zz_phase(iqs_reg* r, int n_edges, const int32_t* edges, const double* w, double gamma) {
  for (int base = 0; base < n_edges || (base == 0 && n_edges == 0); base += kEdgeChunk) {
    EdgesU8 E;
    E.m = n_edges - base < kEdgeChunk ? n_edges - base : kEdgeChunk;
    for (int e = 0; e < E.m; ++e) {
      E.u[e] = (uint8_t)edges[2 * (base + e)];
      E.v[e] = (uint8_t)edges[2 * (base + e) + 1];
    }
    if (E.m == 0) return cudaSuccess;  // no edges: identity
    const cudaError_t err = r->n <= 32 ? zz_chunk<uint32_t>(r, E, w ? w + base : nullptr, gamma)
                                       : zz_chunk<uint64_t>(r, E, w ? w + base : nullptr, gamma);
    if (err != cudaSuccess) return err;
  }
  return cudaSuccess;
}

}  // namespace iqs
