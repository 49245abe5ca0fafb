// Pool engine: many states ("trajectories") of one layered circuit, with
// stochastic noise rotations that differ per trajectory (Section 2, "Pool of
// multiple states": noise gates are one-qubit rotations whose angles vary over
// the pool's states; pool appendix: the probability of a qubit averaged
// incoherently over the pool = sum over pool states / pool size).
//
// Circuit family (brick layers): layer l applies a one-qubit unitary U[l][q]
// to every qubit q, then CNOT(i, i+1) for i = o, o+2, ... with o = l mod 2.
// With noise, every gate is followed, on each qubit it touched, by RX(tx)
// then RZ(tz) with per-trajectory angles.
//
// GB300 mapping.  All trajectories of a call advance together: the
// trajectory is blockIdx.y.  One layer is one or two tiled passes over each
// state: the one-qubit phase of layer l uses, per trajectory and qubit, the
// fused matrix G = N(after the gate) . U[l][q] . N(after the CNOT of layer l-1),
// composed in FP64 at the start of each block; the CNOT brick is a fixed
// permutation of tile indices, l -> l ^ ((l & controls) << 1), applied when
// the tile is written back.  The low pass holds qubits 0..K-1; each further
// pass holds its qubits plus the qubit just below them, so the brick's
// boundary CNOT runs after both its qubits' one-qubit gates.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"
#include "df64.cuh"
#include "internal.h"
#include "qaoa_ops.cuh"
#include "tile.cuh"

namespace iqs {
namespace {

using qops::S2;

constexpr int kPoolMaxQubits = 24;

// ---------------------------------------------------------------- FP64 2x2 algebra (per block, a few matrices)
struct M2 {
  double r[4], i[4];  // row-major U00 U01 U10 U11
};

__device__ M2 mmul(const M2& a, const M2& b) {
  M2 c;
#pragma unroll
  for (int row = 0; row < 2; ++row)
#pragma unroll
    for (int col = 0; col < 2; ++col) {
      double re = 0.0, im = 0.0;
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const double ar = a.r[2 * row + k], ai = a.i[2 * row + k];
        const double br = b.r[2 * k + col], bi = b.i[2 * k + col];
        re += ar * br - ai * bi;
        im += ar * bi + ai * br;
      }
      c.r[2 * row + col] = re;
      c.i[2 * row + col] = im;
    }
  return c;
}

__device__ M2 identity2() {
  M2 m;
  m.r[0] = 1.0; m.i[0] = 0.0; m.r[1] = 0.0; m.i[1] = 0.0;
  m.r[2] = 0.0; m.i[2] = 0.0; m.r[3] = 1.0; m.i[3] = 0.0;
  return m;
}

// RZ(tz) . RX(tx), R(t) = exp(-i t sigma / 2)
__device__ M2 noise_rot(double tx, double tz) {
  double sx, cx, sz, cz;
  sincos(0.5 * tx, &sx, &cx);
  sincos(0.5 * tz, &sz, &cz);
  // RX = [[cx, -i sx], [-i sx, cx]];  RZ = diag(cz - i sz, cz + i sz)
  M2 m;
  m.r[0] = cz * cx;  m.i[0] = -sz * cx;   // (cz - i sz) cx
  m.r[1] = -sz * sx; m.i[1] = -cz * sx;   // (cz - i sz)(-i sx)
  m.r[2] = sz * sx;  m.i[2] = -cz * sx;   // (cz + i sz)(-i sx)
  m.r[3] = cz * cx;  m.i[3] = sz * cx;    // (cz + i sz) cx
  return m;
}

struct Circuit {
  int n, depth;
  const double* U;          // [depth][n][8]
  const double* angles;     // [batch][n_noise][2] or nullptr
  const int* layer_base;    // [depth]: index of the first noise op of layer l
  int n_noise;
};

// Fused one-qubit matrix of phase l (0..depth) for qubit q of trajectory b.
__device__ M2 compose(const Circuit& C, int b, int l, int q) {
  M2 G = identity2();
  const double* ang = C.angles ? C.angles + (uint64_t)b * C.n_noise * 2 : nullptr;
  if (ang && l > 0) {
    const int o = (l - 1) & 1;
    const int d = q - o;
    if (d >= 0) {
      const int j = d >> 1;
      const int ctrl = o + 2 * j;
      if (ctrl + 1 < C.n) {
        const int k = C.layer_base[l - 1] + C.n + 2 * j + (q == ctrl ? 0 : 1);
        G = noise_rot(ang[2 * k], ang[2 * k + 1]);
      }
    }
  }
  if (l < C.depth) {
    M2 U;
    const double* u = C.U + ((uint64_t)l * C.n + q) * 8;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      U.r[e] = u[2 * e];
      U.i[e] = u[2 * e + 1];
    }
    G = mmul(U, G);
    if (ang) {
      const int k = C.layer_base[l] + q;
      G = mmul(noise_rot(ang[2 * k], ang[2 * k + 1]), G);
    }
  }
  return G;
}

// ---------------------------------------------------------------- storage traits
struct P64 {
  using V = float2;
  using W = float2;
  struct Mat {
    float r[4], i[4];
  };
  static constexpr int kTileBits = 12, kRowBits = 4, kRegBits = 4, kSwzBits = 4;
  __device__ static W load(V v, unsigned&) { return v; }
  __device__ static V store(const W& w) { return w; }
  __device__ static Mat make(const M2& g) {
    Mat m;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      m.r[e] = (float)g.r[e];
      m.i[e] = (float)g.i[e];
    }
    return m;
  }
  __device__ static void apply(const Mat& u, W& x0, W& x1) {
    const float2 y0 = make_float2(u.r[0] * x0.x - u.i[0] * x0.y + u.r[1] * x1.x - u.i[1] * x1.y,
                                  u.r[0] * x0.y + u.i[0] * x0.x + u.r[1] * x1.y + u.i[1] * x1.x);
    const float2 y1 = make_float2(u.r[2] * x0.x - u.i[2] * x0.y + u.r[3] * x1.x - u.i[3] * x1.y,
                                  u.r[2] * x0.y + u.i[2] * x0.x + u.r[3] * x1.y + u.i[3] * x1.x);
    x0 = y0;
    x1 = y1;
  }
  __device__ static void abs2(const W& x, float& p, float& e) { qops::abs2(x, p, e); }
};

struct P128 {
  using V = double2;
  using W = S2;
  struct Mat {
    dfx::Coef c[16];  // rows out0.re, out0.im, out1.re, out1.im over (x0.re, x0.im, x1.re, x1.im)
  };
  static constexpr int kTileBits = 11, kRowBits = 3, kRegBits = 3, kSwzBits = 3;
  __device__ static W load(V v, unsigned& bad) { return qops::to_split(v, bad); }
  __device__ static V store(const W& w) { return qops::from_split(w); }
  __device__ static dfx::Coef coef(double v) {
    dfx::Coef c;
    // split on the device with the same recipe as the host (FP64 ops, once per block)
    c.h = (float)v;
    c.l = (float)(v - (double)c.h);
    c.h52 = (float)((double)c.h * 0x1p-52);
    return c;
  }
  __device__ static Mat make(const M2& u) {
    Mat m;
#pragma unroll
    for (int row = 0; row < 2; ++row) {
      const int a = 2 * row, b = 2 * row + 1;
      const double re[4] = {u.r[a], -u.i[a], u.r[b], -u.i[b]};
      const double im[4] = {u.i[a], u.r[a], u.i[b], u.r[b]};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        m.c[8 * row + k] = coef(re[k]);
        m.c[8 * row + 4 + k] = coef(im[k]);
      }
    }
    return m;
  }
  __device__ static void apply(const Mat& u, W& x0, W& x1) {
    const float xh[4] = {x0.rh, x0.ih, x1.rh, x1.ih};
    const float xl[4] = {x0.rl, x0.il, x1.rl, x1.il};
    float p, e;
    S2 y0, y1;
    dfx::dot<4>(&u.c[0], xh, xl, p, e);
    qops::renorm(p, e, y0.rh, y0.rl);
    dfx::dot<4>(&u.c[4], xh, xl, p, e);
    qops::renorm(p, e, y0.ih, y0.il);
    dfx::dot<4>(&u.c[8], xh, xl, p, e);
    qops::renorm(p, e, y1.rh, y1.rl);
    dfx::dot<4>(&u.c[12], xh, xl, p, e);
    qops::renorm(p, e, y1.ih, y1.il);
    x0 = y0;
    x1 = y1;
  }
  __device__ static void abs2(const W& x, float& p, float& e) { qops::abs2(x, p, e); }
};

// ---------------------------------------------------------------- one pass
// Tile: row bits [0, g.c), gate bits [g.s, g.s + g.m).  One-qubit gates on the
// qubits [q_lo, q_hi) (all inside the gate bits), then the CNOTs whose
// controls are the local bits in ``cmask``.
template <class TR>
__global__ void __launch_bounds__(kThreads) k_pool_pass(typename TR::V* __restrict__ psi, uint64_t N, Geo g, int q_lo,
                                                        int q_hi, unsigned cmask, Circuit circ, int layer,
                                                        unsigned* flag) {
  using W = typename TR::W;
  using Mat = typename TR::Mat;
  constexpr int R = TR::kRegBits;
  constexpr int RB = 1 << R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Mat mats[16];
  W* sp = reinterpret_cast<W*>(smem_raw);
  const unsigned K = g.c + g.m;
  const unsigned T = 1u << K;
  const unsigned b = blockIdx.y;
  const int ng = q_hi - q_lo;
  if ((int)threadIdx.x < ng) mats[threadIdx.x] = TR::make(compose(circ, b, layer, q_lo + threadIdx.x));
  __syncthreads();
  // local bit of qubit q: q - s + c for a high pass, q for the low pass
  const int lb0 = (g.c == 0 && g.s == 0) ? q_lo : (q_lo - g.s + g.c);
  typename TR::V* P = psi + (uint64_t)b * N;
  const uint64_t tiles = N >> K;
  unsigned bad = 0;
  for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    for (unsigned l = threadIdx.x; l < T; l += blockDim.x) sp[swz<TR>(l)] = TR::load(P[tile_x(g, t, l)], bad);
    __syncthreads();
    for (int pos = lb0; pos < lb0 + ng; pos += R) {
      const int gb = min(R, lb0 + ng - pos);
      const unsigned nsub = T >> gb;
      for (unsigned sb = threadIdx.x; sb < nsub; sb += blockDim.x) {
        const unsigned base = ((sb >> pos) << (pos + gb)) | (sb & ((1u << pos) - 1u));
        W a[RB];
#pragma unroll
        for (int j = 0; j < RB; ++j)
          if (j < (1 << gb)) a[j] = sp[swz<TR>(base | ((unsigned)j << pos))];
#pragma unroll
        for (int bit = 0; bit < R; ++bit) {
          if (bit < gb) {
            const Mat& u = mats[pos - lb0 + bit];
#pragma unroll
            for (int j = 0; j < RB; ++j)
              if (!(j & (1 << bit)) && j < (1 << gb)) TR::apply(u, a[j], a[j | (1 << bit)]);
          }
        }
#pragma unroll
        for (int j = 0; j < RB; ++j)
          if (j < (1 << gb)) sp[swz<TR>(base | ((unsigned)j << pos))] = a[j];
      }
      __syncthreads();
    }
    // CNOT brick: new[l] = old[l ^ ((l & cmask) << 1)]
    for (unsigned l = threadIdx.x; l < T; l += blockDim.x)
      P[tile_x(g, t, l)] = TR::store(sp[swz<TR>(l ^ ((l & cmask) << 1))]);
    __syncthreads();
  }
  if (bad) atomicOr(flag, 1u);
}

template <class V>
__global__ void k_basis0_batch(V* psi, uint64_t N, int batch) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N * batch; i += (uint64_t)gridDim.x * blockDim.x) {
    V v;
    v.x = (i % N) == 0 ? 1 : 0;
    v.y = 0;
    psi[i] = v;
  }
}

// Per-trajectory P(q = 1) for q < n (n <= 24) and the squared norm; each
// thread keeps one double-float accumulator per qubit.
template <class TR>
__global__ void __launch_bounds__(kThreads) k_pool_probs(const typename TR::V* __restrict__ psi, uint64_t N, int n,
                                                         double* __restrict__ partials, int part_stride, unsigned* flag) {
  const unsigned b = blockIdx.y;
  const typename TR::V* P = psi + (uint64_t)b * N;
  dfx::Acc acc[kPoolMaxQubits + 1];
  unsigned bad = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x) {
    float p, e;
    TR::abs2(TR::load(P[i], bad), p, e);
    acc[kPoolMaxQubits].add(p, e);
#pragma unroll
    for (int q = 0; q < kPoolMaxQubits; ++q)
      if (q < n && ((i >> q) & 1)) acc[q].add(p, e);
  }
  if (bad) atomicOr(flag, 1u);
  for (int q = 0; q <= kPoolMaxQubits; ++q) {
    if (q < n || q == kPoolMaxQubits)
      block_partial(acc[q].value(), partials + (uint64_t)b * part_stride + (uint64_t)q * gridDim.x + blockIdx.x);
  }
}

// probs[b][q] = P_q / norm (one block per trajectory), and the pool average.
__global__ void k_pool_finish(const double* __restrict__ partials, int part_stride, int nblk, int n,
                              double* __restrict__ probs) {
  const unsigned b = blockIdx.x;
  __shared__ double vals[kPoolMaxQubits + 1];
  for (int q = threadIdx.x; q <= kPoolMaxQubits; q += blockDim.x) {
    if (q < n || q == kPoolMaxQubits) {
      double s = 0.0;
      for (int j = 0; j < nblk; ++j) s += partials[(uint64_t)b * part_stride + (uint64_t)q * nblk + j];
      vals[q] = s;
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < n; q += blockDim.x) probs[(uint64_t)b * n + q] = vals[q] / vals[kPoolMaxQubits];
}

__global__ void k_pool_mean(const double* __restrict__ probs, int batch, int n, double* __restrict__ mean) {
  const int q = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < batch; b += blockDim.x) s += probs[(uint64_t)b * n + q];
  __shared__ double red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    mean[q] = t / batch;  // incoherent sum over the pool divided by its size
  }
}

}  // namespace
}  // namespace iqs

struct iqs_pool {
  int n = 0, dtype = IQS_C64, bmax = 0, depth_max = 0;
  uint64_t N = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  void* psi = nullptr;
  double* U = nullptr;
  double* angles = nullptr;
  int* layer_base = nullptr;
  double* partials = nullptr;
  double* probs = nullptr;
  double* mean = nullptr;
  unsigned* flag = nullptr;
  size_t angle_cap = 0;  // doubles
  int part_stride = 0, nblk = 0;
};

namespace iqs {
namespace {

int n_noise_ops(int n, int depth) {
  int k = 0;
  for (int l = 0; l < depth; ++l) k += n + 2 * ((n - (l & 1)) / 2);
  return k;
}

struct Pass {
  Geo g;
  int q_lo, q_hi;
  int cut_lo;  // CNOT pairs (i, i+1) owned by this pass: cut_lo <= i, i + 1 < cut_hi
  int cut_hi;
};

std::vector<Pass> plan_pool(int n, int K, int rows) {
  std::vector<Pass> out;
  const int KA = std::min(n, K);
  out.push_back(Pass{Geo{0, 0, KA}, 0, KA, 0, KA});
  int start = KA;
  while (start < n) {
    const int maxm = K - rows;                 // gate bits per pass incl. the boundary qubit
    const int end = std::min(n, start - 1 + maxm);
    const int s = start - 1, m = end - s;
    out.push_back(Pass{Geo{K - m, s, m}, start, end, s, end});
    start = end;
  }
  return out;
}

unsigned cnot_mask(const Pass& p, int n, int layer) {
  const int o = layer & 1;
  unsigned mask = 0;
  for (int i = o; i + 1 < n; i += 2) {
    if (i >= p.cut_lo && i + 1 < p.cut_hi && i + 1 >= (p.g.c == 0 && p.g.s == 0 ? 0 : p.q_lo)) {
      const int lb = (p.g.c == 0 && p.g.s == 0) ? i : i - p.g.s + p.g.c;
      mask |= 1u << lb;
    }
  }
  return mask;
}

template <class TR>
cudaError_t run_pool(iqs_pool* P, int batch, int depth, bool noisy) {
  using V = typename TR::V;
  const uint64_t N = P->N;
  cudaStream_t s = P->stream;
  V* psi = (V*)P->psi;
  int launches = 0;
  k_basis0_batch<V><<<grid_for(N * batch, 1, 16), kThreads, 0, s>>>(psi, N, batch);
  ++launches;
  Circuit C{P->n, depth, P->U, noisy ? P->angles : nullptr, P->layer_base, n_noise_ops(P->n, depth)};
  const std::vector<Pass> passes = plan_pool(P->n, TR::kTileBits, TR::kRowBits);
  const int phases = noisy ? depth + 1 : depth;
  for (int l = 0; l < phases; ++l) {
    for (const Pass& p : passes) {
      const unsigned K = p.g.c + p.g.m;
      const uint64_t tiles = N >> K;
      const unsigned gx = (unsigned)std::min<uint64_t>(tiles, (uint64_t)std::max(1, 2432 / batch));
      const unsigned cm = l < depth ? cnot_mask(p, P->n, l) : 0u;
      const size_t smem = ((size_t)1 << K) * sizeof(typename TR::W);
      k_pool_pass<TR><<<dim3(std::max(1u, gx), batch), kThreads, smem, s>>>(psi, N, p.g, p.q_lo, p.q_hi, cm, C, l,
                                                                            P->flag);
      ++launches;
    }
  }
  const dim3 gp(P->nblk, batch);
  k_pool_probs<TR><<<gp, kThreads, 0, s>>>(psi, N, P->n, P->partials, P->part_stride, P->flag);
  k_pool_finish<<<batch, 32, 0, s>>>(P->partials, P->part_stride, P->nblk, P->n, P->probs);
  k_pool_mean<<<P->n, kThreads, 0, s>>>(P->probs, batch, P->n, P->mean);
  launches += 3;
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) note_launches(launches);
  return e;
}

template <class TR>
cudaError_t set_pool_attrs() {
  return cudaFuncSetAttribute(k_pool_pass<TR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (1 << TR::kTileBits) * (int)sizeof(typename TR::W));
}

void free_pool(iqs_pool* p) {
  cudaFree(p->psi);
  cudaFree(p->U);
  cudaFree(p->angles);
  cudaFree(p->layer_base);
  cudaFree(p->partials);
  cudaFree(p->probs);
  cudaFree(p->mean);
  cudaFree(p->flag);
  if (p->own_stream && p->stream) cudaStreamDestroy(p->stream);
  delete p;
}

}  // namespace
}  // namespace iqs

extern "C" {

iqs_status iqs_pool_create(int n, int dtype, int batch_max, int depth_max, void* stream, iqs_pool** out) {
  using namespace iqs;
  if (out == nullptr) return report(IQS_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 2 || n > kPoolMaxQubits) return report(IQS_EINVAL, "pool states need 2..%d qubits, got %d", kPoolMaxQubits, n);
  if (dtype != IQS_C64 && dtype != IQS_C128) return report(IQS_EINVAL, "dtype must be IQS_C64 or IQS_C128");
  if (batch_max < 1 || batch_max > 65535) return report(IQS_EINVAL, "batch_max %d outside [1, 65535]", batch_max);
  if (depth_max < 1 || depth_max > 100000) return report(IQS_EINVAL, "depth_max %d outside [1, 100000]", depth_max);
  if (fault_now(1)) return report(IQS_ENOMEM, "injected allocation failure");
  iqs_pool* p = new (std::nothrow) iqs_pool();
  if (p == nullptr) return report(IQS_ENOMEM, "host allocation failed");
  p->n = n;
  p->dtype = dtype;
  p->bmax = batch_max;
  p->depth_max = depth_max;
  p->N = 1ull << n;
  p->stream = (cudaStream_t)stream;
  if (p->stream == nullptr) {
    if (cudaStreamCreate(&p->stream) != cudaSuccess) {
      cudaGetLastError();
      delete p;
      return report(IQS_ECUDA, "cannot create a stream");
    }
    p->own_stream = true;
  }
  const size_t amp = dtype == IQS_C128 ? 16 : 8;
  p->nblk = (int)std::max<uint64_t>(1, std::min<uint64_t>(p->N / 4096, 64));
  p->part_stride = p->nblk * (kPoolMaxQubits + 1);
  p->angle_cap = (size_t)batch_max * n_noise_ops(n, depth_max) * 2;
  const bool ok = cudaMalloc(&p->psi, amp * p->N * batch_max) == cudaSuccess &&
                  cudaMalloc(&p->U, sizeof(double) * 8 * (size_t)n * depth_max) == cudaSuccess &&
                  cudaMalloc(&p->angles, sizeof(double) * p->angle_cap) == cudaSuccess &&
                  cudaMalloc(&p->layer_base, sizeof(int) * (size_t)depth_max) == cudaSuccess &&
                  cudaMalloc(&p->partials, sizeof(double) * (size_t)p->part_stride * batch_max) == cudaSuccess &&
                  cudaMalloc(&p->probs, sizeof(double) * (size_t)n * batch_max) == cudaSuccess &&
                  cudaMalloc(&p->mean, sizeof(double) * (size_t)n) == cudaSuccess &&
                  cudaMalloc(&p->flag, sizeof(unsigned)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_pool(p);
    return report(IQS_ENOMEM, "cannot allocate the pool (%d states of %d qubits, depth %d)", batch_max, n, depth_max);
  }
  cudaError_t e = cudaMemsetAsync(p->flag, 0, sizeof(unsigned), p->stream);
  if (e == cudaSuccess) e = dtype == IQS_C128 ? set_pool_attrs<P128>() : set_pool_attrs<P64>();
  if (e != cudaSuccess) {
    free_pool(p);
    return report(IQS_ECUDA, "pool set-up: %s", cudaGetErrorString(e));
  }
  *out = p;
  return IQS_OK;
}

iqs_status iqs_pool_destroy(iqs_pool* p) {
  if (p == nullptr) return IQS_OK;
  cudaStreamSynchronize(p->stream);
  iqs::free_pool(p);
  return IQS_OK;
}

int iqs_pool_noise_count(int n, int depth) { return iqs::n_noise_ops(n, depth); }

iqs_status iqs_pool_run_brick(iqs_pool* p, int batch, int depth, const double* unitaries, const double* angles,
                              double* probs, double* mean) {
  using namespace iqs;
  if (p == nullptr) return report(IQS_EINVAL, "handle is NULL");
  if (batch < 1 || batch > p->bmax) return report(IQS_EINVAL, "batch %d outside [1, %d]", batch, p->bmax);
  if (depth < 1 || depth > p->depth_max) return report(IQS_EINVAL, "depth %d outside [1, %d]", depth, p->depth_max);
  if (unitaries == nullptr || mean == nullptr) return report(IQS_EINVAL, "unitaries and mean must not be NULL");
  if (fault_now(2)) return report(IQS_ECUDA, "iqs_pool_run_brick: injected launch failure");
  const int nn = n_noise_ops(p->n, depth);
  std::vector<int> base(depth);
  for (int l = 0, k = 0; l < depth; ++l) {
    base[l] = k;
    k += p->n + 2 * ((p->n - (l & 1)) / 2);
  }
  cudaStream_t s = p->stream;
  cudaError_t e = cudaMemcpyAsync(p->U, unitaries, sizeof(double) * 8 * (size_t)p->n * depth, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->layer_base, base.data(), sizeof(int) * depth, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && angles)
    e = cudaMemcpyAsync(p->angles, angles, sizeof(double) * 2 * (size_t)nn * batch, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return report(IQS_ECUDA, "pool upload: %s", cudaGetErrorString(e));
  e = p->dtype == IQS_C128 ? run_pool<P128>(p, batch, depth, angles != nullptr)
                           : run_pool<P64>(p, batch, depth, angles != nullptr);
  if (e != cudaSuccess) return report(IQS_ECUDA, "pool launch: %s", cudaGetErrorString(e));
  if (probs) e = cudaMemcpyAsync(probs, p->probs, sizeof(double) * (size_t)p->n * batch, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(mean, p->mean, sizeof(double) * p->n, cudaMemcpyDeviceToHost, s);
  unsigned f = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&f, p->flag, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return report(IQS_ECUDA, "pool results: %s", cudaGetErrorString(e));
  if (f) {
    cudaMemsetAsync(p->flag, 0, sizeof(unsigned), s);
    return report(IQS_ERANGE, "an amplitude outside the emulated-FP64 range was met");
  }
  return IQS_OK;
}

iqs_status iqs_pool_download_state(iqs_pool* p, int index, void* host, size_t bytes) {
  using namespace iqs;
  if (p == nullptr || host == nullptr) return report(IQS_EINVAL, "NULL argument");
  const size_t amp = p->dtype == IQS_C128 ? 16 : 8;
  if (index < 0 || index >= p->bmax || bytes != amp * p->N) return report(IQS_EINVAL, "bad index or size");
  cudaError_t e = cudaMemcpyAsync(host, (const char*)p->psi + amp * p->N * index, bytes, cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return report(IQS_ECUDA, "download: %s", cudaGetErrorString(e));
  return IQS_OK;
}

}  // extern "C"
