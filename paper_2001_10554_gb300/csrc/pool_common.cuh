// Device pieces shared by the pool engines: FP64 2x2 algebra for composing a
// trajectory's fused one-qubit matrices, the brick-circuit description, and
// the storage traits (complex64 / split complex128) of the pool tiles.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "df64.cuh"
#include "qaoa_ops.cuh"
#include "tile.cuh"

namespace iqs {
namespace pool {

using qops::S2;

constexpr int kPoolMaxQubits = 24;

// ---------------------------------------------------------------- FP64 2x2 algebra (per block, a few matrices)
struct M2 {
  double r[4], i[4];  // row-major U00 U01 U10 U11
};

__device__ __forceinline__ M2 mmul(const M2& a, const M2& b) {
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

__device__ __forceinline__ M2 identity2() {
  M2 m;
  m.r[0] = 1.0; m.i[0] = 0.0; m.r[1] = 0.0; m.i[1] = 0.0;
  m.r[2] = 0.0; m.i[2] = 0.0; m.r[3] = 1.0; m.i[3] = 0.0;
  return m;
}

// RZ(tz) . RX(tx), R(t) = exp(-i t sigma / 2)
__device__ __forceinline__ M2 noise_rot(double tx, double tz) {
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

// RZ(tz) . RY(ty) . RX(tx): the T1/T2 noise gate (RX acts first).
__device__ __forceinline__ M2 noise_rot3(double tx, double ty, double tz) {
  double sy, cy;
  sincos(0.5 * ty, &sy, &cy);
  M2 ry;  // [[cy, -sy], [sy, cy]]
  ry.r[0] = cy;  ry.i[0] = 0.0; ry.r[1] = -sy; ry.i[1] = 0.0;
  ry.r[2] = sy;  ry.i[2] = 0.0; ry.r[3] = cy;  ry.i[3] = 0.0;
  const M2 x = noise_rot(tx, 0.0);  // RX
  const M2 z = noise_rot(0.0, tz);  // RZ
  return mmul(z, mmul(ry, x));
}

struct Circuit {
  int n, depth;
  const double* U;          // [depth][n][8]
  const double* angles;     // [batch][n_noise][width] or nullptr
  const int* layer_base;    // [depth]: index of the first noise op of layer l
  int n_noise;
  // noise model: 0 = angle pairs (tx, tz) as given (RX then RZ); 1 = T1/T2
  // gates: standard normal triples scaled by sig (RX, RY, RZ)
  int model = 0;
  double sig[3] = {0.0, 0.0, 0.0};
  __host__ __device__ int width() const { return model == 1 ? 3 : 2; }
};

// Noise rotation k of one trajectory whose draws start at ``ang``.
__device__ __forceinline__ M2 noise_op(const Circuit& C, const double* ang, int k) {
  if (C.model == 1) {
    const double* z = ang + 3 * k;
    return noise_rot3(C.sig[0] * z[0], C.sig[1] * z[1], C.sig[2] * z[2]);
  }
  return noise_rot(ang[2 * k], ang[2 * k + 1]);
}

// Fused one-qubit matrix of phase l (0..depth) for qubit q of one trajectory
// whose noise draws start at ``ang`` (nullptr: noiseless).
__device__ __forceinline__ M2 compose_traj(const Circuit& C, const double* ang, int l, int q) {
  M2 G = identity2();
  if (ang && l > 0) {
    const int o = (l - 1) & 1;
    const int d = q - o;
    if (d >= 0) {
      const int j = d >> 1;
      const int ctrl = o + 2 * j;
      if (ctrl + 1 < C.n) {
        const int k = C.layer_base[l - 1] + C.n + 2 * j + (q == ctrl ? 0 : 1);
        G = noise_op(C, ang, k);
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
    if (ang) G = mmul(noise_op(C, ang, C.layer_base[l] + q), G);
  }
  return G;
}

// The same for trajectory b of a circuit whose draws are stored [b][n_noise][width].
__device__ __forceinline__ M2 compose(const Circuit& C, int b, int l, int q) {
  return compose_traj(C, C.angles ? C.angles + (uint64_t)b * C.n_noise * C.width() : nullptr, l, q);
}

// One trajectory for the cluster-resident engine.
struct ClusterJob {
  const void* mats;  // [phases][n] fused matrices in the dtype's Mat format
  void* psi;         // the final state, 2^n amplitudes
  double* probs;     // P(q = 1) / norm, n values
  int n, phases, depth;
};

// ---------------------------------------------------------------- storage traits
struct P64 {
  using V = float2;
  using W = float2;
  struct Mat {
    float r[4], i[4];
  };
  static constexpr int kTileBits = 12, kRowBits = 4, kRegBits = 4, kSwzBits = 4;
  static constexpr int kMinBlocks = 3;  // resident pass blocks per SM the registers are sized for
  static constexpr bool kTmaSwizzle = false;
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
  static constexpr int kMinBlocks = 2;
  static constexpr bool kTmaSwizzle = false;
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

// One tile of one pass: load the tile (L2 loads: another SM may have written
// the state), apply the one-qubit matrices ``mats`` of the ``ng`` qubits whose
// local bits start at ``lb0`` in register rounds, then write back through the
// CNOT permutation new[l] = old[l ^ ((l & cmask) << 1)].
template <class TR>
__device__ __forceinline__ void pool_tile(typename TR::W* sp, const typename TR::Mat* mats, typename TR::V* P,
                                          const Geo& g, uint64_t t, int lb0, int ng, unsigned cmask, unsigned& bad) {
  using W = typename TR::W;
  using Mat = typename TR::Mat;
  constexpr int R = TR::kRegBits;
  constexpr int RB = 1 << R;
  const unsigned T = 1u << (g.c + g.m);
  for (unsigned l = threadIdx.x; l < T; l += blockDim.x) sp[swz<TR>(l)] = TR::load(__ldcg(P + tile_x(g, t, l)), bad);
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
  for (unsigned l = threadIdx.x; l < T; l += blockDim.x) P[tile_x(g, t, l)] = TR::store(sp[swz<TR>(l ^ ((l & cmask) << 1))]);
  __syncthreads();
}

}  // namespace pool
}  // namespace iqs
