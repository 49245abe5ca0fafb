// Cluster-resident pool engine: one thread-block cluster holds a whole
// trajectory's state in its distributed shared memory and runs every layer
// of the brick circuit on chip (Section 2, "Pool of multiple states"; the
// circuit family, noise and fused matrices are those of pool.cu).
//
// A cluster of C = 2^logc CTAs splits the 2^n amplitudes by their top logc
// bits: CTA r holds the 2^L amplitudes (L = n - logc) whose top bits equal r,
// in shared memory, XOR-swizzled within 16-element blocks so that register
// rounds on the lowest bits do not collide in the banks.  Per phase:
//   1. the fused one-qubit matrices of the phase (composed once per run by
//      k_pool_compose) are read into shared memory;
//   2. local register rounds apply the gates of qubits 0..L-1, up to
//      kRegBits qubits per round, one thread per 2^kRegBits-amplitude group;
//   3. the CNOT pairs with both qubits local swap their amplitudes in place
//      (the brick is a product of disjoint transpositions);
//   4. after a cluster barrier, an exchange round gathers, through
//      distributed shared memory, groups of 2C amplitudes spanning qubit L-1
//      and the logc top qubits: the top qubits' one-qubit gates are applied
//      and the amplitudes are stored back through the CNOT pairs that touch
//      the top qubits (the pair (L-1, L) included); a cluster barrier closes
//      the phase.
// After the last phase the state is written to HBM once (for inspection) and
// P(q = 1) / norm of every qubit is reduced across the cluster, in a fixed
// order.  Work comes as a table of jobs (one per trajectory: its matrices,
// qubit count, phases, and where its state and probabilities go), so one
// launch covers trajectories of different circuits, depths and qubit counts
// (all with the same cluster size).  HBM traffic per trajectory is that one write instead of two passes
// over the state per layer.
#include <algorithm>
#include <cooperative_groups.h>

#include "common.cuh"
#include "df64.cuh"
#include "internal.h"
#include "pool_common.cuh"
#include "qaoa_ops.cuh"

namespace cg = cooperative_groups;

namespace iqs {
namespace {

using namespace iqs::pool;

// Threads per CTA and resident CTAs per SM the registers are sized for: one
// 512-thread CTA holding a 128 KB slice per SM.
template <class TR>
struct CT {
  static constexpr int kThreads = 512;
  static constexpr int kMinBlocks = 1;
};
constexpr int kMaxLogC = 4;       // 16-CTA clusters need the non-portable size opt-in
// shared-memory slice per CTA
constexpr size_t kSliceBytes64 = 128 << 10, kSliceBytes128 = 128 << 10;

__device__ __forceinline__ unsigned phys(unsigned i) { return i ^ ((i >> 4) & 15u); }

template <class TR>
__device__ __forceinline__ typename TR::W zero_w();
template <>
__device__ __forceinline__ float2 zero_w<P64>() { return make_float2(0.f, 0.f); }
template <>
__device__ __forceinline__ qops::S2 zero_w<P128>() { return qops::S2{0.f, 0.f, 0.f, 0.f}; }
template <class TR>
__device__ __forceinline__ typename TR::W one_w();
template <>
__device__ __forceinline__ float2 one_w<P64>() { return make_float2(1.f, 0.f); }
template <>
__device__ __forceinline__ qops::S2 one_w<P128>() { return qops::S2{1.f, 0.f, 0.f, 0.f}; }

// Gates of the qubits [b0, b0 + RBT) on every local group (RBT <= kRegBits,
// a compile-time width so the group loops carry no predicates).  The round's
// matrices are read once into registers when they are small (complex64: 8
// floats each) and from shared memory otherwise.
template <class TR, int kCT, int RBT>
__device__ __forceinline__ void local_round(typename TR::W* st, const typename TR::Mat* mats, int b0, unsigned NL) {
  using W = typename TR::W;
  using Mat = typename TR::Mat;
  constexpr bool kRegMats = sizeof(Mat) <= 32;
  Mat mr[kRegMats ? RBT : 1];
  if constexpr (kRegMats) {
#pragma unroll
    for (int j = 0; j < RBT; ++j) mr[j] = mats[b0 + j];
  }
  const unsigned ngr = NL >> RBT;
  const unsigned lowm = (1u << b0) - 1u;
  auto apply_group = [&](W (&x)[1 << RBT]) {
#pragma unroll
    for (int j = 0; j < RBT; ++j) {
#pragma unroll
      for (int c = 0; c < (1 << RBT); ++c)
        if (!((c >> j) & 1)) {
          if constexpr (kRegMats) TR::apply(mr[j], x[c], x[c | (1 << j)]);
          else TR::apply(mats[b0 + j], x[c], x[c | (1 << j)]);
        }
    }
  };
  // complex64: two groups per iteration (their shared-memory loads overlap),
  // then a tail of one; complex128 groups are too large for two in registers
  unsigned g = threadIdx.x;
  for (; sizeof(W) == 8 && g + kCT < ngr; g += 2 * kCT) {
    const unsigned base0 = ((g >> b0) << (b0 + RBT)) | (g & lowm);
    const unsigned g1 = g + kCT;
    const unsigned base1 = ((g1 >> b0) << (b0 + RBT)) | (g1 & lowm);
    W x0[1 << RBT], x1[1 << RBT];
#pragma unroll
    for (int c = 0; c < (1 << RBT); ++c) {
      x0[c] = st[phys(base0 | ((unsigned)c << b0))];
      x1[c] = st[phys(base1 | ((unsigned)c << b0))];
    }
    apply_group(x0);
    apply_group(x1);
#pragma unroll
    for (int c = 0; c < (1 << RBT); ++c) {
      st[phys(base0 | ((unsigned)c << b0))] = x0[c];
      st[phys(base1 | ((unsigned)c << b0))] = x1[c];
    }
  }
  for (; g < ngr; g += kCT) {
    const unsigned base = ((g >> b0) << (b0 + RBT)) | (g & lowm);
    W x[1 << RBT];
#pragma unroll
    for (int c = 0; c < (1 << RBT); ++c) x[c] = st[phys(base | ((unsigned)c << b0))];
    apply_group(x);
#pragma unroll
    for (int c = 0; c < (1 << RBT); ++c) st[phys(base | ((unsigned)c << b0))] = x[c];
  }
}

template <class TR, int kCT>
__device__ __forceinline__ void local_round_any(typename TR::W* st, const typename TR::Mat* mats, int b0, int rb,
                                                unsigned NL) {
  switch (rb) {
    case 1: local_round<TR, kCT, 1>(st, mats, b0, NL); break;
    case 2: local_round<TR, kCT, 2>(st, mats, b0, NL); break;
    case 3: local_round<TR, kCT, 3>(st, mats, b0, NL); break;
    default:
      if constexpr (TR::kRegBits >= 4) local_round<TR, kCT, 4>(st, mats, b0, NL);
      break;
  }
}

// Exchange round: groups of 2C amplitudes whose element c has bit 0 = qubit
// L-1 (local) and bits 1.. = the CTA rank (the top qubits).  Rank r handles
// a 1/C share of the 2^(L-1) groups: it gathers each group through
// distributed shared memory, applies the gates of the top qubits (mats[L..]),
// and stores it back through the involution c -> c ^ ((c & cmg) << 1) (the
// CNOT pairs that touch the top qubits; cmg = 0 for none).  Callers bracket it
// with cluster barriers.
template <class TR, int LOGC, int kCT>
__device__ __forceinline__ void exchange_round(cg::cluster_group& cl, typename TR::W* st,
                                               const typename TR::Mat* mats, int L, unsigned rank, unsigned cmg) {
  using W = typename TR::W;
  constexpr int C = 1 << LOGC;
  const unsigned NL = 1u << L;
  const unsigned G = NL >> 1, per = G / C;
  const unsigned hib = 1u << (L - 1);
  for (unsigned g = rank * per + threadIdx.x; g < (rank + 1) * per; g += kCT) {
    W x[2 * C];
#pragma unroll
    for (int c = 0; c < 2 * C; ++c) {
      const W* rs = cl.map_shared_rank(st, (unsigned)(c >> 1));
      x[c] = rs[phys(g | ((c & 1) ? hib : 0u))];
    }
#pragma unroll
    for (int j = 0; j < LOGC; ++j) {
#pragma unroll
      for (int c = 0; c < 2 * C; ++c)
        if (!((c >> (j + 1)) & 1)) TR::apply(mats[L + j], x[c], x[c | (2 << j)]);
    }
#pragma unroll
    for (int c = 0; c < 2 * C; ++c) {
      const unsigned d = (unsigned)c ^ (((unsigned)c & cmg) << 1);
      W* rs = cl.map_shared_rank(st, d >> 1);
      rs[phys(g | ((d & 1) ? hib : 0u))] = x[c];
    }
  }
}

template <class TR, int LOGC>
__global__ void __launch_bounds__(CT<TR>::kThreads, CT<TR>::kMinBlocks)
    k_pool_cluster(const ClusterJob* __restrict__ jobs, int n_jobs) {
  constexpr int kCT = CT<TR>::kThreads;
  using W = typename TR::W;
  using Mat = typename TR::Mat;
  constexpr int C = 1 << LOGC;
  constexpr int RB = TR::kRegBits;
  cg::cluster_group cl = cg::this_cluster();
  const unsigned rank = cl.block_rank();
  extern __shared__ __align__(16) unsigned char raw[];
  W* st = reinterpret_cast<W*>(raw);
  __shared__ Mat mats[kPoolMaxQubits];
  __shared__ double part[C][kPoolMaxQubits + 1];  // read on rank 0: every rank's slice sums
  __shared__ double red[kCT / 32][kPoolMaxQubits + 1];
  const unsigned cid = blockIdx.x / C, ncl = gridDim.x / C;
  for (unsigned jb = cid; jb < (unsigned)n_jobs; jb += ncl) {
    const ClusterJob J = jobs[jb];
    const int n = J.n, phases = J.phases, depth = J.depth;
    const Mat* allm = static_cast<const Mat*>(J.mats);
    const int L = n - LOGC;
    const unsigned NL = 1u << L;
    for (unsigned i = threadIdx.x; i < NL; i += kCT) st[i] = zero_w<TR>();
    __syncthreads();
    if (rank == 0 && threadIdx.x == 0) st[0] = one_w<TR>();
    for (int l = 0; l < phases; ++l) {
      if ((int)threadIdx.x < n) mats[threadIdx.x] = allm[(uint64_t)l * n + threadIdx.x];
      __syncthreads();
      for (int b0 = 0; b0 < L; b0 += RB) {
        local_round_any<TR, kCT>(st, mats, b0, min(RB, L - b0), NL);
        __syncthreads();
      }
      const int o = l & 1;
      if (l < depth) {  // CNOT pairs (i, i + 1), i = o, o + 2, ..., both local
        unsigned cm = 0;
        for (int i = o; i + 1 < L; i += 2) cm |= 1u << i;
        if (cm) {
          for (unsigned x = threadIdx.x; x < NL; x += kCT) {
            const unsigned y = x ^ ((x & cm) << 1);
            if (y > x) {
              const W t = st[phys(x)];
              st[phys(x)] = st[phys(y)];
              st[phys(y)] = t;
            }
          }
        }
      }
      if constexpr (LOGC > 0) {
        cl.sync();
        unsigned cmg = 0;
        if (l < depth)
          for (int i = o; i + 1 < n; i += 2)
            if (i >= L - 1) cmg |= 1u << (i - (L - 1));
        exchange_round<TR, LOGC, kCT>(cl, st, mats, L, rank, cmg);
        cl.sync();
      } else {
        __syncthreads();
      }
    }
    // the final state, once, to HBM (logical order)
    typename TR::V* out = static_cast<typename TR::V*>(J.psi) + (uint64_t)rank * NL;
    for (unsigned i = threadIdx.x; i < NL; i += kCT) out[i] = TR::store(st[phys(i)]);
    // P(q = 1) and the norm of this slice: double-float per thread, FP64
    // across; in groups of 8 sums (slot 24 is the norm) to bound registers
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q0 = 0; q0 <= kPoolMaxQubits; q0 += 8) {
      dfx::Acc acc[8];
      for (unsigned i = threadIdx.x; i < NL; i += kCT) {
        float p, e;
        TR::abs2(st[phys(i)], p, e);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int q = q0 + k;
          if (q == kPoolMaxQubits || (q < L && ((i >> q) & 1u))) acc[k].add(p, e);
        }
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (q0 + k > kPoolMaxQubits) break;
        double v = acc[k].value();
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][q0 + k] = v;
      }
    }
    __syncthreads();
    if ((int)threadIdx.x <= kPoolMaxQubits) {
      double s = 0.0;
      for (int w = 0; w < kCT / 32; ++w) s += red[w][threadIdx.x];
      double* p0 = cl.map_shared_rank(&part[0][0], 0u);
      p0[rank * (kPoolMaxQubits + 1) + threadIdx.x] = s;
    }
    cl.sync();
    if (rank == 0 && (int)threadIdx.x < n) {
      const int q = threadIdx.x;
      double norm = 0.0, pq = 0.0;
      for (int r = 0; r < C; ++r) {
        norm += part[r][kPoolMaxQubits];
        if (q < L) pq += part[r][q];
        else if ((r >> (q - L)) & 1) pq += part[r][kPoolMaxQubits];
      }
      J.probs[q] = pq / norm;
    }
    cl.sync();  // rank 0 has read part[] before any rank writes the next trajectory's sums
  }
}

// ---------------------------------------------------------------- QAOA forward on clusters
// Section 4's objective, energies only: state b (graph b / per_graph) starts
// in |+>^n (every amplitude 2^(-n/2)); each layer multiplies amplitude x by the
// phase table entry T_b[C(x)] (C read from the graph's one-byte cut table),
// then applies RX(2 beta) to every qubit through the local rounds and one
// exchange round; at the end E_b = sum C(x) |psi_x|^2 / sum |psi_x|^2
// (double-float per thread, FP64 across the cluster in a fixed order) goes to
// results[b * rstride] and the final state to phi[b] (complex64).
template <int LOGC>
__global__ void __launch_bounds__(CT<P64>::kThreads, 1)
    k_qaoa_cluster(const uint8_t* __restrict__ cut, uint64_t N, int per_graph, const float2* __restrict__ rx,
                   const float2* __restrict__ tables, int tsize, int bmax, int n, int p, int batch,
                   float2* __restrict__ phi, double* __restrict__ results, int rstride) {
  using TR = P64;
  using W = float2;
  using Mat = P64::Mat;
  constexpr int kCT = CT<P64>::kThreads;
  constexpr int C = 1 << LOGC;
  constexpr int RB = TR::kRegBits;
  cg::cluster_group cl = cg::this_cluster();
  const unsigned rank = cl.block_rank();
  const int L = n - LOGC;
  const unsigned NL = 1u << L;
  extern __shared__ __align__(16) unsigned char raw[];
  W* st = reinterpret_cast<W*>(raw);
  __shared__ Mat mats[kPoolMaxQubits];
  __shared__ float2 ph[256];
  __shared__ double part[C][2];
  __shared__ double red[kCT / 32][2];
  const float amp0 = (float)exp2(-0.5 * n);
  const unsigned cid = blockIdx.x / C, ncl = gridDim.x / C;
  for (unsigned b = cid; b < (unsigned)batch; b += ncl) {
    const uint8_t* cb = cut + (uint64_t)(b / (unsigned)per_graph) * N + (uint64_t)rank * NL;
    for (unsigned i = threadIdx.x; i < NL; i += kCT) st[i] = make_float2(amp0, 0.f);
    for (int l = 0; l < p; ++l) {
      const uint64_t lb = (uint64_t)l * bmax + b;
      for (int k = threadIdx.x; k < tsize; k += kCT) ph[k] = tables[lb * tsize + k];
      if ((int)threadIdx.x < n) {
        const float2 k = rx[lb];  // (cos beta, sin beta): RX(2 beta) = [[c, -i s], [-i s, c]]
        Mat m;
        m.r[0] = k.x; m.i[0] = 0.f; m.r[1] = 0.f;  m.i[1] = -k.y;
        m.r[2] = 0.f; m.i[2] = -k.y; m.r[3] = k.x; m.i[3] = 0.f;
        mats[threadIdx.x] = m;
      }
      __syncthreads();
      for (unsigned i = threadIdx.x; i < NL; i += kCT) {  // cost phase
        const float2 t = ph[cb[i]];
        const float2 x = st[phys(i)];
        st[phys(i)] = make_float2(t.x * x.x - t.y * x.y, t.x * x.y + t.y * x.x);
      }
      __syncthreads();
      for (int b0 = 0; b0 < L; b0 += RB) {
        local_round_any<TR, kCT>(st, mats, b0, min(RB, L - b0), NL);
        __syncthreads();
      }
      if constexpr (LOGC > 0) {
        cl.sync();
        exchange_round<TR, LOGC, kCT>(cl, st, mats, L, rank, 0u);
        cl.sync();
      }
    }
    float2* out = phi + (uint64_t)b * N + (uint64_t)rank * NL;
    dfx::Acc ae, an;
    for (unsigned i = threadIdx.x; i < NL; i += kCT) {
      const float2 x = st[phys(i)];
      out[i] = x;
      float pp, ee;
      dfx::abs2_c64(x.x, x.y, pp, ee);
      an.add(pp, ee);
      const float cf = (float)cb[i];
      const float q = cf * pp;
      ae.add(q, fmaf(cf, pp, -q) + cf * ee);
    }
    double v[2] = {ae.value(), an.value()};
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
      if (lane == 0) red[warp][k] = v[k];
    }
    __syncthreads();
    if (threadIdx.x < 2) {
      double sum = 0.0;
      for (int w = 0; w < kCT / 32; ++w) sum += red[w][threadIdx.x];
      double* p0 = cl.map_shared_rank(&part[0][0], 0u);
      p0[rank * 2 + threadIdx.x] = sum;
    }
    cl.sync();
    if (rank == 0 && threadIdx.x == 0) {
      double e = 0.0, nn = 0.0;
      for (int r = 0; r < C; ++r) {
        e += part[r][0];
        nn += part[r][1];
      }
      results[(uint64_t)b * rstride] = e / nn;
    }
    cl.sync();
  }
}

// Launch configuration; with ``clusters`` it also sets the kernel's
// attributes and queries the co-resident cluster count (done once, outside
// any stream capture).
template <int LOGC>
cudaError_t qaoa_cluster_config(int n, cudaLaunchConfig_t& cfg, cudaLaunchAttribute* attr, int* clusters) {
  auto kern = k_qaoa_cluster<LOGC>;
  const size_t smem = ((size_t)1 << (n - LOGC)) * sizeof(float2);
  cudaError_t e = cudaSuccess;
  if (clusters) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && LOGC > 3) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cfg = {};
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 1u << LOGC;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(CT<P64>::kThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(1u << LOGC, 1, 1);
  return clusters ? cudaOccupancyMaxActiveClusters(clusters, kern, &cfg) : cudaSuccess;
}

template <int LOGC>
cudaError_t launch_qaoa_t(int clusters, const uint8_t* cut, uint64_t N, int per_graph, const float2* rx,
                          const float2* tables, int tsize, int bmax, int n, int p, int batch, float2* phi,
                          double* results, int rstride, cudaStream_t s) {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  cudaError_t e = qaoa_cluster_config<LOGC>(n, cfg, attr, nullptr);
  if (e != cudaSuccess) return e;
  cfg.stream = s;
  cfg.gridDim = dim3((unsigned)std::max(1, std::min(clusters, batch)) << LOGC, 1, 1);
  return cudaLaunchKernelEx(&cfg, k_qaoa_cluster<LOGC>, cut, N, per_graph, rx, tables, tsize, bmax, n, p, batch, phi,
                            results, rstride);
}

int cluster_logc(int n, int dtype) {
  const size_t w = dtype == IQS_C128 ? sizeof(qops::S2) : sizeof(float2);
  const size_t slice = dtype == IQS_C128 ? kSliceBytes128 : kSliceBytes64;
  const size_t bytes = ((size_t)1 << n) * w;
  for (int lc = 0; lc <= kMaxLogC; ++lc)
    if ((bytes >> lc) <= slice && n >= 2 * lc + 1 && n - lc >= 8) return lc;
  return -1;
}

template <class TR, int LOGC>
cudaError_t launch_cluster_t(const ClusterJob* jobs, int n_jobs, int max_n, cudaStream_t s) {
  auto kern = k_pool_cluster<TR, LOGC>;
  const size_t smem = ((size_t)1 << (max_n - LOGC)) * sizeof(typename TR::W);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && LOGC > 3) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 1u << LOGC;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(CT<TR>::kThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(1u << LOGC, 1, 1);
  int clusters = 0;
  e = cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg);
  if (e != cudaSuccess) return e;
  if (clusters < 1) return cudaErrorInvalidConfiguration;  // this cluster size cannot be scheduled
  clusters = std::min(clusters, n_jobs);
  cfg.gridDim = dim3((unsigned)clusters << LOGC, 1, 1);
  return cudaLaunchKernelEx(&cfg, kern, jobs, n_jobs);
}

}  // namespace

bool pool_cluster_eligible(int n, int dtype) { return cluster_logc(n, dtype) >= 0; }

int pool_cluster_logc(int n, int dtype) { return cluster_logc(n, dtype); }

// Whether an n-qubit state may be split over 2^lc CTAs: at least the smallest
// cluster that holds it, at most kMaxLogC, n >= 2 lc + 1 and n - lc >= 8.
bool pool_cluster_logc_ok(int n, int dtype, int lc) {
  const int lo = cluster_logc(n, dtype);
  return lo >= 0 && lc >= lo && lc <= kMaxLogC && n >= 2 * lc + 1 && n - lc >= 8;
}

cudaError_t launch_pool_cluster_raw(const ClusterJob* jobs, int n_jobs, int max_n, int dtype, cudaStream_t s, int logc);

// Jobs of qubit counts in [2 logc + 1, max_n] on clusters of 2^logc CTAs
// (logc = ``logc`` when pool_cluster_logc_ok, else pool_cluster_logc(max_n,
// dtype)); ``jobs`` is a device array.
cudaError_t launch_pool_cluster(const ClusterJob* jobs, int n_jobs, int max_n, int dtype, cudaStream_t s, int logc) {
  const cudaError_t e = launch_pool_cluster_raw(jobs, n_jobs, max_n, dtype, s, logc);
  return e == cudaSuccess && n_jobs >= 1 ? launched(1) : e;
}

cudaError_t launch_pool_cluster_raw(const ClusterJob* jobs, int n_jobs, int max_n, int dtype, cudaStream_t s,
                                    int logc) {
  const int lc = pool_cluster_logc_ok(max_n, dtype, logc) ? logc : cluster_logc(max_n, dtype);
  cudaError_t e = cudaErrorInvalidValue;
  if (n_jobs < 1) return cudaSuccess;
  if (dtype == IQS_C128) {
    switch (lc) {
      case 0: e = launch_cluster_t<P128, 0>(jobs, n_jobs, max_n, s); break;
      case 1: e = launch_cluster_t<P128, 1>(jobs, n_jobs, max_n, s); break;
      case 2: e = launch_cluster_t<P128, 2>(jobs, n_jobs, max_n, s); break;
      case 3: e = launch_cluster_t<P128, 3>(jobs, n_jobs, max_n, s); break;
      case 4: e = launch_cluster_t<P128, 4>(jobs, n_jobs, max_n, s); break;
      default: break;
    }
  } else {
    switch (lc) {
      case 0: e = launch_cluster_t<P64, 0>(jobs, n_jobs, max_n, s); break;
      case 1: e = launch_cluster_t<P64, 1>(jobs, n_jobs, max_n, s); break;
      case 2: e = launch_cluster_t<P64, 2>(jobs, n_jobs, max_n, s); break;
      case 3: e = launch_cluster_t<P64, 3>(jobs, n_jobs, max_n, s); break;
      case 4: e = launch_cluster_t<P64, 4>(jobs, n_jobs, max_n, s); break;
      default: break;
    }
  }
  return e;
}

// QAOA forward on clusters (complex64): the cluster size for n qubits and the
// number of co-resident clusters (0 when the kernel cannot run), queried once.
int qaoa_cluster_setup(int n, int* logc) {
  const int lc = cluster_logc(n, IQS_C64);
  *logc = lc;
  if (lc < 0) return 0;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  int clusters = 0;
  cudaError_t e = cudaErrorInvalidValue;
  switch (lc) {
    case 0: e = qaoa_cluster_config<0>(n, cfg, attr, &clusters); break;
    case 1: e = qaoa_cluster_config<1>(n, cfg, attr, &clusters); break;
    case 2: e = qaoa_cluster_config<2>(n, cfg, attr, &clusters); break;
    case 3: e = qaoa_cluster_config<3>(n, cfg, attr, &clusters); break;
    case 4: e = qaoa_cluster_config<4>(n, cfg, attr, &clusters); break;
    default: break;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return clusters;
}

cudaError_t launch_qaoa_cluster(int logc, int clusters, const uint8_t* cut, uint64_t N, int per_graph,
                                const float2* rx, const float2* tables, int tsize, int bmax, int n, int p, int batch,
                                float2* phi, double* results, int rstride, cudaStream_t s) {
  switch (logc) {
    case 0: return launch_qaoa_t<0>(clusters, cut, N, per_graph, rx, tables, tsize, bmax, n, p, batch, phi, results, rstride, s);
    case 1: return launch_qaoa_t<1>(clusters, cut, N, per_graph, rx, tables, tsize, bmax, n, p, batch, phi, results, rstride, s);
    case 2: return launch_qaoa_t<2>(clusters, cut, N, per_graph, rx, tables, tsize, bmax, n, p, batch, phi, results, rstride, s);
    case 3: return launch_qaoa_t<3>(clusters, cut, N, per_graph, rx, tables, tsize, bmax, n, p, batch, phi, results, rstride, s);
    case 4: return launch_qaoa_t<4>(clusters, cut, N, per_graph, rx, tables, tsize, bmax, n, p, batch, phi, results, rstride, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace iqs
