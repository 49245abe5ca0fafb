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
constexpr int kMaxLogC = 3;       // portable clusters (8 CTAs)
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
  for (unsigned g = threadIdx.x; g < ngr; g += kCT) {
    const unsigned base = ((g >> b0) << (b0 + RBT)) | (g & lowm);
    W x[1 << RBT];
#pragma unroll
    for (int c = 0; c < (1 << RBT); ++c) x[c] = st[phys(base | ((unsigned)c << b0))];
#pragma unroll
    for (int j = 0; j < RBT; ++j) {
#pragma unroll
      for (int c = 0; c < (1 << RBT); ++c)
        if (!((c >> j) & 1)) {
          if constexpr (kRegMats) TR::apply(mr[j], x[c], x[c | (1 << j)]);
          else TR::apply(mats[b0 + j], x[c], x[c | (1 << j)]);
        }
    }
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
        // exchange: element c of a group has bit 0 = qubit L-1 and bits 1.. = the rank
        unsigned cmg = 0;
        if (l < depth)
          for (int i = o; i + 1 < n; i += 2)
            if (i >= L - 1) cmg |= 1u << (i - (L - 1));
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
          // new[perm(c)] = old[c] for the involution perm(c) = c ^ ((c & cmg) << 1)
#pragma unroll
          for (int c = 0; c < 2 * C; ++c) {
            const unsigned d = (unsigned)c ^ (((unsigned)c & cmg) << 1);
            W* rs = cl.map_shared_rank(st, d >> 1);
            rs[phys(g | ((d & 1) ? hib : 0u))] = x[c];
          }
        }
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
  clusters = std::max(1, std::min(clusters, n_jobs));
  cfg.gridDim = dim3((unsigned)clusters << LOGC, 1, 1);
  return cudaLaunchKernelEx(&cfg, kern, jobs, n_jobs);
}

}  // namespace

bool pool_cluster_eligible(int n, int dtype) { return cluster_logc(n, dtype) >= 0; }

int pool_cluster_logc(int n, int dtype) { return cluster_logc(n, dtype); }

// Jobs of qubit counts in [2 logc + 1, max_n] on clusters of 2^logc CTAs
// (logc = pool_cluster_logc(max_n, dtype)); ``jobs`` is a device array.
cudaError_t launch_pool_cluster(const ClusterJob* jobs, int n_jobs, int max_n, int dtype, cudaStream_t s) {
  const int lc = cluster_logc(max_n, dtype);
  cudaError_t e = cudaErrorInvalidValue;
  if (n_jobs < 1) return cudaSuccess;
  if (dtype == IQS_C128) {
    switch (lc) {
      case 0: e = launch_cluster_t<P128, 0>(jobs, n_jobs, max_n, s); break;
      case 1: e = launch_cluster_t<P128, 1>(jobs, n_jobs, max_n, s); break;
      case 2: e = launch_cluster_t<P128, 2>(jobs, n_jobs, max_n, s); break;
      case 3: e = launch_cluster_t<P128, 3>(jobs, n_jobs, max_n, s); break;
      default: break;
    }
  } else {
    switch (lc) {
      case 0: e = launch_cluster_t<P64, 0>(jobs, n_jobs, max_n, s); break;
      case 1: e = launch_cluster_t<P64, 1>(jobs, n_jobs, max_n, s); break;
      case 2: e = launch_cluster_t<P64, 2>(jobs, n_jobs, max_n, s); break;
      case 3: e = launch_cluster_t<P64, 3>(jobs, n_jobs, max_n, s); break;
      default: break;
    }
  }
  return e == cudaSuccess ? launched(1) : e;
}

}  // namespace iqs
