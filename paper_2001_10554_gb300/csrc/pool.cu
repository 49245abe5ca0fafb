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
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "df64.cuh"
#include "internal.h"
#include "qaoa_ops.cuh"
#include "tile.cuh"
#include "pool_common.cuh"

namespace iqs {

// pool_cluster.cu
bool pool_cluster_eligible(int n, int dtype);
int pool_cluster_logc(int n, int dtype);
cudaError_t launch_pool_cluster(const pool::ClusterJob* jobs, int n_jobs, int max_n, int dtype, cudaStream_t s,
                                int logc);
bool pool_cluster_logc_ok(int n, int dtype, int lc);
// the same launch without counting it (for graph capture)
cudaError_t launch_pool_cluster_raw(const pool::ClusterJob* jobs, int n_jobs, int max_n, int dtype, cudaStream_t s,
                                    int logc);

namespace {

using qops::S2;
using namespace iqs::pool;

// ---------------------------------------------------------------- one pass
// Tile: row bits [0, g.c), gate bits [g.s, g.s + g.m).  One-qubit gates on the
// qubits [q_lo, q_hi) (all inside the gate bits), then the CNOTs whose
// controls are the local bits in ``cmask``.
template <class TR>
__global__ void __launch_bounds__(kThreads, TR::kMinBlocks) k_pool_pass(typename TR::V* __restrict__ psi, uint64_t N, Geo g, int q_lo,
                                                        int q_hi, unsigned cmask,
                                                        const typename TR::Mat* __restrict__ allm, int phases, int nq,
                                                        int layer,
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
  // fused matrices composed once per run by k_pool_compose: [b][phase][qubit]
  if ((int)threadIdx.x < ng) mats[threadIdx.x] = allm[((uint64_t)b * phases + layer) * nq + q_lo + threadIdx.x];
  __syncthreads();
  // local bit of qubit q: q - s + c for a high pass, q for the low pass
  const int lb0 = (g.c == 0 && g.s == 0) ? q_lo : (q_lo - g.s + g.c);
  typename TR::V* P = psi + (uint64_t)b * N;
  const uint64_t tiles = N >> K;
  unsigned bad = 0;
  for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) pool_tile<TR>(sp, mats, P, g, t, lb0, ng, cmask, bad);
  if (bad) atomicOr(flag, 1u);
}

// Fused one-qubit matrix of every (trajectory, phase, qubit), composed once
// in FP64 (sincos of the noise angles) instead of once per tile.
template <class TR>
__global__ void k_pool_compose(Circuit C, int batch, int phases, typename TR::Mat* __restrict__ out) {
  const uint64_t total = (uint64_t)batch * phases * C.n;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total; i += (uint64_t)gridDim.x * blockDim.x) {
    const int q = (int)(i % C.n);
    const uint64_t bl = i / C.n;
    const int l = (int)(bl % phases);
    const int b = (int)(bl / phases);
    out[i] = TR::make(compose(C, b, l, q));
  }
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
  void* mats = nullptr;  // [batch_max][depth_max + 1][n] fused matrices in the kernel's format
  iqs::pool::ClusterJob* cjobs = nullptr;  // [batch_max] job table of the cluster-resident engine
  double* partials = nullptr;
  double* probs = nullptr;
  double* mean = nullptr;
  unsigned* flag = nullptr;
  size_t angle_cap = 0;  // doubles
  int part_stride = 0, nblk = 0;
  int engine = 0;  // 0 auto (cluster-resident when the state fits), 1 tiled passes, 2 cluster-resident
  int logc = -1;   // cluster size 2^logc of the cluster-resident engine (-1: the smallest that holds a state)
  int noise_model = 0;       // 0 angle pairs (tx, tz); 1 T1/T2 gates from normal triples
  double sig[3] = {0, 0, 0};  // T1/T2 gate angle standard deviations (x, y, z)
  // runs captured as CUDA graphs, per (batch, depth, noisy, engine path): the
  // executable graph and the kernels it launches (path 0: tiled passes;
  // 1 + logc: the cluster-resident engine on clusters of 2^logc CTAs)
  std::map<std::tuple<int, int, int, int>, std::pair<cudaGraphExec_t, int>> graphs;
  std::tuple<int, int, int> cjobs_key{-1, -1, -1};  // (batch, depth, noisy) of the job table in cjobs
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

// The circuit description the compose kernel reads (device pointers and the noise law).
Circuit circuit_of(const iqs_pool* P, int depth, bool noisy) {
  Circuit C{P->n, depth, P->U, noisy ? P->angles : nullptr, P->layer_base, n_noise_ops(P->n, depth)};
  C.model = P->noise_model;
  for (int k = 0; k < 3; ++k) C.sig[k] = P->sig[k];
  return C;
}

// The tiled-pass run: fused matrices, |0>, the layer passes, then per-trajectory
// P(1) and the pool mean.  ``launches`` counts the kernels enqueued.
template <class TR>
void enqueue_tiled(iqs_pool* P, int batch, int depth, bool noisy, int* launches) {
  using V = typename TR::V;
  using Mat = typename TR::Mat;
  const uint64_t N = P->N;
  cudaStream_t s = P->stream;
  V* psi = (V*)P->psi;
  Mat* allm = (Mat*)P->mats;
  const int phases = noisy ? depth + 1 : depth;
  const std::vector<Pass> passes = plan_pool(P->n, TR::kTileBits, TR::kRowBits);
  k_pool_compose<TR><<<grid_for((uint64_t)batch * phases * P->n, 1, 8), kThreads, 0, s>>>(circuit_of(P, depth, noisy),
                                                                                        batch, phases, allm);
  k_basis0_batch<V><<<grid_for(N * batch, 1, 16), kThreads, 0, s>>>(psi, N, batch);
  int count = 2;
  for (int l = 0; l < phases; ++l) {
    for (const Pass& p : passes) {
      const unsigned K = p.g.c + p.g.m;
      const uint64_t tiles = N >> K;
      const unsigned gx = (unsigned)std::min<uint64_t>(tiles, (uint64_t)std::max(1, 2432 / batch));
      const unsigned cm = l < depth ? cnot_mask(p, P->n, l) : 0u;
      const size_t smem = ((size_t)1 << K) * sizeof(typename TR::W);
      k_pool_pass<TR><<<dim3(std::max(1u, gx), batch), kThreads, smem, s>>>(psi, N, p.g, p.q_lo, p.q_hi, cm, allm,
                                                                            phases, P->n, l, P->flag);
      ++count;
    }
  }
  const dim3 gp(P->nblk, batch);
  k_pool_probs<TR><<<gp, kThreads, 0, s>>>(psi, N, P->n, P->partials, P->part_stride, P->flag);
  k_pool_finish<<<batch, 32, 0, s>>>(P->partials, P->part_stride, P->nblk, P->n, P->probs);
  k_pool_mean<<<P->n, kThreads, 0, s>>>(P->probs, batch, P->n, P->mean);
  *launches = count + 3;
}

template <class TR>
cudaError_t run_pool(iqs_pool* P, int batch, int depth, bool noisy) {
  using V = typename TR::V;
  const uint64_t N = P->N;
  cudaStream_t s = P->stream;
  V* psi = (V*)P->psi;
  const int phases = noisy ? depth + 1 : depth;
  using Mat = typename TR::Mat;
  Mat* allm = (Mat*)P->mats;
  // auto: the cluster-resident engine for complex64; complex128 runs faster in the tiled passes
  // (up to 4-CTA clusters: larger clusters keep fewer states on chip at once)
  const bool cluster = P->engine == 2 || (P->engine == 0 && P->dtype == IQS_C64 && pool_cluster_eligible(P->n, P->dtype) &&
                                          pool_cluster_logc(P->n, P->dtype) <= 2);
  if (cluster) {
    // the whole circuit of every trajectory in one launch, states resident in
    // cluster shared memory; compose, cluster launch and mean are captured as a
    // CUDA graph per shape and replayed (the job table, fixed per shape, is
    // uploaded before the capture when the shape changes)
    const auto jkey = std::make_tuple(batch, depth, noisy ? 1 : 0);
    if (P->cjobs_key != jkey) {
      std::vector<ClusterJob> jobs(batch);
      for (int b = 0; b < batch; ++b)
        jobs[b] = ClusterJob{allm + (uint64_t)b * phases * P->n, psi + (uint64_t)b * N, P->probs + (uint64_t)b * P->n,
                             P->n, phases, depth};
      cudaError_t e = cudaMemcpyAsync(P->cjobs, jobs.data(), sizeof(ClusterJob) * batch, cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return e;
      P->cjobs_key = jkey;
    }
    auto enqueue_cluster = [&](int* launches) {
      k_pool_compose<TR><<<grid_for((uint64_t)batch * phases * P->n, 1, 8), kThreads, 0, s>>>(
          circuit_of(P, depth, noisy), batch, phases, allm);
      cudaError_t e = cudaGetLastError();
      if (e == cudaSuccess) e = launch_pool_cluster_raw(P->cjobs, batch, P->n, P->dtype, s, P->logc);
      if (e == cudaSuccess) {
        k_pool_mean<<<P->n, kThreads, 0, s>>>(P->probs, batch, P->n, P->mean);
        e = cudaGetLastError();
      }
      *launches = 3;
      return e;
    };
    const int lc = pool_cluster_logc_ok(P->n, P->dtype, P->logc) ? P->logc : pool_cluster_logc(P->n, P->dtype);
    const auto key = std::make_tuple(batch, depth, noisy ? 1 : 0, 1 + lc);
    auto it = P->graphs.find(key);
    if (it == P->graphs.end()) {
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed);
      if (e != cudaSuccess) {  // a stream that cannot be captured (the legacy default stream): launch directly
        cudaGetLastError();
        int launches = 0;
        e = enqueue_cluster(&launches);
        if (e == cudaSuccess) note_launches(launches);
        return e;
      }
      int launches = 0;
      const cudaError_t ee = enqueue_cluster(&launches);
      e = cudaStreamEndCapture(s, &graph);
      if (ee != cudaSuccess) e = ee;
      cudaGraphExec_t exec = nullptr;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (e != cudaSuccess) return e;
      it = P->graphs.emplace(key, std::make_pair(exec, launches)).first;
    }
    const cudaError_t e = cudaGraphLaunch(it->second.first, s);
    if (e == cudaSuccess) note_launches(it->second.second);
    return e;
  }
  // tiled passes: about two launches per layer, replayed from a CUDA graph
  // captured on the first run of each (batch, depth, noisy) shape; the inputs
  // live in fixed device buffers, so a replay reads each call's unitaries and angles
  const auto key = std::make_tuple(batch, depth, noisy ? 1 : 0, 0);
  auto it = P->graphs.find(key);
  if (it == P->graphs.end()) {
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {  // a stream that cannot be captured (the legacy default stream): launch directly
      cudaGetLastError();
      int launches = 0;
      enqueue_tiled<TR>(P, batch, depth, noisy, &launches);
      e = cudaGetLastError();
      if (e == cudaSuccess) note_launches(launches);
      return e;
    }
    int launches = 0;
    enqueue_tiled<TR>(P, batch, depth, noisy, &launches);
    const cudaError_t ee = cudaGetLastError();
    e = cudaStreamEndCapture(s, &graph);
    if (ee != cudaSuccess) e = ee;
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) return e;
    it = P->graphs.emplace(key, std::make_pair(exec, launches)).first;
  }
  const cudaError_t e = cudaGraphLaunch(it->second.first, s);
  if (e == cudaSuccess) note_launches(it->second.second);
  return e;
}

template <class TR>
cudaError_t set_pool_attrs() {
  return cudaFuncSetAttribute(k_pool_pass<TR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (1 << TR::kTileBits) * (int)sizeof(typename TR::W));
}

void drop_graphs(iqs_pool* p) {
  for (auto& kv : p->graphs) cudaGraphExecDestroy(kv.second.first);
  p->graphs.clear();
}

void free_pool(iqs_pool* p) {
  drop_graphs(p);
  cudaFree(p->psi);
  cudaFree(p->U);
  cudaFree(p->angles);
  cudaFree(p->layer_base);
  cudaFree(p->mats);
  cudaFree(p->cjobs);
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
  p->angle_cap = (size_t)batch_max * n_noise_ops(n, depth_max) * 3;  // pairs or triples
  const bool ok = cudaMalloc(&p->psi, amp * p->N * batch_max) == cudaSuccess &&
                  cudaMalloc(&p->U, sizeof(double) * 8 * (size_t)n * depth_max) == cudaSuccess &&
                  cudaMalloc(&p->angles, sizeof(double) * p->angle_cap) == cudaSuccess &&
                  cudaMalloc(&p->layer_base, sizeof(int) * (size_t)depth_max) == cudaSuccess &&
                  cudaMalloc(&p->mats, (dtype == IQS_C128 ? sizeof(P128::Mat) : sizeof(P64::Mat)) * (size_t)batch_max *
                                           (size_t)(depth_max + 1) * (size_t)n) == cudaSuccess &&
                  cudaMalloc(&p->cjobs, sizeof(iqs::pool::ClusterJob) * (size_t)batch_max) == cudaSuccess &&
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
  // index of each layer's first noise rotation: depends on n and the layer only, so it is built once
  std::vector<int> base(depth_max);
  for (int l = 0, k = 0; l < depth_max; ++l) {
    base[l] = k;
    k += n + 2 * ((n - (l & 1)) / 2);
  }
  if (e == cudaSuccess)
    e = cudaMemcpy(p->layer_base, base.data(), sizeof(int) * (size_t)depth_max, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    free_pool(p);
    return report(IQS_ECUDA, "pool set-up: %s", cudaGetErrorString(e));
  }
  // choices persisted by iqs_pool_autotune: lines "pool <dtype> <n> <batch_max> <engine> <logc>"
  if (const char* path = std::getenv("IQS_AUTOTUNE_CACHE")) {
    if (FILE* f = std::fopen(path, "r")) {
      char line[256];
      while (std::fgets(line, sizeof(line), f)) {
        char kind[16], dt[8];
        int cn, cb, ce, cl;
        if (std::sscanf(line, "%15s %7s %d %d %d %d", kind, dt, &cn, &cb, &ce, &cl) == 6 &&
            std::strcmp(kind, "pool") == 0 && std::strcmp(dt, dtype == IQS_C128 ? "c128" : "c64") == 0 &&
            cn == n && cb == batch_max && ce >= 0 && ce <= 2 && (ce != 2 || pool_cluster_logc_ok(n, dtype, cl))) {
          p->engine = ce;  // the last matching line wins
          p->logc = cl;
        }
      }
      std::fclose(f);
    }
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

iqs_status iqs_pool_set_noise_t1t2(iqs_pool* p, double T1, double T2, double gate_time) {
  using namespace iqs;
  if (p == nullptr) return report(IQS_EINVAL, "handle is NULL");
  drop_graphs(p);  // captured runs embed the noise law
  if (T1 <= 0.0) {  // back to explicit angle pairs
    p->noise_model = 0;
    return IQS_OK;
  }
  if (!(T2 > 0.0) || T2 > 2.0 * T1 || !(gate_time >= 0.0) || !std::isfinite(T1) || !std::isfinite(gate_time))
    return report(IQS_EINVAL, "need T1 > 0, 0 < T2 <= 2 T1 and a finite gate time >= 0");
  // Bloch factors of the averaged gate: transverse exp(-t/T2), longitudinal
  // exp(-t/T1); the rotation variances that give them (see the header)
  const double vx = gate_time / T1, vz = 2.0 * gate_time / T2 - gate_time / T1;
  p->sig[0] = std::sqrt(vx);
  p->sig[1] = std::sqrt(vx);
  p->sig[2] = std::sqrt(vz > 0.0 ? vz : 0.0);
  p->noise_model = 1;
  return IQS_OK;
}

iqs_status iqs_pool_set_engine(iqs_pool* p, int engine) {
  using namespace iqs;
  if (p == nullptr) return report(IQS_EINVAL, "handle is NULL");
  if (engine < 0 || engine > 2) return report(IQS_EINVAL, "engine must be 0 (auto), 1 (tiled passes) or 2 (cluster)");
  if (engine == 2 && !pool_cluster_eligible(p->n, p->dtype))
    return report(IQS_EINVAL, "a %d-qubit state of this dtype does not fit a cluster's shared memory", p->n);
  p->engine = engine;
  return IQS_OK;
}

iqs_status iqs_pool_run_brick(iqs_pool* p, int batch, int depth, const double* unitaries, const double* angles,
                              double* probs, double* mean) {
  using namespace iqs;
  if (p == nullptr) return report(IQS_EINVAL, "handle is NULL");
  if (batch < 1 || batch > p->bmax) return report(IQS_EINVAL, "batch %d outside [1, %d]", batch, p->bmax);
  if (depth < 1 || depth > p->depth_max) return report(IQS_EINVAL, "depth %d outside [1, %d]", depth, p->depth_max);
  if (unitaries == nullptr || mean == nullptr) return report(IQS_EINVAL, "unitaries and mean must not be NULL");
  if (fault_now(2)) return report(IQS_ECUDA, "iqs_pool_run_brick: injected launch failure");
  const int nn = n_noise_ops(p->n, depth);
  cudaStream_t s = p->stream;
  cudaError_t e = cudaMemcpyAsync(p->U, unitaries, sizeof(double) * 8 * (size_t)p->n * depth, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && angles)
    e = cudaMemcpyAsync(p->angles, angles, sizeof(double) * (p->noise_model == 1 ? 3 : 2) * (size_t)nn * batch,
                        cudaMemcpyHostToDevice, s);
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

iqs_status iqs_pool_run_brick_async(iqs_pool* p, int batch, int depth, const double* d_unitaries,
                                    const double* d_angles, double* d_probs, double* d_mean) {
  using namespace iqs;
  if (p == nullptr) return report(IQS_EINVAL, "handle is NULL");
  if (batch < 1 || batch > p->bmax) return report(IQS_EINVAL, "batch %d outside [1, %d]", batch, p->bmax);
  if (depth < 1 || depth > p->depth_max) return report(IQS_EINVAL, "depth %d outside [1, %d]", depth, p->depth_max);
  if (d_unitaries == nullptr || d_mean == nullptr) return report(IQS_EINVAL, "unitaries and mean must not be NULL");
  if (fault_now(2)) return report(IQS_ECUDA, "iqs_pool_run_brick_async: injected launch failure");
  const int nn = n_noise_ops(p->n, depth);
  cudaStream_t s = p->stream;
  cudaError_t e = cudaMemcpyAsync(p->U, d_unitaries, sizeof(double) * 8 * (size_t)p->n * depth,
                                  cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && d_angles)
    e = cudaMemcpyAsync(p->angles, d_angles, sizeof(double) * (p->noise_model == 1 ? 3 : 2) * (size_t)nn * batch,
                        cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess)
    e = p->dtype == IQS_C128 ? run_pool<P128>(p, batch, depth, d_angles != nullptr)
                             : run_pool<P64>(p, batch, depth, d_angles != nullptr);
  if (e == cudaSuccess && d_probs)
    e = cudaMemcpyAsync(d_probs, p->probs, sizeof(double) * (size_t)p->n * batch, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_mean, p->mean, sizeof(double) * p->n, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return report(IQS_ECUDA, "pool asynchronous launch: %s", cudaGetErrorString(e));
  return IQS_OK;
}

iqs_status iqs_pool_synchronize(iqs_pool* p) {
  using namespace iqs;
  if (p == nullptr) return report(IQS_EINVAL, "handle is NULL");
  unsigned f = 0;
  cudaError_t e = cudaStreamSynchronize(p->stream);
  if (e == cudaSuccess) e = cudaMemcpy(&f, p->flag, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return report(IQS_ECUDA, "pool synchronize: %s", cudaGetErrorString(e));
  if (f) {
    cudaMemset(p->flag, 0, sizeof(unsigned));
    return report(IQS_ERANGE, "an amplitude outside the emulated-FP64 range was met");
  }
  return IQS_OK;
}

iqs_status iqs_pool_autotune(iqs_pool* p, int batch, int depth, int noisy, double* best_ms) {
  using namespace iqs;
  if (p == nullptr) return report(IQS_EINVAL, "handle is NULL");
  if (batch < 1 || batch > p->bmax || depth < 1 || depth > p->depth_max)
    return report(IQS_EINVAL, "batch %d or depth %d outside the pool's limits", batch, depth);
  // timing inputs: rotations with varied angles and small noise angles (the speed does not depend on them)
  std::vector<double> U((size_t)8 * p->n * depth);
  for (size_t g = 0; g < (size_t)p->n * depth; ++g) {
    const double a = 0.37 * (double)(g % 97) + 0.1, c = std::cos(a), s = std::sin(a);
    const double u[8] = {c, 0.0, -s * 0.6, -s * 0.8, s * 0.6, -s * 0.8, c, 0.0};
    std::memcpy(&U[8 * g], u, sizeof(u));
  }
  const int width = p->noise_model == 1 ? 3 : 2;
  std::vector<double> ang(noisy ? (size_t)batch * n_noise_ops(p->n, depth) * width : 0);
  for (size_t i = 0; i < ang.size(); ++i) ang[i] = 0.02 * std::sin(0.7 * (double)i);
  std::vector<double> mean(p->n);
  const int engine0 = p->engine, logc0 = p->logc;
  struct Cand { int engine, logc; };
  std::vector<Cand> cands{{1, -1}};
  for (int lc = 0; lc <= 4; ++lc)
    if (pool_cluster_logc_ok(p->n, p->dtype, lc)) cands.push_back({2, lc});
  double best = 1e300;
  Cand pick{engine0, logc0};
  for (const Cand& c : cands) {
    p->engine = c.engine;
    p->logc = c.logc;
    iqs_status st = iqs_pool_run_brick(p, batch, depth, U.data(), noisy ? ang.data() : nullptr, nullptr, mean.data());
    if (st != IQS_OK) {  // a cluster size that cannot be scheduled here is skipped
      if (c.engine == 1) return st;
      continue;
    }
    double t = 1e300;
    for (int rep = 0; rep < 3; ++rep) {
      const auto t0 = std::chrono::steady_clock::now();
      st = iqs_pool_run_brick(p, batch, depth, U.data(), noisy ? ang.data() : nullptr, nullptr, mean.data());
      const double dt = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      if (st != IQS_OK) return st;
      t = std::min(t, dt);
    }
    if (t < best) {
      best = t;
      pick = c;
    }
  }
  p->engine = pick.engine;
  p->logc = pick.logc;
  if (const char* path = std::getenv("IQS_AUTOTUNE_CACHE")) {
    if (FILE* f = std::fopen(path, "a")) {
      std::fprintf(f, "pool %s %d %d %d %d\n", p->dtype == IQS_C128 ? "c128" : "c64", p->n, p->bmax, p->engine,
                   p->logc);
      std::fclose(f);
    }
  }
  if (best_ms) *best_ms = best;
  return IQS_OK;
}

iqs_status iqs_pool_tuning(const iqs_pool* p, int* engine, int* logc) {
  if (p == nullptr) return iqs::report(IQS_EINVAL, "handle is NULL");
  if (engine) *engine = p->engine;
  if (logc) *logc = p->logc;
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
