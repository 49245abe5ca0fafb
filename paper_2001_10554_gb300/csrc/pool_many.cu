// One persistent launch for a pool of brick circuits of uneven qubit counts,
// depths and trajectory counts (Section 2, "Pool of multiple states": many
// circuits and their stochastic-noise ensembles simulated side by side; pool
// appendix: per-circuit incoherent average over the pool).
//
// Work items are (step, job, tile): a job is one trajectory of one circuit;
// step s = layer * P_max + pass (one tiled pass of the job's state), plus a
// final probability step.  Tickets are handed out by one global atomic
// counter in step-major order, so an item only ever depends on items with
// smaller tickets: every job keeps a counter of its completed tiles, and the
// CTA holding an item waits until its job has finished all tiles of the
// previous step.  Claimed items are always being processed by running CTAs,
// so progress needs no co-residency guarantee.  Every wait is bounded by the
// GPU global timer: on expiry the CTA records IQS_ETIMEOUT, raises an abort
// flag that makes all CTAs leave, and the host reports the status.
//
// Jobs are grouped by qubit count (one tile geometry per group) and, inside a
// group, sorted by decreasing depth, so the jobs still alive at a step form a
// prefix of the group and the ticket -> item decode is arithmetic.
//
// When every state fits a thread-block cluster (pool_cluster.cu), the same
// job list instead runs on the cluster-resident engine: one compose launch
// builds all fused matrices and one cluster launch runs every trajectory of
// every circuit to its end, each state resident on chip.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "pool_common.cuh"
#include "pool_many_ws.h"

namespace iqs {

// pool_cluster.cu
int pool_cluster_logc(int n, int dtype);
cudaError_t launch_pool_cluster(const pool::ClusterJob* jobs, int n_jobs, int max_n, int dtype, cudaStream_t s,
                                int logc);

namespace {

using namespace iqs::pool;

constexpr int kMaxGroups = 8;
constexpr int kMaxPasses = 4;

struct Job {
  uint64_t state_off;      // first amplitude in the arena
  void* mats;              // [phases][n] fused matrices (the dtype's Mat format), built by k_many_compose
  const double* U;         // [depth][n][8] on the device
  const double* ang;       // this trajectory's [n_noise][2] or nullptr
  const int* layer_base;   // [depth]
  uint64_t part_off;       // first slot of this job's probability partials
  int n, depth, phases, n_noise;
  int group, out_index;    // position of the job in the caller's order
};

struct PassInfo {
  Geo g;
  int q_lo, q_hi, lb0;
  unsigned cmask[2];       // CNOT controls (local bits) for even / odd layers
  uint32_t tiles, prefix;  // tiles of this pass; tiles of the passes before it in a layer
};

struct Group {
  int n, passes, prob_bits;  // prob_bits: tile bits of the probability step
  uint32_t tiles_per_layer, prob_tiles;
  int job_start, job_count;
  PassInfo pass[kMaxPasses];
};

struct Plan {
  int G, P, steps;           // groups, max passes per layer, steps including the probability step
  Group grp[kMaxGroups];
};

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// step_start[s] (s = 0..steps) and, per (s, g), grp_start and alive counts.
struct StepTables {
  const uint64_t* step_start;  // [steps + 1]
  const uint64_t* grp_start;   // [steps][G]
  const int* alive;            // [steps][G]
};

template <class TR>
__global__ void __launch_bounds__(kThreads) k_pool_persistent(typename TR::V* __restrict__ arena,
                                                              const Job* __restrict__ jobs, const Plan plan,
                                                              StepTables tab, unsigned* __restrict__ done,
                                                              unsigned long long* __restrict__ ticket,
                                                              double* __restrict__ partials, unsigned* status,
                                                              unsigned* abort_flag, unsigned* flag,
                                                              uint64_t timeout_ns, int debug_never) {
  using W = typename TR::W;
  using Mat = typename TR::Mat;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Mat mats[16];
  __shared__ unsigned long long s_ticket;
  __shared__ int s_quit;
  W* sp = reinterpret_cast<W*>(smem_raw);
  const uint64_t total = tab.step_start[plan.steps];
  unsigned bad = 0;
  for (;;) {
    if (threadIdx.x == 0) {
      s_quit = *(volatile unsigned*)abort_flag ? 1 : 0;
      s_ticket = s_quit ? 0ull : atomicAdd(ticket, 1ull);
    }
    __syncthreads();
    const unsigned long long T = s_ticket;
    if (s_quit || T >= total) break;
    // ---- decode the ticket
    int lo = 0, hi = plan.steps;  // step_start[lo] <= T < step_start[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (tab.step_start[mid] <= T) lo = mid; else hi = mid;
    }
    const int s = lo;
    int g = 0;
    uint64_t r = 0;
    uint32_t tiles = 1;
    for (g = 0; g < plan.G; ++g) {
      const bool prob = s == plan.steps - 1;
      const int p = s % plan.P;
      const Group& gr = plan.grp[g];
      tiles = prob ? gr.prob_tiles : (p < gr.passes ? gr.pass[p].tiles : 0u);
      const uint64_t cnt = (uint64_t)tab.alive[s * plan.G + g] * tiles;
      const uint64_t st = tab.grp_start[s * plan.G + g];
      if (T < st + cnt) {
        r = T - st;
        break;
      }
    }
    if (g >= plan.G || tiles == 0) {  // inconsistent tables: stop everything, report
      if (threadIdx.x == 0) {
        atomicCAS(status, 0u, (unsigned)IQS_EINTERNAL);
        atomicExch(abort_flag, 1u);
      }
      break;
    }
    const Group& gr = plan.grp[g];
    const int jid = gr.job_start + (int)(r / tiles);
    const uint64_t t = r % tiles;
    const Job& job = jobs[jid];
    const bool prob = s == plan.steps - 1;
    const int layer = prob ? job.phases : s / plan.P;
    const int p = prob ? 0 : s % plan.P;
    const uint32_t need = (jid == 0 && debug_never && s == 0)
                              ? 0xffffffffu
                              : (uint32_t)layer * gr.tiles_per_layer + (prob ? 0u : gr.pass[p].prefix);
    // ---- wait for the job's previous step (bounded)
    if (threadIdx.x == 0) {
      const uint64_t t0 = gtimer();
      for (;;) {
        if (ld_acquire(done + jid) >= need) break;
        if (*(volatile unsigned*)abort_flag) { s_quit = 1; break; }
        if (gtimer() - t0 > timeout_ns) {
          atomicCAS(status, 0u, (unsigned)IQS_ETIMEOUT);
          atomicExch(abort_flag, 1u);
          s_quit = 1;
          break;
        }
        __nanosleep(256);
      }
    }
    __syncthreads();
    if (s_quit) break;
    typename TR::V* P = arena + job.state_off;
    if (!prob) {
      const PassInfo& pi = gr.pass[p];
      const int ng = pi.q_hi - pi.q_lo;
      if ((int)threadIdx.x < ng)
        mats[threadIdx.x] = static_cast<const Mat*>(job.mats)[(uint64_t)layer * job.n + pi.q_lo + threadIdx.x];
      __syncthreads();
      const unsigned cm = layer < job.depth ? pi.cmask[layer & 1] : 0u;
      pool_tile<TR>(sp, mats, P, pi.g, t, pi.lb0, ng, cm, bad);
    } else {
      // probability step: tile t = 2^prob_bits contiguous amplitudes
      const unsigned TT = 1u << gr.prob_bits;
      dfx::Acc acc[kPoolMaxQubits + 1];
      const typename TR::V* Q = P + t * TT;
      for (unsigned l = threadIdx.x; l < TT; l += blockDim.x) {
        float pp, ee;
        TR::abs2(TR::load(__ldcg(Q + l), bad), pp, ee);
        const uint64_t x = t * TT + l;
        acc[kPoolMaxQubits].add(pp, ee);
#pragma unroll
        for (int q = 0; q < kPoolMaxQubits; ++q)
          if (q < job.n && ((x >> q) & 1)) acc[q].add(pp, ee);
      }
      double* out = partials + job.part_off + t * (uint64_t)(job.n + 1);
      for (int q = 0; q < job.n; ++q) block_partial(acc[q].value(), out + q);
      block_partial(acc[kPoolMaxQubits].value(), out + job.n);
    }
    // ---- publish: all of this item's writes happen before the counter moves
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(done + jid, 1u);
    }
  }
  if (bad) atomicOr(flag, 1u);
}

// Fused matrices of every job, composed once in FP64 before the simulation
// launch (job j's [phases][n] matrices at job.mats); blockIdx.y strides over jobs.
template <class TR>
__global__ void k_many_compose(const Job* __restrict__ jobs, int njobs) {
  for (int j = blockIdx.y; j < njobs; j += gridDim.y) {
    const Job job = jobs[j];
    const Circuit C{job.n, job.depth, job.U, job.ang, job.layer_base, job.n_noise};
    typename TR::Mat* m = static_cast<typename TR::Mat*>(job.mats);
    const int total = job.phases * job.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x)
      m[i] = TR::make(compose_traj(C, job.ang, i / job.n, i % job.n));
  }
}

// |0...0> for every job (the arena is zeroed first).
template <class V>
__global__ void k_many_init(V* arena, const Job* __restrict__ jobs, int njobs) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < njobs; j += gridDim.x * blockDim.x) {
    V v;
    v.x = 1;
    v.y = 0;
    arena[jobs[j].state_off] = v;
  }
}

// probs[out][q] = sum over tiles / norm for every job; one block per job.
__global__ void k_many_finish(const Job* __restrict__ jobs, const double* __restrict__ partials, const Plan plan,
                              const uint64_t* __restrict__ out_off, double* __restrict__ probs) {
  const Job& job = jobs[blockIdx.x];
  const uint32_t tiles = plan.grp[job.group].prob_tiles;
  __shared__ double vals[kPoolMaxQubits + 1];
  for (int q = threadIdx.x; q <= job.n; q += blockDim.x) {
    double s = 0.0;
    for (uint32_t t = 0; t < tiles; ++t) s += partials[job.part_off + (uint64_t)t * (job.n + 1) + q];
    vals[q] = s;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < job.n; q += blockDim.x) probs[out_off[job.out_index] + q] = vals[q] / vals[job.n];
}

// means[c][q] = sum over the circuit's trajectories / their number; one block per circuit.
__global__ void k_many_means(const double* __restrict__ probs, const uint64_t* __restrict__ circ_first,
                             const int* __restrict__ circ_traj, const int* __restrict__ circ_n,
                             const uint64_t* __restrict__ mean_off, double* __restrict__ means) {
  const int c = blockIdx.x;
  const int n = circ_n[c], T = circ_traj[c];
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < T; ++b) s += probs[circ_first[c] + (uint64_t)b * n + q];
    means[mean_off[c] + q] = s / T;
  }
}

}  // namespace
}  // namespace iqs

// ================================================================ host workspace: pool_many_ws.h

namespace iqs {
namespace {

struct HostPass {
  Geo g;
  int q_lo, q_hi, cut_lo, cut_hi;
};

std::vector<HostPass> plan_passes(int n, int K, int rows) {
  std::vector<HostPass> out;
  const int KA = std::min(n, K);
  out.push_back(HostPass{Geo{0, 0, KA}, 0, KA, 0, KA});
  int start = KA;
  while (start < n) {
    const int end = std::min(n, start - 1 + (K - rows));
    const int s = start - 1, m = end - s;
    out.push_back(HostPass{Geo{K - m, s, m}, start, end, s, end});
    start = end;
  }
  return out;
}

unsigned pass_cmask(const HostPass& p, int n, int parity) {
  const bool low = p.g.c == 0 && p.g.s == 0;
  unsigned mask = 0;
  for (int i = parity; i + 1 < n; i += 2)
    if (i >= p.cut_lo && i + 1 < p.cut_hi && i + 1 >= (low ? 0 : p.q_lo)) mask |= 1u << (low ? i : i - p.g.s + p.g.c);
  return mask;
}

int noise_ops(int n, int depth) {
  int k = 0;
  for (int l = 0; l < depth; ++l) k += n + 2 * ((n - (l & 1)) / 2);
  return k;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

template <class TR>
iqs_status run_many(iqs_pool_many* W, int nc, const iqs_circuit_desc* cd, double* probs_out, double* means_out);

}  // namespace
}  // namespace iqs

extern "C" {

iqs_status iqs_pool_many_create(int dtype, void* stream, iqs_pool_many** out) {
  using namespace iqs;
  if (out == nullptr) return report(IQS_EINVAL, "out is NULL");
  *out = nullptr;
  if (dtype != IQS_C64 && dtype != IQS_C128) return report(IQS_EINVAL, "dtype must be IQS_C64 or IQS_C128");
  iqs_pool_many* w = new (std::nothrow) iqs_pool_many();
  if (w == nullptr) return report(IQS_ENOMEM, "host allocation failed");
  w->dtype = dtype;
  w->stream = (cudaStream_t)stream;
  if (w->stream == nullptr) {
    if (cudaStreamCreate(&w->stream) != cudaSuccess) {
      cudaGetLastError();
      delete w;
      return report(IQS_ECUDA, "cannot create a stream");
    }
    w->own_stream = true;
  }
  *out = w;
  return IQS_OK;
}

iqs_status iqs_pool_many_destroy(iqs_pool_many* w) {
  if (w == nullptr) return IQS_OK;
  cudaStreamSynchronize(w->stream);
  cudaFree(w->arena);
  cudaFree(w->blob);
  cudaFree(w->mats);
  cudaFree(w->ops_buf);
  if (w->own_stream) cudaStreamDestroy(w->stream);
  delete w;
  return IQS_OK;
}

iqs_status iqs_pool_many_set_wait_limit(iqs_pool_many* w, double seconds, int debug_never) {
  if (w == nullptr) return iqs::report(IQS_EINVAL, "handle is NULL");
  if (!(seconds > 0.0) || seconds > 600.0) return iqs::report(IQS_EINVAL, "wait limit must be in (0, 600] s");
  w->timeout_ns = (uint64_t)(seconds * 1e9);
  w->debug_never = debug_never ? 1 : 0;
  return IQS_OK;
}

iqs_status iqs_pool_many_set_engine(iqs_pool_many* w, int engine) {
  if (w == nullptr) return iqs::report(IQS_EINVAL, "handle is NULL");
  if (engine < 0 || engine > 2) return iqs::report(IQS_EINVAL, "engine must be 0 (auto), 1 (persistent) or 2 (cluster)");
  w->engine = engine;
  return IQS_OK;
}

iqs_status iqs_pool_many_run(iqs_pool_many* w, int n_circuits, const iqs_circuit_desc* circuits, double* probs,
                             double* means) {
  using namespace iqs;
  if (w == nullptr || circuits == nullptr || means == nullptr) return report(IQS_EINVAL, "NULL argument");
  if (n_circuits < 1 || n_circuits > 100000) return report(IQS_EINVAL, "n_circuits %d outside [1, 100000]", n_circuits);
  for (int c = 0; c < n_circuits; ++c) {
    const iqs_circuit_desc& d = circuits[c];
    if (d.n < 2 || d.n > kPoolMaxQubits || d.depth < 1 || d.depth > 100000 || d.trajectories < 1 ||
        d.unitaries == nullptr)
      return report(IQS_EINVAL, "circuit %d: n %d (2..%d), depth %d, trajectories %d or unitaries invalid", c, d.n,
                    kPoolMaxQubits, d.depth, d.trajectories);
    if (d.angles == nullptr && d.trajectories != 1)
      return report(IQS_EINVAL, "circuit %d: a noiseless circuit has exactly one trajectory", c);
  }
  if (fault_now(2)) return report(IQS_ECUDA, "iqs_pool_many_run: injected launch failure");
  return w->dtype == IQS_C128 ? run_many<pool::P128>(w, n_circuits, circuits, probs, means)
                              : run_many<pool::P64>(w, n_circuits, circuits, probs, means);
}

}  // extern "C"

namespace iqs {
namespace {

template <class TR>
iqs_status run_many(iqs_pool_many* W, int nc, const iqs_circuit_desc* cd, double* probs_out, double* means_out) {
  using V = typename TR::V;
  const int K = TR::kTileBits, rows = TR::kRowBits;
  // ---- groups by qubit count
  std::vector<int> ns;
  for (int c = 0; c < nc; ++c) ns.push_back(cd[c].n);
  std::sort(ns.begin(), ns.end());
  ns.erase(std::unique(ns.begin(), ns.end()), ns.end());
  if ((int)ns.size() > kMaxGroups) return report(IQS_EINVAL, "at most %d distinct qubit counts per call", kMaxGroups);
  Plan plan{};
  plan.G = (int)ns.size();
  plan.P = 1;
  std::vector<std::vector<HostPass>> hp(plan.G);
  for (int g = 0; g < plan.G; ++g) {
    hp[g] = plan_passes(ns[g], K, rows);
    if ((int)hp[g].size() > kMaxPasses) return report(IQS_EINVAL, "too many passes for %d qubits", ns[g]);
    plan.P = std::max(plan.P, (int)hp[g].size());
  }
  // ---- jobs: per group, sorted by decreasing phase count
  struct HJob {
    int c, b, phases;
  };
  std::vector<std::vector<HJob>> gj(plan.G);
  int max_phases = 0;
  for (int c = 0; c < nc; ++c) {
    const int g = (int)(std::lower_bound(ns.begin(), ns.end(), cd[c].n) - ns.begin());
    const int ph = cd[c].depth + (cd[c].angles ? 1 : 0);
    max_phases = std::max(max_phases, ph);
    for (int b = 0; b < cd[c].trajectories; ++b) gj[g].push_back(HJob{c, b, ph});
  }
  for (auto& v : gj)
    std::stable_sort(v.begin(), v.end(), [](const HJob& a, const HJob& b) { return a.phases > b.phases; });
  plan.steps = max_phases * plan.P + 1;
  // ---- layout of the device blob
  std::vector<uint64_t> circ_first(nc), mean_off(nc);
  std::vector<int> circ_traj(nc), circ_n(nc);
  uint64_t nprob = 0, nmean = 0;
  size_t u_doubles = 0, a_doubles = 0, lb_ints = 0;
  std::vector<size_t> u_off(nc), a_off(nc), lb_off(nc);
  for (int c = 0; c < nc; ++c) {
    circ_first[c] = nprob;
    mean_off[c] = nmean;
    circ_traj[c] = cd[c].trajectories;
    circ_n[c] = cd[c].n;
    nprob += (uint64_t)cd[c].trajectories * cd[c].n;
    nmean += cd[c].n;
    u_off[c] = u_doubles;
    u_doubles += (size_t)cd[c].depth * cd[c].n * 8;
    a_off[c] = a_doubles;
    if (cd[c].angles) a_doubles += (size_t)cd[c].trajectories * noise_ops(cd[c].n, cd[c].depth) * 2;
    lb_off[c] = lb_ints;
    lb_ints += cd[c].depth;
  }
  size_t njobs = 0;
  for (auto& v : gj) njobs += v.size();
  std::vector<uint64_t> out_off(njobs);
  // arena and partials
  uint64_t arena_amps = 0, parts = 0;
  std::vector<Job> jobs;
  jobs.reserve(njobs);
  std::vector<size_t> job_u, job_lb;
  std::vector<int64_t> job_a;  // -1: noiseless
  // caller order index: circuits in order, trajectories in order
  std::vector<uint64_t> caller_first(nc);
  {
    uint64_t k = 0;
    for (int c = 0; c < nc; ++c) {
      caller_first[c] = k;
      k += cd[c].trajectories;
    }
  }
  for (int g = 0; g < plan.G; ++g) {
    Group& gr = plan.grp[g];
    gr.n = ns[g];
    gr.passes = (int)hp[g].size();
    gr.job_start = (int)jobs.size();
    gr.job_count = (int)gj[g].size();
    const uint64_t N = 1ull << gr.n;
    uint32_t pre = 0;
    for (int p = 0; p < gr.passes; ++p) {
      const HostPass& h = hp[g][p];
      PassInfo& pi = gr.pass[p];
      pi.g = h.g;
      pi.q_lo = h.q_lo;
      pi.q_hi = h.q_hi;
      pi.lb0 = (h.g.c == 0 && h.g.s == 0) ? h.q_lo : h.q_lo - h.g.s + h.g.c;
      pi.cmask[0] = pass_cmask(h, gr.n, 0);
      pi.cmask[1] = pass_cmask(h, gr.n, 1);
      pi.tiles = (uint32_t)(N >> (h.g.c + h.g.m));
      pi.prefix = pre;
      pre += pi.tiles;
    }
    gr.tiles_per_layer = pre;
    gr.prob_bits = std::min(gr.n, K);
    gr.prob_tiles = (uint32_t)(N >> gr.prob_bits);
    for (const HJob& hj : gj[g]) {
      const iqs_circuit_desc& d = cd[hj.c];
      Job j{};
      j.state_off = arena_amps;
      arena_amps += N;
      j.n = d.n;
      j.depth = d.depth;
      j.phases = hj.phases;
      j.n_noise = noise_ops(d.n, d.depth);
      j.group = g;
      j.out_index = (int)(caller_first[hj.c] + hj.b);
      out_off[j.out_index] = circ_first[hj.c] + (uint64_t)hj.b * d.n;
      j.part_off = parts;
      parts += (uint64_t)gr.prob_tiles * (d.n + 1);
      // device pointers are set below once the blob address is known
      job_u.push_back(u_off[hj.c]);
      job_a.push_back(d.angles ? (int64_t)(a_off[hj.c] + (size_t)hj.b * j.n_noise * 2) : (int64_t)-1);
      job_lb.push_back(lb_off[hj.c]);
      jobs.push_back(j);
    }
  }
  // ---- step tables
  const int S = plan.steps;
  std::vector<uint64_t> step_start(S + 1), grp_start((size_t)S * plan.G);
  std::vector<int> alive((size_t)S * plan.G);
  uint64_t tk = 0;
  for (int s = 0; s < S; ++s) {
    step_start[s] = tk;
    const bool prob = s == S - 1;
    const int layer = s / plan.P, p = s % plan.P;
    for (int g = 0; g < plan.G; ++g) {
      const Group& gr = plan.grp[g];
      int a = 0;
      uint32_t tiles = 0;
      if (prob) {
        a = gr.job_count;
        tiles = gr.prob_tiles;
      } else if (p < gr.passes) {
        for (const HJob& hj : gj[g]) a += hj.phases > layer ? 1 : 0;
        tiles = gr.pass[p].tiles;
      }
      grp_start[(size_t)s * plan.G + g] = tk;
      alive[(size_t)s * plan.G + g] = a;
      tk += (uint64_t)a * tiles;
    }
  }
  step_start[S] = tk;
  // ---- device memory: arena + blob
  const size_t amp = sizeof(V);
  if (W->arena_bytes < arena_amps * amp) {
    cudaFree(W->arena);
    W->arena = nullptr;
    W->arena_bytes = 0;
    if (cudaMalloc(&W->arena, arena_amps * amp) != cudaSuccess) {
      cudaGetLastError();
      return report(IQS_ENOMEM, "cannot allocate %zu bytes of pool states", (size_t)(arena_amps * amp));
    }
    W->arena_bytes = arena_amps * amp;
  }
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align256(off + bytes);
    return o;
  };
  const size_t o_u = take(u_doubles * 8), o_a = take(a_doubles * 8), o_lb = take(lb_ints * 4);
  const size_t o_jobs = take(njobs * sizeof(Job)), o_done = take(njobs * 4);
  const size_t o_ss = take((S + 1) * 8), o_gs = take(grp_start.size() * 8), o_al = take(alive.size() * 4);
  const size_t o_part = take(parts * 8), o_probs = take(nprob * 8), o_means = take(nmean * 8);
  const size_t o_outoff = take(njobs * 8), o_cf = take(nc * 8), o_ct = take(nc * 4), o_cn = take(nc * 4);
  const size_t o_mo = take(nc * 8), o_ctrl = take(64);
  if (W->blob_bytes < off) {
    cudaFree(W->blob);
    W->blob = nullptr;
    W->blob_bytes = 0;
    if (cudaMalloc(&W->blob, off) != cudaSuccess) {
      cudaGetLastError();
      return report(IQS_ENOMEM, "cannot allocate %zu bytes of pool tables", off);
    }
    W->blob_bytes = off;
  }
  char* B = static_cast<char*>(W->blob);
  // fused matrices of every job: [phases][n] each
  using Mat = typename TR::Mat;
  uint64_t nmat = 0;
  for (const Job& j : jobs) nmat += (uint64_t)j.phases * j.n;
  if (W->mats_bytes < nmat * sizeof(Mat)) {
    cudaFree(W->mats);
    W->mats = nullptr;
    W->mats_bytes = 0;
    if (cudaMalloc(&W->mats, nmat * sizeof(Mat)) != cudaSuccess) {
      cudaGetLastError();
      return report(IQS_ENOMEM, "cannot allocate %zu bytes of fused matrices", (size_t)(nmat * sizeof(Mat)));
    }
    W->mats_bytes = nmat * sizeof(Mat);
  }
  {
    uint64_t mo = 0;
    for (Job& j : jobs) {
      j.mats = static_cast<Mat*>(W->mats) + mo;
      mo += (uint64_t)j.phases * j.n;
    }
  }
  for (size_t i = 0; i < jobs.size(); ++i) {
    jobs[i].U = reinterpret_cast<const double*>(B + o_u) + job_u[i];
    jobs[i].ang = job_a[i] >= 0 ? reinterpret_cast<const double*>(B + o_a) + job_a[i] : nullptr;
    jobs[i].layer_base = reinterpret_cast<const int*>(B + o_lb) + job_lb[i];
  }
  // ---- uploads (from pageable host memory: copied before the call returns)
  cudaStream_t st = W->stream;
  cudaError_t e = cudaSuccess;
  auto up = [&](size_t o, const void* src, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(B + o, src, bytes, cudaMemcpyHostToDevice, st);
  };
  std::vector<int> lbs(lb_ints);
  for (int c = 0; c < nc; ++c) {
    up(o_u + u_off[c] * 8, cd[c].unitaries, (size_t)cd[c].depth * cd[c].n * 64);
    if (cd[c].angles) up(o_a + a_off[c] * 8, cd[c].angles, (size_t)cd[c].trajectories * noise_ops(cd[c].n, cd[c].depth) * 16);
    for (int l = 0, k = 0; l < cd[c].depth; ++l) {
      lbs[lb_off[c] + l] = k;
      k += cd[c].n + 2 * ((cd[c].n - (l & 1)) / 2);
    }
  }
  up(o_lb, lbs.data(), lb_ints * 4);
  up(o_jobs, jobs.data(), njobs * sizeof(Job));
  up(o_ss, step_start.data(), (S + 1) * 8);
  up(o_gs, grp_start.data(), grp_start.size() * 8);
  up(o_al, alive.data(), alive.size() * 4);
  up(o_outoff, out_off.data(), njobs * 8);
  up(o_cf, circ_first.data(), nc * 8);
  up(o_ct, circ_traj.data(), nc * 4);
  up(o_cn, circ_n.data(), nc * 4);
  up(o_mo, mean_off.data(), nc * 8);
  if (e == cudaSuccess) e = cudaMemsetAsync(W->arena, 0, arena_amps * amp, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(B + o_done, 0, njobs * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(B + o_ctrl, 0, 64, st);
  if (e != cudaSuccess) return report(IQS_ECUDA, "pool upload: %s", cudaGetErrorString(e));
  {
    const dim3 cg(8, (unsigned)std::min<size_t>(njobs, 65535));
    k_many_compose<TR><<<cg, kThreads, 0, st>>>(reinterpret_cast<const Job*>(B + o_jobs), (int)njobs);
    e = cudaGetLastError();
    if (e != cudaSuccess) return report(IQS_ECUDA, "compose launch: %s", cudaGetErrorString(e));
    note_launches(1);
  }
  // ---- cluster-resident path: every trajectory in one cluster launch
  int max_n = 0, min_n = 1 << 30;
  for (int c = 0; c < nc; ++c) {
    max_n = std::max(max_n, cd[c].n);
    min_n = std::min(min_n, cd[c].n);
  }
  const int lc = pool_cluster_logc(max_n, W->dtype);
  const bool fits = lc >= 0 && min_n >= 2 * lc + 1;
  if (W->engine == 2 && !fits)
    return report(IQS_EINVAL, "the cluster engine takes these circuits only if every state fits (%d..%d qubits)",
                  min_n, max_n);
  if (W->engine == 2 || (W->engine == 0 && W->dtype == IQS_C64 && fits && lc <= 2)) {
    // the job table: scratch from the stream-ordered allocator
    void* scratch = nullptr;
    const size_t tb = njobs * sizeof(ClusterJob);
    if (cudaMallocAsync(&scratch, tb, st) != cudaSuccess) {
      cudaGetLastError();
      return report(IQS_ENOMEM, "cannot allocate the cluster job table");
    }
    ClusterJob* dcj = static_cast<ClusterJob*>(scratch);
    double* dprobs = reinterpret_cast<double*>(B + o_probs);
    std::vector<ClusterJob> cj(njobs);
    for (size_t j = 0; j < njobs; ++j)
      cj[j] = ClusterJob{jobs[j].mats, static_cast<V*>(W->arena) + jobs[j].state_off,
                         dprobs + out_off[jobs[j].out_index], jobs[j].n, jobs[j].phases, jobs[j].depth};
    e = cudaMemcpyAsync(dcj, cj.data(), njobs * sizeof(ClusterJob), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_pool_cluster(dcj, (int)njobs, max_n, W->dtype, st, -1);
    if (e == cudaSuccess) {
      k_many_means<<<nc, 32, 0, st>>>(dprobs, reinterpret_cast<const uint64_t*>(B + o_cf),
                                      reinterpret_cast<const int*>(B + o_ct), reinterpret_cast<const int*>(B + o_cn),
                                      reinterpret_cast<const uint64_t*>(B + o_mo), reinterpret_cast<double*>(B + o_means));
      e = cudaGetLastError();
    }
    cudaFreeAsync(scratch, st);
    if (e != cudaSuccess) return report(IQS_ECUDA, "cluster pool launch: %s", cudaGetErrorString(e));
    note_launches(1);  // means (compose and the cluster launch are counted where they launch)
    if (probs_out) e = cudaMemcpyAsync(probs_out, dprobs, nprob * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(means_out, B + o_means, nmean * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return report(IQS_ECUDA, "pool results: %s", cudaGetErrorString(e));
    return IQS_OK;
  }
  unsigned long long* ticket = reinterpret_cast<unsigned long long*>(B + o_ctrl);
  unsigned* status = reinterpret_cast<unsigned*>(B + o_ctrl + 8);
  unsigned* abort_flag = reinterpret_cast<unsigned*>(B + o_ctrl + 12);
  unsigned* rflag = reinterpret_cast<unsigned*>(B + o_ctrl + 16);
  // ---- the persistent launch
  const size_t smem = ((size_t)1 << K) * sizeof(typename TR::W);
  e = cudaFuncSetAttribute(k_pool_persistent<TR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pool_persistent<TR>, kThreads, smem);
  int dev = 0, sms = kSMs;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess || per_sm < 1) return report(IQS_ECUDA, "persistent occupancy: %s", cudaGetErrorString(e));
  StepTables tabs{reinterpret_cast<const uint64_t*>(B + o_ss), reinterpret_cast<const uint64_t*>(B + o_gs),
                  reinterpret_cast<const int*>(B + o_al)};
  const Job* djobs = reinterpret_cast<const Job*>(B + o_jobs);
  k_many_init<V><<<(unsigned)((njobs + kThreads - 1) / kThreads), kThreads, 0, st>>>(static_cast<V*>(W->arena), djobs,
                                                                                    (int)njobs);
  k_pool_persistent<TR><<<sms * per_sm, kThreads, smem, st>>>(
      static_cast<V*>(W->arena), djobs, plan, tabs, reinterpret_cast<unsigned*>(B + o_done), ticket,
      reinterpret_cast<double*>(B + o_part), status, abort_flag, rflag, W->timeout_ns, W->debug_never);
  k_many_finish<<<(unsigned)njobs, 32, 0, st>>>(djobs, reinterpret_cast<double*>(B + o_part), plan,
                                                 reinterpret_cast<const uint64_t*>(B + o_outoff),
                                                 reinterpret_cast<double*>(B + o_probs));
  k_many_means<<<nc, 32, 0, st>>>(reinterpret_cast<double*>(B + o_probs), reinterpret_cast<const uint64_t*>(B + o_cf),
                                  reinterpret_cast<const int*>(B + o_ct), reinterpret_cast<const int*>(B + o_cn),
                                  reinterpret_cast<const uint64_t*>(B + o_mo), reinterpret_cast<double*>(B + o_means));
  e = cudaGetLastError();
  if (e != cudaSuccess) return report(IQS_ECUDA, "persistent launch: %s", cudaGetErrorString(e));
  note_launches(4);
  unsigned ctrl[5] = {0, 0, 0, 0, 0};
  e = cudaMemcpyAsync(ctrl, B + o_ctrl, sizeof(ctrl), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && probs_out) e = cudaMemcpyAsync(probs_out, B + o_probs, nprob * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(means_out, B + o_means, nmean * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return report(IQS_ECUDA, "pool results: %s", cudaGetErrorString(e));
  if (ctrl[2] == (unsigned)IQS_ETIMEOUT)
    return report(IQS_ETIMEOUT, "a persistent-kernel wait exceeded %.3f s; the results are incomplete",
                  W->timeout_ns * 1e-9);
  if (ctrl[2] != 0u) return report(IQS_EINTERNAL, "persistent pool kernel: inconsistent work tables");
  if (ctrl[4]) return report(IQS_ERANGE, "an amplitude outside the emulated-FP64 range was met");
  return IQS_OK;
}

}  // namespace
}  // namespace iqs
