// Pools of circuits given as gate lists (Section 2, "Pool of multiple states":
// each pool state runs its own circuit, and stochastic one-qubit rotations
// after the gates give the trajectories of a noisy ensemble; pool appendix:
// per-circuit incoherent averages over the pool).
//
// A circuit is an ordered list of one-qubit gates U on a target and
// controlled one-qubit gates (U on the target of the basis states whose
// control qubit is 1).  With noise, every gate is followed, on each qubit it
// touched (the target; for a controlled gate the control, then the target),
// by RX(tx) then RZ(tz), with angles that differ per trajectory.
//
// Host compilation, once per circuit and shared by its trajectories:
//   - Steps.  A one-qubit gate with the noise after it is one step with a
//     per-trajectory matrix.  A controlled gate is a step with a shared
//     matrix; the noise after it becomes one-qubit steps on its control and
//     target.  Consecutive one-qubit steps on a qubit that nothing touches in
//     between fuse into one (their matrices multiply).
//   - Rounds.  Each step goes, in circuit order, into the latest round at or
//     after the last round that touches its qubits whose window of R target
//     bits holds its target (else into a new round).  One round applies all
//     of its steps to register blocks of 2^R amplitudes in one sweep of the
//     state.  A control is an index bit, so it may lie inside or outside the
//     window.
// Device:
//   - k_ops_compose: the fused per-trajectory step matrices (FP64 products,
//     rounded once into the dtype's matrix form) and the shared
//     controlled-gate matrices;
//   - k_pool_ops: one CTA per trajectory, a grid-stride loop over every
//     trajectory of every circuit (one launch); the state lives in shared
//     memory when it fits (up to 2^14 complex64 or 2^13 complex128 amplitudes),
//     otherwise in an L2-resident slot of a global arena owned by the CTA; the
//     rounds run in order, then P(q = 1) / norm of every qubit is reduced in
//     FP64-equivalent (double-float) arithmetic.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "pool_common.cuh"
#include "pool_many_ws.h"

namespace iqs {
namespace {

using namespace iqs::pool;

constexpr int kOpsRoundSteps = 32;  // step matrices staged in shared memory per round

struct OpsStep {
  int16_t target, control;  // control -1: one-qubit step
  int32_t mat;              // >= 0: per-trajectory matrix slot; < 0: shared matrix -1 - mat
};

struct OpsRound {
  int32_t pos, bits, first, count;  // window [pos, pos + bits) of target bits; steps [first, first + count)
};

struct OpsProg {  // one circuit
  const OpsRound* rounds;
  const OpsStep* steps;
  const void* shared;  // shared controlled-gate matrices (the dtype's Mat)
  int n, n_rounds;
};

struct OpsJob {  // one trajectory
  const void* mats;  // its fused step matrices
  double* probs;     // P(q = 1) / norm, n values
  int prog;
};

struct ComposeJob {    // the matrices of one trajectory (or a circuit's shared matrices when ang == nullptr
  const double* U;     // and shared != 0): [n_ops][8] op matrices of the circuit
  const int* fact_off; // [slots + 1]
  const int* facts;    // >= 0: op index; < 0: noise rotation -1 - f
  const double* ang;   // [n_noise][2] of the trajectory, or nullptr (noiseless)
  void* out;           // [slots] matrices
  int slots;
};

template <class TR>
__global__ void k_ops_compose(const ComposeJob* __restrict__ jobs, int njobs) {
  for (int j = blockIdx.y; j < njobs; j += gridDim.y) {
    const ComposeJob cj = jobs[j];
    typename TR::Mat* out = static_cast<typename TR::Mat*>(cj.out);
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < cj.slots; s += gridDim.x * blockDim.x) {
      M2 m = identity2();
      for (int i = cj.fact_off[s]; i < cj.fact_off[s + 1]; ++i) {
        const int f = cj.facts[i];
        M2 g;
        if (f >= 0) {
          const double* u = cj.U + (uint64_t)f * 8;
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            g.r[e] = u[2 * e];
            g.i[e] = u[2 * e + 1];
          }
        } else {
          const int k = -1 - f;
          g = cj.ang ? noise_rot(cj.ang[2 * k], cj.ang[2 * k + 1]) : identity2();
        }
        m = mmul(g, m);  // the later factor acts after the earlier ones
      }
      out[s] = TR::make(m);
    }
  }
}

// Apply one step matrix along local bit T of a register block of 2^R
// amplitudes, to the pairs whose element index j has bit j of ``cm`` set.
template <class TR, int T, int RB>
__device__ __forceinline__ void apply_bit(typename TR::W* a, const typename TR::Mat& u, uint32_t cm, int nb) {
#pragma unroll
  for (int j = 0; j < RB; ++j)
    if (!(j & (1 << T)) && j < nb && ((cm >> j) & 1u)) TR::apply(u, a[j], a[j | (1 << T)]);
}

template <class TR>
__device__ __forceinline__ void apply_step(typename TR::W* a, const typename TR::Mat& u, int t, uint32_t cm, int nb) {
  constexpr int RB = 1 << TR::kRegBits;
  switch (t) {
    case 0: apply_bit<TR, 0, RB>(a, u, cm, nb); break;
    case 1: apply_bit<TR, 1, RB>(a, u, cm, nb); break;
    case 2: apply_bit<TR, 2, RB>(a, u, cm, nb); break;
    default:
      if constexpr (TR::kRegBits > 3) apply_bit<TR, 3, RB>(a, u, cm, nb);
      break;
  }
}

// Bits j of a register block (j < 16) whose local bit b is set.
__device__ __forceinline__ uint32_t bit_set_mask(int b) {
  return b == 0 ? 0xAAAAu : b == 1 ? 0xCCCCu : b == 2 ? 0xF0F0u : 0xFF00u;
}

// Double-float warp sum (h, l) -> lane 0.
__device__ __forceinline__ void warp_sum_df(float& h, float& l) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, l, o);
    float s, t;
    dfx::two_sum(h, oh, s, t);
    const float lo = l + ol + t;
    h = s + lo;
    l = lo - (h - s);
  }
}

template <class TR>
__global__ void __launch_bounds__(kThreads) k_pool_ops(typename TR::W* __restrict__ arena, uint64_t slot_amps,
                                                       const OpsJob* __restrict__ jobs, int njobs,
                                                       const OpsProg* __restrict__ progs, int smem_max_n,
                                                       unsigned* __restrict__ flag) {
  using V = typename TR::V;
  using W = typename TR::W;
  using Mat = typename TR::Mat;
  constexpr int R = TR::kRegBits;
  constexpr int RB = 1 << R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  W* sstate = reinterpret_cast<W*>(smem_raw);
  __shared__ Mat mats_s[kOpsRoundSteps];
  __shared__ OpsStep steps_s[kOpsRoundSteps];
  __shared__ float red_h[kThreads / 32][kPoolMaxQubits + 1], red_l[kThreads / 32][kPoolMaxQubits + 1];
  const unsigned tid = threadIdx.x;
  unsigned bad = 0;
  V v0, v1;
  v0.x = 0; v0.y = 0;
  v1.x = 1; v1.y = 0;
  const W zero = TR::load(v0, bad), one = TR::load(v1, bad);
  for (int jb = blockIdx.x; jb < njobs; jb += gridDim.x) {
    const OpsJob job = jobs[jb];
    const OpsProg P = progs[job.prog];
    const int n = P.n;
    const uint32_t N = 1u << n;
    W* st = n <= smem_max_n ? sstate : arena + (uint64_t)blockIdx.x * slot_amps;
    for (uint32_t i = tid; i < N; i += kThreads) st[swz<TR>(i)] = i == 0 ? one : zero;  // |0...0>
    __syncthreads();
    for (int r = 0; r < P.n_rounds; ++r) {
      const OpsRound rd = P.rounds[r];
      for (int k = tid; k < rd.count; k += kThreads) {
        const OpsStep sp = P.steps[rd.first + k];
        steps_s[k] = sp;
        mats_s[k] = sp.mat >= 0 ? static_cast<const Mat*>(job.mats)[sp.mat]
                                : static_cast<const Mat*>(P.shared)[-1 - sp.mat];
      }
      __syncthreads();
      const int nb = 1 << rd.bits;
      const uint32_t all = (1u << nb) - 1u;
      const uint32_t nblk = N >> rd.bits;
      for (uint32_t blk = tid; blk < nblk; blk += kThreads) {
        const uint32_t base = ((blk >> rd.pos) << (rd.pos + rd.bits)) | (blk & ((1u << rd.pos) - 1u));
        W a[RB];
#pragma unroll
        for (int j = 0; j < RB; ++j)
          if (j < nb) a[j] = st[swz<TR>(base | ((uint32_t)j << rd.pos))];
        for (int k = 0; k < rd.count; ++k) {
          const OpsStep sp = steps_s[k];
          uint32_t cm = all;
          if (sp.control >= 0) {
            const int cl = sp.control - rd.pos;
            if (cl >= 0 && cl < rd.bits) cm = bit_set_mask(cl) & all;
            else cm = ((base >> sp.control) & 1u) ? all : 0u;
          }
          if (cm) apply_step<TR>(a, mats_s[k], sp.target - rd.pos, cm, nb);
        }
#pragma unroll
        for (int j = 0; j < RB; ++j)
          if (j < nb) st[swz<TR>(base | ((uint32_t)j << rd.pos))] = a[j];
      }
      __syncthreads();
    }
    // P(q = 1) and the squared norm, double-float per thread, then over the block
    dfx::Acc acc[kPoolMaxQubits + 1];
    for (uint32_t i = tid; i < N; i += kThreads) {
      float p, e;
      TR::abs2(st[swz<TR>(i)], p, e);
      acc[kPoolMaxQubits].add(p, e);
#pragma unroll
      for (int q = 0; q < kPoolMaxQubits; ++q)
        if (q < n && ((i >> q) & 1u)) acc[q].add(p, e);
    }
#pragma unroll
    for (int q = 0; q <= kPoolMaxQubits; ++q) {
      float h = acc[q].h, l = acc[q].l;
      warp_sum_df(h, l);
      if ((tid & 31) == 0) {
        red_h[tid >> 5][q] = h;
        red_l[tid >> 5][q] = l;
      }
    }
    __syncthreads();
    if (tid <= (unsigned)kPoolMaxQubits) {
      dfx::Acc s;
      for (int w = 0; w < kThreads / 32; ++w) s.add(red_h[w][tid], red_l[w][tid]);
      red_h[0][tid] = s.h;  // row 0 is read back only below, after the barrier
      red_l[0][tid] = s.l;
    }
    __syncthreads();
    if (tid < (unsigned)n) {
      const double norm = (double)red_h[0][kPoolMaxQubits] + (double)red_l[0][kPoolMaxQubits];
      job.probs[tid] = ((double)red_h[0][tid] + (double)red_l[0][tid]) / norm;
    }
    __syncthreads();  // the next job reuses the state and the reduction buffers
  }
  if (bad) atomicOr(flag, 1u);
}

// means[c][q] = sum over the circuit's trajectories / their number; one block per circuit.
__global__ void k_ops_means(const double* __restrict__ probs, const uint64_t* __restrict__ first,
                            const int* __restrict__ traj, const int* __restrict__ nq, const uint64_t* __restrict__ moff,
                            double* __restrict__ means) {
  const int c = blockIdx.x;
  for (int q = threadIdx.x; q < nq[c]; q += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < traj[c]; ++b) s += probs[first[c] + (uint64_t)b * nq[c] + q];
    means[moff[c] + q] = s / traj[c];
  }
}

// ---------------------------------------------------------------- host compilation
struct HStep {
  int target, control;      // control -1: one-qubit step
  int slot;                 // per-trajectory slot (one-qubit) or shared index (controlled)
  std::vector<int> facts;   // one-qubit: factors in the order they act (op index >= 0, noise -1 - k)
};

struct HProg {
  int n = 0;
  std::vector<OpsStep> steps;      // in round order
  std::vector<OpsRound> rounds;
  std::vector<int> fact_off, facts;  // per-trajectory slots
  std::vector<int> shared_off, shared_facts;  // shared slots (op index each)
  int slots = 0, shared = 0, n_noise = 0;
};

HProg compile_ops(int n, int n_ops, const iqs_op* ops, bool noisy, int R) {
  HProg P;
  P.n = n;
  std::vector<HStep> steps;
  std::vector<int> last_touch(n, -1);  // index of the last step touching each qubit
  int noise = 0;
  auto one_qubit = [&](int q, const std::vector<int>& f) {
    const int lt = last_touch[q];
    if (lt >= 0 && steps[lt].control < 0 && steps[lt].target == q) {  // fuse with the open step on q
      steps[lt].facts.insert(steps[lt].facts.end(), f.begin(), f.end());
      return;
    }
    steps.push_back(HStep{q, -1, -1, f});
    last_touch[q] = (int)steps.size() - 1;
  };
  for (int i = 0; i < n_ops; ++i) {
    const iqs_op& o = ops[i];
    if (o.control < 0) {
      std::vector<int> f{i};
      if (noisy) f.push_back(-1 - noise++);
      one_qubit(o.target, f);
    } else {
      steps.push_back(HStep{o.target, o.control, -1, {i}});
      last_touch[o.target] = last_touch[o.control] = (int)steps.size() - 1;
      if (noisy) {
        one_qubit(o.control, {-1 - noise++});
        one_qubit(o.target, {-1 - noise++});
      }
    }
  }
  P.n_noise = noise;
  // slots
  P.fact_off.push_back(0);
  P.shared_off.push_back(0);
  for (HStep& h : steps) {
    if (h.control < 0) {
      h.slot = P.slots++;
      P.facts.insert(P.facts.end(), h.facts.begin(), h.facts.end());
      P.fact_off.push_back((int)P.facts.size());
    } else {
      h.slot = P.shared++;
      P.shared_facts.push_back(h.facts[0]);
      P.shared_off.push_back((int)P.shared_facts.size());
    }
  }
  // rounds: step i goes into the latest round r >= (last round touching its qubits) with its window
  struct HR { int win; uint32_t touch; std::vector<int> idx; };
  std::vector<HR> rounds;
  for (int i = 0; i < (int)steps.size(); ++i) {
    const HStep& h = steps[i];
    const uint32_t q = (1u << h.target) | (h.control >= 0 ? 1u << h.control : 0u);
    int dep = -1;
    for (int r = (int)rounds.size() - 1; r >= 0; --r)
      if (rounds[r].touch & q) { dep = r; break; }
    const int win = h.target / R;
    int dest = -1;
    for (int r = (int)rounds.size() - 1; r >= std::max(dep, 0); --r)
      if (rounds[r].win == win && (int)rounds[r].idx.size() < kOpsRoundSteps) { dest = r; break; }
    if (dest < 0) {
      rounds.push_back(HR{win, 0u, {}});
      dest = (int)rounds.size() - 1;
    }
    rounds[dest].touch |= q;
    rounds[dest].idx.push_back(i);
  }
  for (const HR& r : rounds) {
    OpsRound o;
    o.pos = r.win * R;
    o.bits = std::min(R, n - o.pos);
    o.first = (int)P.steps.size();
    o.count = (int)r.idx.size();
    for (int i : r.idx) {
      const HStep& h = steps[i];
      OpsStep st;
      st.target = (int16_t)h.target;
      st.control = (int16_t)h.control;
      st.mat = h.control < 0 ? h.slot : -1 - h.slot;
      P.steps.push_back(st);
    }
    P.rounds.push_back(o);
  }
  return P;
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

template <class TR>
iqs_status run_ops(iqs_pool_many* W, int nc, const iqs_ops_circuit* cd, double* probs_out, double* means_out) {
  using Mat = typename TR::Mat;
  using Wt = typename TR::W;
  const int R = TR::kRegBits;
  const int smem_cap_n = sizeof(Wt) == 8 ? 14 : 13;  // 128 KiB of state in shared memory
  std::vector<HProg> progs(nc);
  uint64_t total_traj = 0, total_probs = 0, total_means = 0, total_mats = 0;
  int max_n = 0, smem_max_n = 0, max_global_n = 0;
  size_t n_steps = 0, n_rounds = 0, n_facts = 0, n_sfacts = 0, n_ops = 0, n_ang = 0;
  for (int c = 0; c < nc; ++c) {
    progs[c] = compile_ops(cd[c].n, cd[c].n_ops, cd[c].ops, cd[c].angles != nullptr, R);
    total_traj += cd[c].trajectories;
    total_probs += (uint64_t)cd[c].trajectories * cd[c].n;
    total_means += cd[c].n;
    total_mats += (uint64_t)cd[c].trajectories * progs[c].slots + progs[c].shared;
    max_n = std::max(max_n, cd[c].n);
    n_steps += progs[c].steps.size();
    n_rounds += progs[c].rounds.size();
    n_facts += progs[c].facts.size() + progs[c].fact_off.size();
    n_sfacts += progs[c].shared_facts.size() + progs[c].shared_off.size();
    n_ops += (size_t)cd[c].n_ops;
    if (cd[c].angles) n_ang += (size_t)cd[c].trajectories * progs[c].n_noise * 2;
  }
  smem_max_n = std::min(max_n, smem_cap_n);
  for (int c = 0; c < nc; ++c)
    if (cd[c].n > smem_max_n) max_global_n = std::max(max_global_n, cd[c].n);
  // one CTA per SM slot: grid = trajectories, capped at what is resident
  int dev = 0, sms = 0, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = (size_t)sizeof(Wt) << smem_max_n;
  if (cudaFuncSetAttribute(k_pool_ops<TR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pool_ops<TR>, kThreads, smem) != cudaSuccess)
    return report(IQS_ECUDA, "gate-list pool kernel set-up: %s", cudaGetErrorString(cudaGetLastError()));
  const int grid = (int)std::min<uint64_t>(total_traj, (uint64_t)std::max(1, sms * std::max(per_sm, 1)));
  const uint64_t slot_amps = max_global_n > 0 ? (1ull << max_global_n) : 0;
  // device buffer layout
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = al256(off + bytes);
    return o;
  };
  const size_t o_arena = take(sizeof(Wt) * slot_amps * grid);
  const size_t o_mats = take(sizeof(Mat) * total_mats);
  const size_t o_U = take(sizeof(double) * 8 * n_ops);
  const size_t o_ang = take(sizeof(double) * n_ang);
  const size_t o_fact = take(sizeof(int) * (n_facts + n_sfacts));
  const size_t o_steps = take(sizeof(OpsStep) * n_steps);
  const size_t o_rounds = take(sizeof(OpsRound) * n_rounds);
  const size_t o_progs = take(sizeof(OpsProg) * nc);
  const size_t o_jobs = take(sizeof(OpsJob) * total_traj);
  const size_t o_cjobs = take(sizeof(ComposeJob) * (total_traj + nc));
  const size_t o_probs = take(sizeof(double) * total_probs);
  const size_t o_means = take(sizeof(double) * total_means);
  const size_t o_meta = take((sizeof(uint64_t) * 2 + sizeof(int) * 2) * nc);
  const size_t o_flag = take(sizeof(unsigned));
  const size_t bytes = off;
  cudaStream_t s = W->stream;
  if (bytes > W->ops_bytes) {
    cudaStreamSynchronize(s);
    cudaFree(W->ops_buf);
    W->ops_buf = nullptr;
    W->ops_bytes = 0;
    if (cudaMalloc(&W->ops_buf, bytes) != cudaSuccess) {
      cudaGetLastError();
      return report(IQS_ENOMEM, "gate-list pool: cannot allocate %zu bytes", bytes);
    }
    W->ops_bytes = bytes;
  }
  char* D = static_cast<char*>(W->ops_buf);
  // host image of everything after the arena and the matrices
  const size_t host_from = o_U;
  std::vector<char> H(bytes - host_from, 0);
  auto hptr = [&](size_t o) { return H.data() + (o - host_from); };
  size_t iU = 0, iA = 0, iF = 0, iS = 0, iR = 0;
  uint64_t iM = 0, iP = 0, iMe = 0, iJ = 0;
  std::vector<OpsProg> hp(nc);
  std::vector<OpsJob> hj(total_traj);
  std::vector<ComposeJob> hc;
  std::vector<uint64_t> first(nc), moff(nc);
  std::vector<int> trj(nc), nq(nc);
  for (int c = 0; c < nc; ++c) {
    const HProg& P = progs[c];
    const iqs_ops_circuit& d = cd[c];
    double* Ud = reinterpret_cast<double*>(D + o_U) + iU;
    for (int i = 0; i < d.n_ops; ++i) std::memcpy(reinterpret_cast<double*>(hptr(o_U)) + iU + 8 * i, d.ops[i].U, 64);
    iU += 8 * (size_t)d.n_ops;
    int* fo = reinterpret_cast<int*>(D + o_fact) + iF;
    std::memcpy(reinterpret_cast<int*>(hptr(o_fact)) + iF, P.fact_off.data(), sizeof(int) * P.fact_off.size());
    iF += P.fact_off.size();
    int* ff = reinterpret_cast<int*>(D + o_fact) + iF;
    std::memcpy(reinterpret_cast<int*>(hptr(o_fact)) + iF, P.facts.data(), sizeof(int) * P.facts.size());
    iF += P.facts.size();
    int* so = reinterpret_cast<int*>(D + o_fact) + iF;
    std::memcpy(reinterpret_cast<int*>(hptr(o_fact)) + iF, P.shared_off.data(), sizeof(int) * P.shared_off.size());
    iF += P.shared_off.size();
    int* sf = reinterpret_cast<int*>(D + o_fact) + iF;
    std::memcpy(reinterpret_cast<int*>(hptr(o_fact)) + iF, P.shared_facts.data(), sizeof(int) * P.shared_facts.size());
    iF += P.shared_facts.size();
    const double* Ad = d.angles ? reinterpret_cast<double*>(D + o_ang) + iA : nullptr;
    if (d.angles) {
      const size_t na = (size_t)d.trajectories * P.n_noise * 2;
      std::memcpy(reinterpret_cast<double*>(hptr(o_ang)) + iA, d.angles, sizeof(double) * na);
      iA += na;
    }
    OpsStep* Sd = reinterpret_cast<OpsStep*>(D + o_steps) + iS;
    std::memcpy(reinterpret_cast<OpsStep*>(hptr(o_steps)) + iS, P.steps.data(), sizeof(OpsStep) * P.steps.size());
    iS += P.steps.size();
    OpsRound* Rd = reinterpret_cast<OpsRound*>(D + o_rounds) + iR;
    std::memcpy(reinterpret_cast<OpsRound*>(hptr(o_rounds)) + iR, P.rounds.data(), sizeof(OpsRound) * P.rounds.size());
    iR += P.rounds.size();
    Mat* shared = reinterpret_cast<Mat*>(D + o_mats) + iM;
    iM += P.shared;
    hp[c] = OpsProg{Rd, Sd, shared, d.n, (int)P.rounds.size()};
    if (P.shared > 0) hc.push_back(ComposeJob{Ud, so, sf, nullptr, shared, P.shared});
    first[c] = iP;
    trj[c] = d.trajectories;
    nq[c] = d.n;
    moff[c] = iMe;
    iMe += d.n;
    for (int b = 0; b < d.trajectories; ++b) {
      Mat* m = reinterpret_cast<Mat*>(D + o_mats) + iM;
      iM += P.slots;
      double* pr = reinterpret_cast<double*>(D + o_probs) + iP;
      iP += d.n;
      hj[iJ++] = OpsJob{m, pr, c};
      if (P.slots > 0)
        hc.push_back(ComposeJob{Ud, fo, ff, Ad ? Ad + (size_t)b * P.n_noise * 2 : nullptr, m, P.slots});
    }
  }
  std::memcpy(hptr(o_progs), hp.data(), sizeof(OpsProg) * nc);
  std::memcpy(hptr(o_jobs), hj.data(), sizeof(OpsJob) * total_traj);
  std::memcpy(hptr(o_cjobs), hc.data(), sizeof(ComposeJob) * hc.size());
  char* meta = hptr(o_meta);
  std::memcpy(meta, first.data(), sizeof(uint64_t) * nc);
  std::memcpy(meta + sizeof(uint64_t) * nc, moff.data(), sizeof(uint64_t) * nc);
  std::memcpy(meta + sizeof(uint64_t) * 2 * nc, trj.data(), sizeof(int) * nc);
  std::memcpy(meta + sizeof(uint64_t) * 2 * nc + sizeof(int) * nc, nq.data(), sizeof(int) * nc);
  cudaError_t e = cudaMemcpyAsync(D + host_from, H.data(), H.size(), cudaMemcpyHostToDevice, s);
  unsigned* flag = reinterpret_cast<unsigned*>(D + o_flag);
  if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, sizeof(unsigned), s);
  if (e == cudaSuccess && !hc.empty()) {
    const ComposeJob* cj = reinterpret_cast<const ComposeJob*>(D + o_cjobs);
    k_ops_compose<TR><<<dim3(4, (unsigned)std::min<size_t>(hc.size(), 65535)), 128, 0, s>>>(cj, (int)hc.size());
    e = launched(1);
  }
  if (e == cudaSuccess) {
    k_pool_ops<TR><<<grid, kThreads, smem, s>>>(reinterpret_cast<Wt*>(D + o_arena), slot_amps,
                                                reinterpret_cast<const OpsJob*>(D + o_jobs), (int)total_traj,
                                                reinterpret_cast<const OpsProg*>(D + o_progs), smem_max_n, flag);
    e = launched(1);
  }
  double* dprobs = reinterpret_cast<double*>(D + o_probs);
  double* dmeans = reinterpret_cast<double*>(D + o_means);
  if (e == cudaSuccess) {
    const char* m = D + o_meta;
    k_ops_means<<<nc, 64, 0, s>>>(dprobs, reinterpret_cast<const uint64_t*>(m),
                                  reinterpret_cast<const int*>(m + sizeof(uint64_t) * 2 * nc),
                                  reinterpret_cast<const int*>(m + sizeof(uint64_t) * 2 * nc + sizeof(int) * nc),
                                  reinterpret_cast<const uint64_t*>(m + sizeof(uint64_t) * nc), dmeans);
    e = launched(1);
  }
  if (e == cudaSuccess && probs_out)
    e = cudaMemcpyAsync(probs_out, dprobs, sizeof(double) * total_probs, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(means_out, dmeans, sizeof(double) * total_means, cudaMemcpyDeviceToHost, s);
  unsigned f = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&f, flag, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return report(IQS_ECUDA, "gate-list pool: %s", cudaGetErrorString(e));
  if (f) return report(IQS_ERANGE, "an amplitude outside the emulated-FP64 range was met");
  return IQS_OK;
}

}  // namespace
}  // namespace iqs

extern "C" {

int iqs_ops_noise_count(int n_ops, const iqs_op* ops) {
  if (n_ops < 0 || (n_ops > 0 && ops == nullptr)) return -1;
  int k = 0;
  for (int i = 0; i < n_ops; ++i) k += ops[i].control < 0 ? 1 : 2;
  return k;
}

iqs_status iqs_pool_many_run_ops(iqs_pool_many* w, int n_circuits, const iqs_ops_circuit* circuits, double* probs,
                                 double* means) {
  using namespace iqs;
  if (w == nullptr || circuits == nullptr || means == nullptr) return report(IQS_EINVAL, "NULL argument");
  if (n_circuits < 1 || n_circuits > 100000) return report(IQS_EINVAL, "n_circuits %d outside [1, 100000]", n_circuits);
  for (int c = 0; c < n_circuits; ++c) {
    const iqs_ops_circuit& d = circuits[c];
    if (d.n < 2 || d.n > pool::kPoolMaxQubits || d.n_ops < 0 || d.n_ops > 10000000 || (d.n_ops > 0 && !d.ops) ||
        d.trajectories < 1 || d.trajectories > 1000000)
      return report(IQS_EINVAL, "circuit %d: n %d (2..%d), n_ops %d or trajectories %d invalid", c, d.n,
                    pool::kPoolMaxQubits, d.n_ops, d.trajectories);
    if (d.angles == nullptr && d.trajectories != 1)
      return report(IQS_EINVAL, "circuit %d: a noiseless circuit has exactly one trajectory", c);
    for (int i = 0; i < d.n_ops; ++i) {
      const iqs_op& o = d.ops[i];
      if (o.target < 0 || o.target >= d.n || o.control < -1 || o.control >= d.n || o.control == o.target)
        return report(IQS_EINVAL, "circuit %d, op %d: target %d / control %d invalid for %d qubits", c, i, o.target,
                      o.control, d.n);
      for (int k = 0; k < 8; ++k)
        if (!std::isfinite(o.U[k])) return report(IQS_EINVAL, "circuit %d, op %d: non-finite matrix entry", c, i);
    }
  }
  if (fault_now(2)) return report(IQS_ECUDA, "iqs_pool_many_run_ops: injected launch failure");
  return w->dtype == IQS_C128 ? run_ops<pool::P128>(w, n_circuits, circuits, probs, means)
                              : run_ops<pool::P64>(w, n_circuits, circuits, probs, means);
}

}  // extern "C"
