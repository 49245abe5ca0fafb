// Measurement of qubit groups (Section 2, "Scope and basic use": qubits can
// be measured in groups, which gives the joint statistics of their outcomes):
//
//   marginal : out[m] = sum of |alpha_i|^2 over the indices whose bits at
//              qubits[j] equal bit j of m (k <= 10 qubits, 2^k outcomes);
//   sample   : basis states drawn by inverse transform from |alpha_i|^2 with
//              caller-supplied uniforms u: the first index whose cumulative
//              weight exceeds u * (total weight).
//
// Marginal.  Targets below bit 5 are fixed per lane (a warp reads 32
// consecutive amplitudes); up to four targets at bit 5 or above are unrolled
// into per-thread accumulators (a thread visits the 2^KR amplitudes of its
// group, each load coalesced across the warp), and the remaining targets pick
// a slice of the grid (blockIdx.y).  Accumulation: error-free FP32 products
// into double-float, FP64 across lanes, warps and blocks, summed in a fixed
// order, so the result is deterministic.
//
// Sampling.  Three levels: elements in runs of E = 2^min(n, 8), runs grouped
// into chunks of up to 256.  One pass stores every run's weight (double-float)
// and every chunk's weight (FP64); one block forms the chunk prefix P with a
// chained scan (each thread scans a segment sequentially and the segment
// offsets are chained, so P never decreases and stays equal across chunks of
// zero weight); each shot then binary-searches P in FP64 and walks the chunk's
// runs and the run's elements sequentially in double-float (FP32 pipe), against
// its target taken relative to the level's base (about 2^-44 of the chunk's
// weight).  At every level the choice is the first entry of nonzero weight
// whose running sum exceeds the target, else the last entry of nonzero weight
// (rounding can leave the target above the level's last running value); a
// zero-weight entry leaves the running sum unchanged and is never chosen.
#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "df64.cuh"
#include "internal.h"

namespace iqs {
namespace {

constexpr int kWarps = kThreads / 32;
constexpr int kMaxMarginal = 10;

// ---------------------------------------------------------------- marginal
struct MargPlan {
  uint32_t lane_free;     // lane bits (0..4) that are not targets: reduced over
  int kl;                 // targets below bit 5
  int lpos[5];            // their positions, ascending
  int rpos[4];            // register-bin targets (bit >= 5)
  int ky;                 // slice targets (bit >= 5)
  int ypos[kMaxMarginal]; // their positions
  int zpos[kMaxMarginal]; // all positions >= 5 of rpos and ypos, ascending (zero insertion)
  int kz;
};

__device__ __forceinline__ void abs2(float2 a, float& p, float& e, unsigned&) { dfx::abs2_c64(a.x, a.y, p, e); }
__device__ __forceinline__ void abs2(double2 a, float& p, float& e, unsigned& bad) {
  dfx::abs2_c128(a.x, a.y, p, e, bad);
}

// Grid (gx, 2^ky); partials[(y * gx + bx) * (2^kl * 2^KR) + pl * 2^KR + rb].
template <class V, int KR>
__global__ void __launch_bounds__(kThreads, 2) k_marginal(const V* __restrict__ a, uint64_t n_groups, MargPlan P,
                                                          double* __restrict__ partials, unsigned* flag) {
  constexpr int R = 1 << KR;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ uint64_t roff[R];  // register bin m -> index offset (with this slice's bits)
  if (threadIdx.x < R) {
    uint64_t o = 0;
    for (int j = 0; j < P.ky; ++j) o |= (uint64_t)((blockIdx.y >> j) & 1u) << P.ypos[j];
    for (int j = 0; j < KR; ++j) o |= (uint64_t)((threadIdx.x >> j) & 1u) << P.rpos[j];
    roff[threadIdx.x] = o;
  }
  __syncthreads();
  dfx::Acc acc[R];
  unsigned bad = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  // two groups per iteration: 2^(KR+1) independent loads in flight per thread
  for (; g + stride < n_groups; g += 2 * stride) {
    uint64_t b0 = g, b1 = g + stride;
    for (int j = 0; j < P.kz; ++j) {
      b0 = insert_zero(b0, P.zpos[j]);
      b1 = insert_zero(b1, P.zpos[j]);
    }
    V x0[R], x1[R];
#pragma unroll
    for (int m = 0; m < R; ++m) {
      x0[m] = a[b0 + roff[m]];
      x1[m] = a[b1 + roff[m]];
    }
#pragma unroll
    for (int m = 0; m < R; ++m) {
      float p, e;
      abs2(x0[m], p, e, bad);
      acc[m].add(p, e);
      abs2(x1[m], p, e, bad);
      acc[m].add(p, e);
    }
  }
  if (g < n_groups) {
    uint64_t b0 = g;
    for (int j = 0; j < P.kz; ++j) b0 = insert_zero(b0, P.zpos[j]);
#pragma unroll
    for (int m = 0; m < R; ++m) {
      float p, e;
      abs2(a[b0 + roff[m]], p, e, bad);
      acc[m].add(p, e);
    }
  }
  if (bad) atomicOr(flag, 1u);
  double v[R];
#pragma unroll
  for (int m = 0; m < R; ++m) v[m] = acc[m].value();
  // lanes that differ only in non-target lane bits hold the same outcome
#pragma unroll
  for (int b = 0; b < 5; ++b)
    if ((P.lane_free >> b) & 1u) {
#pragma unroll
      for (int m = 0; m < R; ++m) v[m] += __shfl_xor_sync(0xffffffffu, v[m], 1 << b);
    }
  __shared__ double sm[kWarps][32][R];
  if ((lane & P.lane_free) == 0) {
    int pl = 0;
    for (int j = 0; j < P.kl; ++j) pl |= ((lane >> P.lpos[j]) & 1) << j;
#pragma unroll
    for (int m = 0; m < R; ++m) sm[warp][pl][m] = v[m];
  }
  __syncthreads();
  const int outs = (1 << P.kl) * R;
  double* dst = partials + ((uint64_t)blockIdx.y * gridDim.x + blockIdx.x) * outs;
  for (int o = threadIdx.x; o < outs; o += blockDim.x) {
    const int pl = o / R, m = o % R;
    double s = 0.0;
    for (int w = 0; w < kWarps; ++w) s += sm[w][pl][m];
    dst[o] = s;
  }
}

// out[m] for m < 2^k: target j is (cls[j], idx[j]) with cls 0 = lane, 1 = register bin, 2 = slice.
struct MargMap {
  int k, kl, kr, gx;
  int cls[kMaxMarginal], idx[kMaxMarginal];
};

__global__ void k_marginal_finish(const double* __restrict__ partials, MargMap M, double* __restrict__ out) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= (1 << M.k)) return;
  int pl = 0, rb = 0, y = 0;
  for (int j = 0; j < M.k; ++j) {
    const int b = (m >> j) & 1;
    if (M.cls[j] == 0) pl |= b << M.idx[j];
    else if (M.cls[j] == 1) rb |= b << M.idx[j];
    else y |= b << M.idx[j];
  }
  const int outs = (1 << M.kl) << M.kr;
  const int o = (pl << M.kr) | rb;
  double s = 0.0;
  for (int bx = 0; bx < M.gx; ++bx) s += partials[((uint64_t)y * M.gx + bx) * outs + o];
  out[m] = s;
}

// States below 32 amplitudes: one thread per outcome, FP64, index order.
template <class V>
__global__ void k_marginal_small(const V* __restrict__ a, int N, int k, uint32_t qmask0, uint32_t qmask1,
                                 uint32_t qmask2, uint32_t qmask3, double* __restrict__ out) {
  const int m = threadIdx.x;
  if (m >= (1 << k)) return;
  const uint32_t qm[4] = {qmask0, qmask1, qmask2, qmask3};
  double s = 0.0;
  for (int i = 0; i < N; ++i) {
    int mi = 0;
    for (int j = 0; j < k; ++j) mi |= ((i & qm[j]) ? 1 : 0) << j;
    if (mi != m) continue;
    const double re = (double)a[i].x, im = (double)a[i].y;
    s += re * re + im * im;
  }
  out[m] = s;
}

template <class V, int KR>
cudaError_t launch_marginal_kr(const iqs_reg* r, const MargPlan& P, unsigned gx, double* partials) {
  const uint64_t n_groups = num_amps(r) >> (KR + P.ky);
  const dim3 grid(gx, 1u << P.ky);
  k_marginal<V, KR><<<grid, kThreads, 0, r->stream>>>((const V*)r->data, n_groups, P, partials, r->flag);
  return launched(1);
}

// ---------------------------------------------------------------- sampling
struct SampleGeo {
  int e;            // log2 of the run length E
  int c;            // log2 of the runs per chunk
  uint64_t n_runs;  // N / E
  uint64_t n_chunks;
};

// One block per chunk: run weights (double-float, kept as (h, l) float
// pairs for the walks) and the chunk weight (FP64, runs in order).
template <class V>
__global__ void __launch_bounds__(kThreads) k_sample_runs(const V* __restrict__ a, SampleGeo G,
                                                          float2* __restrict__ run_w, double* __restrict__ chunk_w,
                                                          unsigned* flag) {
  __shared__ double sw[256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int E = 1 << G.e, runs = 1 << G.c;
  unsigned bad = 0;
  for (uint64_t ch = blockIdx.x; ch < G.n_chunks; ch += gridDim.x) {
    for (int s = warp; s < runs; s += kWarps) {
      const uint64_t run = ch * (uint64_t)runs + s;
      const V* p = a + run * (uint64_t)E;
      dfx::Acc acc;
      for (int j = lane; j < E; j += 32) {
        float pp, ee;
        abs2(p[j], pp, ee, bad);
        acc.add(pp, ee);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float h = __shfl_xor_sync(0xffffffffu, acc.h, o);
        const float l = __shfl_xor_sync(0xffffffffu, acc.l, o);
        // lanes combine in the same (lower, upper) order so all lanes agree
        if (lane & o) {
          dfx::Acc lo;
          lo.h = h;
          lo.l = l;
          lo.add(acc.h, acc.l);
          acc = lo;
        } else {
          acc.add(h, l);
        }
      }
      if (lane == 0) {
        run_w[run] = make_float2(acc.h, acc.l);
        sw[s] = acc.value();
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int s = 0; s < runs; ++s) t += sw[s];
      chunk_w[ch] = t;
    }
    __syncthreads();
  }
  if (bad) atomicOr(flag, 1u);
}

// One block: prefix[b] = weight of chunks before b, chained (see the file
// comment); prefix[n_chunks] = total.  ``active`` threads (about the square
// root of n_chunks, so the sequential segment sums and the sequential chain of
// segment offsets are both short) each own one segment.
__global__ void __launch_bounds__(1024) k_sample_scan(const double* __restrict__ chunk_w, uint64_t n_chunks, int active,
                                                      double* __restrict__ prefix) {
  __shared__ double seg[1025];
  const uint64_t per = (n_chunks + active - 1) / active;
  const uint64_t lo = threadIdx.x < (unsigned)active ? threadIdx.x * per : n_chunks;
  const uint64_t hi = min(lo + per, n_chunks);
  double r = 0.0;
  for (uint64_t b = lo; b < hi; ++b) r += chunk_w[b];
  seg[threadIdx.x + 1] = r;
  __syncthreads();
  if (threadIdx.x == 0) {
    double o = 0.0;
    for (int t = 0; t < active; ++t) {
      const double w = seg[t + 1];
      seg[t] = o;
      o = o + w;
    }
    seg[active] = o;
    prefix[n_chunks] = o;
  }
  __syncthreads();
  if (threadIdx.x >= (unsigned)active) return;
  const double base = seg[threadIdx.x];
  r = 0.0;
  for (uint64_t b = lo; b < hi; ++b) {
    prefix[b] = base + r;
    r += chunk_w[b];
  }
}



// (r - target) > 0 for a double-float running sum r and target (th, tl).
__device__ __forceinline__ bool above(const dfx::Acc& r, float th, float tl) { return (r.h - th) + (r.l - tl) > 0.f; }

// One thread per shot.  out[s] = sampled index, or ~0 when the state has zero
// weight.  Below the chunk level the walks run in double-float on the FP32
// pipe, against a target taken relative to the level's base: an entry of
// zero weight leaves the running sum unchanged and is never picked.
template <class V>
__global__ void __launch_bounds__(kThreads) k_sample_draw(const V* __restrict__ a, SampleGeo G,
                                                          const float2* __restrict__ run_w,
                                                          const double* __restrict__ prefix,
                                                          const double* __restrict__ u, uint64_t shots,
                                                          unsigned long long* __restrict__ out) {
  const uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (s >= shots) return;
  const double total = prefix[G.n_chunks];
  if (!(total > 0.0)) {
    out[s] = ~0ull;
    return;
  }
  const double t = u[s] * total;
  // chunk: smallest b with t < prefix[b + 1]
  uint64_t lo = 0, hi = G.n_chunks;
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    if (t < prefix[mid + 1]) hi = mid;
    else lo = mid + 1;
  }
  uint64_t b = lo;
  if (b == G.n_chunks) {  // t rounded up to the total: last chunk of nonzero weight
    b = G.n_chunks - 1;
    while (b > 0 && !(prefix[b + 1] > prefix[b])) --b;
  }
  // run within the chunk: the first run of nonzero weight whose running sum
  // exceeds the target, else the last run of nonzero weight.  Weights are
  // read 8 at a time so their loads overlap; the walk itself is sequential.
  const int runs = 1 << G.c;
  const float2* rw = run_w + b * (uint64_t)runs;
  double tau = t - prefix[b];
  float th = (float)tau, tl = (float)(tau - (double)th);
  dfx::Acc r, pick_start, nz_start;
  int pick = -1, last_nz = 0;
  for (int j0 = 0; j0 < runs && pick < 0; j0 += 8) {
    float2 w8[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) w8[q] = j0 + q < runs ? rw[j0 + q] : make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (pick < 0 && j0 + q < runs) {
        const dfx::Acc start = r;
        r.add(w8[q].x, w8[q].y);
        if (w8[q].x != 0.f || w8[q].y != 0.f) {
          last_nz = j0 + q;
          nz_start = start;
          if (above(r, th, tl)) {
            pick = j0 + q;
            pick_start = start;
          }
        }
      }
    }
  }
  if (pick < 0) {
    pick = last_nz;
    pick_start = nz_start;
  }
  // element within the run, the same rule
  tau -= (double)pick_start.h + (double)pick_start.l;
  th = (float)tau;
  tl = (float)(tau - (double)th);
  const int E = 1 << G.e;
  const uint64_t run = b * (uint64_t)runs + pick;
  const V* p = a + run * (uint64_t)E;
  int el = -1, el_nz = 0;
  unsigned unused = 0;
  dfx::Acc r2;
  for (int j0 = 0; j0 < E && el < 0; j0 += 8) {
    V x8[8];
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (j0 + q < E) x8[q] = p[j0 + q];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (el < 0 && j0 + q < E) {
        float pp, ee;
        abs2(x8[q], pp, ee, unused);
        r2.add(pp, ee);
        if (pp != 0.f || ee != 0.f) {
          el_nz = j0 + q;
          if (above(r2, th, tl)) el = j0 + q;
        }
      }
    }
  }
  if (el < 0) el = el_nz;
  out[s] = run * (uint64_t)E + (uint64_t)el;
}

}  // namespace

int max_marginal_qubits() { return kMaxMarginal; }

namespace {

template <class V, int KR>
int occupancy_of() {
  static PerDevice resident;
  int per_sm = 0;
  if (resident.get(&per_sm, [](int* x) {
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(x, k_marginal<V, KR>, kThreads, 0);
      }) != cudaSuccess) {
    cudaGetLastError();
    per_sm = 2;  // the kernel's launch bound
  }
  return per_sm;
}

int marginal_blocks_per_sm(int dtype, int kr) {
  const bool c64 = dtype == IQS_C64;
  switch (kr) {
    case 0: return c64 ? occupancy_of<float2, 0>() : occupancy_of<double2, 0>();
    case 1: return c64 ? occupancy_of<float2, 1>() : occupancy_of<double2, 1>();
    case 2: return c64 ? occupancy_of<float2, 2>() : occupancy_of<double2, 2>();
    case 3: return c64 ? occupancy_of<float2, 3>() : occupancy_of<double2, 3>();
    default: return c64 ? occupancy_of<float2, 4>() : occupancy_of<double2, 4>();
  }
}

struct MarginalLaunch {
  MargPlan P;
  MargMap M;
  int kr;
  uint64_t gx;
};

// Classify the targets: below bit 5 by lane; of the rest, the lowest four
// become register bins and the others grid slices.
MarginalLaunch plan_marginal(const iqs_reg* r, int k, const int* qubits) {
  MarginalLaunch L;
  std::memset(&L, 0, sizeof(L));
  MargPlan& P = L.P;
  MargMap& M = L.M;
  M.k = k;
  int order[kMaxMarginal];
  for (int j = 0; j < k; ++j) order[j] = j;
  std::sort(order, order + k, [&](int x, int y) { return qubits[x] < qubits[y]; });
  P.lane_free = 31u;
  for (int t = 0; t < k; ++t) {
    const int j = order[t], q = qubits[j];
    if (q < 5) {
      M.cls[j] = 0;
      M.idx[j] = P.kl;
      P.lpos[P.kl++] = q;
      P.lane_free &= ~(1u << q);
    } else if (L.kr < 4) {
      M.cls[j] = 1;
      M.idx[j] = L.kr;
      P.rpos[L.kr++] = q;
      P.zpos[P.kz++] = q;  // ascending: targets are visited in ascending order
    } else {
      M.cls[j] = 2;
      M.idx[j] = P.ky;
      P.ypos[P.ky++] = q;
      P.zpos[P.kz++] = q;
    }
  }
  M.kl = P.kl;
  M.kr = L.kr;
  // one resident wave: blocks per SM (from the occupancy of this variant) x SMs, over the slices
  const uint64_t n_groups = num_amps(r) >> (L.kr + P.ky);
  const uint64_t gx = (n_groups + kThreads - 1) / kThreads;
  const uint64_t cap = std::max<uint64_t>(1, (uint64_t)(marginal_blocks_per_sm(r->dtype, L.kr) * kSMs) >> P.ky);
  L.gx = std::min(gx, cap);
  M.gx = (int)L.gx;
  return L;
}

}  // namespace

size_t marginal_scratch_bytes(const iqs_reg* r, int k, const int* qubits) {
  if (r->n < 5) return 0;
  const MarginalLaunch L = plan_marginal(r, k, qubits);
  return sizeof(double) * (size_t)L.gx * ((size_t)1 << k);
}

// out_dev: 2^k doubles (device); partials: marginal_scratch_bytes() bytes.
cudaError_t launch_marginal(iqs_reg* r, int k, const int* qubits, double* out_dev, double* partials) {
  const bool c64 = r->dtype == IQS_C64;
  if (r->n < 5) {
    uint32_t qm[4] = {0, 0, 0, 0};
    for (int j = 0; j < k; ++j) qm[j] = 1u << qubits[j];
    if (c64)
      k_marginal_small<float2><<<1, 32, 0, r->stream>>>((const float2*)r->data, 1 << r->n, k, qm[0], qm[1], qm[2],
                                                        qm[3], out_dev);
    else
      k_marginal_small<double2><<<1, 32, 0, r->stream>>>((const double2*)r->data, 1 << r->n, k, qm[0], qm[1],
                                                         qm[2], qm[3], out_dev);
    return launched(1);
  }
  const MarginalLaunch L = plan_marginal(r, k, qubits);
  const unsigned gx = (unsigned)L.gx;
  cudaError_t e = cudaSuccess;
  switch (L.kr) {
    case 0: e = c64 ? launch_marginal_kr<float2, 0>(r, L.P, gx, partials) : launch_marginal_kr<double2, 0>(r, L.P, gx, partials); break;
    case 1: e = c64 ? launch_marginal_kr<float2, 1>(r, L.P, gx, partials) : launch_marginal_kr<double2, 1>(r, L.P, gx, partials); break;
    case 2: e = c64 ? launch_marginal_kr<float2, 2>(r, L.P, gx, partials) : launch_marginal_kr<double2, 2>(r, L.P, gx, partials); break;
    case 3: e = c64 ? launch_marginal_kr<float2, 3>(r, L.P, gx, partials) : launch_marginal_kr<double2, 3>(r, L.P, gx, partials); break;
    default: e = c64 ? launch_marginal_kr<float2, 4>(r, L.P, gx, partials) : launch_marginal_kr<double2, 4>(r, L.P, gx, partials); break;
  }
  if (e != cudaSuccess) return e;
  const int outs = 1 << k;
  k_marginal_finish<<<(outs + kThreads - 1) / kThreads, kThreads, 0, r->stream>>>(partials, L.M, out_dev);
  return launched(1);
}

namespace {
SampleGeo sample_geo(int n) {
  SampleGeo G;
  G.e = std::min(n, 8);
  G.c = std::min(n - G.e, 8);
  G.n_runs = 1ull << (n - G.e);
  G.n_chunks = 1ull << (n - G.e - G.c);
  return G;
}
}  // namespace

size_t sample_scratch_bytes(int n) {
  const SampleGeo G = sample_geo(n);
  return sizeof(double) * (G.n_runs + G.n_chunks + G.n_chunks + 1);
}

// scratch: sample_scratch_bytes(n) bytes; u_dev: shots uniforms; out_dev: shots indices.
cudaError_t launch_sample(iqs_reg* r, uint64_t shots, const double* u_dev, unsigned long long* out_dev,
                          double* scratch) {
  const SampleGeo G = sample_geo(r->n);
  float2* run_w = reinterpret_cast<float2*>(scratch);  // n_runs (h, l) pairs: 8 bytes each
  double* chunk_w = scratch + G.n_runs;
  double* prefix = chunk_w + G.n_chunks;
  const unsigned gblocks = (unsigned)std::min<uint64_t>(G.n_chunks, 16ull * kSMs);
  const unsigned dblocks = (unsigned)((shots + kThreads - 1) / kThreads);
  if (r->dtype == IQS_C64)
    k_sample_runs<float2><<<gblocks, kThreads, 0, r->stream>>>((const float2*)r->data, G, run_w, chunk_w, r->flag);
  else
    k_sample_runs<double2><<<gblocks, kThreads, 0, r->stream>>>((const double2*)r->data, G, run_w, chunk_w, r->flag);
  cudaError_t e = launched(1);
  if (e != cudaSuccess) return e;
  int lg = 0;
  while ((1ull << lg) < G.n_chunks) ++lg;
  const int active = std::min(1024, 1 << ((lg + 1) / 2));
  k_sample_scan<<<1, 1024, 0, r->stream>>>(chunk_w, G.n_chunks, active, prefix);
  if ((e = launched(1)) != cudaSuccess) return e;
  if (shots == 0) return cudaSuccess;
  if (r->dtype == IQS_C64)
    k_sample_draw<float2><<<dblocks, kThreads, 0, r->stream>>>((const float2*)r->data, G, run_w, prefix, u_dev, shots,
                                                              out_dev);
  else
    k_sample_draw<double2><<<dblocks, kThreads, 0, r->stream>>>((const double2*)r->data, G, run_w, prefix, u_dev,
                                                               shots, out_dev);
  return launched(1);
}

}  // namespace iqs
