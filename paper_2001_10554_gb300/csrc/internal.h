// Internal declarations shared by the C-ABI layer and the kernel files.
#pragma once

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "iqs.h"

struct iqs_reg {
  int n = 0;
  int dtype = IQS_C64;
  int math = IQS_MATH_AUTO;
  int device = 0;
  bool owns = false;
  void* data = nullptr;          // 2^n amplitudes, interleaved (re, im)
  cudaStream_t stream = nullptr;
  // scratch: per-block FP64 partials of reductions, their final values, and
  // the out-of-range flag of the emulated complex128 arithmetic
  double* partials = nullptr;    // kRedBlocks * kRedSlots doubles
  double* results = nullptr;     // kRedSlots doubles
  unsigned* flag = nullptr;      // 1 unsigned
  double* host_results = nullptr;  // pinned, kRedSlots doubles
  // queued one-qubit gates on the qubits of one shared-memory tile (iqs_set_fusion):
  // fmat[q] is the FP64 product of the gates queued on qubit q (bit q of fmask set)
  bool fuse = false;
  uint32_t fmask = 0;
  double fmat[16][8];
};

namespace iqs {

constexpr int kRedBlocks = 1024;        // blocks of every reduction kernel (fixed: deterministic order)
constexpr int kRedSlots = 40;           // values reduced at once (n + 1 for all-qubit probabilities)
constexpr int kMaxEdgesFast = 255;      // unweighted ZZ phase: table-driven fast path bound
constexpr int kMaxEdges = 4096;

// A positive integer worked out once per device (kernel attributes and
// occupancy belong to a device).  Threads that race on the first call each
// compute it and store the same value; devices past kDevices are not cached.
struct PerDevice {
  static constexpr int kDevices = 64;
  std::atomic<int> v[kDevices] = {};
  // ``compute(&x)`` sets x (> 0) for the current device.
  template <class F>
  cudaError_t get(int* out, F&& compute) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const bool cached = dev >= 0 && dev < kDevices;
    if (cached && (*out = v[dev].load(std::memory_order_acquire)) > 0) return cudaSuccess;
    int x = 0;
    e = compute(&x);
    if (e != cudaSuccess) return e;
    *out = x > 0 ? x : 1;
    if (cached) v[dev].store(*out, std::memory_order_release);
    return cudaSuccess;
  }
};

// Kernel-launch accounting (iqs_kernel_launches).
void note_launches(int k);
// cudaGetLastError(), counting ``k`` launches when it reports success.
inline cudaError_t launched(int k) {
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) note_launches(k);
  return e;
}

inline uint64_t num_amps(const iqs_reg* r) { return 1ull << r->n; }
inline size_t amp_bytes(const iqs_reg* r) { return r->dtype == IQS_C128 ? 16 : 8; }
inline bool use_emulated(const iqs_reg* r) {
  if (r->dtype != IQS_C128) return false;
  if (r->math == IQS_MATH_EMULATED) return true;
  if (r->math == IQS_MATH_NATIVE) return false;
  return r->n >= 20;
}

// 2x2 gate in FP64, row-major: U[2*row + col] = (re, im)
struct Mat2 {
  double re[4], im[4];
};

// Monomial gate with unit entries in {1, i, -1, -i}: row r takes input
// (perm ? 1 - r : r) times i^k[r].
struct Mono {
  bool perm;
  int k[2];
};
bool as_monomial(const Mat2& u, Mono* m);

// ---- gates.cu
cudaError_t launch_1q(iqs_reg* r, int q, const Mat2& u);
// kgate.cu: iqs_kq_autotune's timing of the k-qubit gate variants.
cudaError_t tune_kq(iqs_reg* r, int k, const int* qubits, const double* U, double* best_ms, int* variant, int* per_sm);
// fuse.cu: qubits [0, fuse_bits(r)) are queued under iqs_set_fusion; launch_fused
// applies the queued products in one tiled pass (it does not clear them).
int fuse_bits(const iqs_reg* r);
cudaError_t launch_fused(iqs_reg* r);
cudaError_t launch_c1q(iqs_reg* r, int c, int t, const Mat2& u);

// ---- phase.cu
cudaError_t launch_init_basis(iqs_reg* r, uint64_t index);
cudaError_t launch_init_uniform(iqs_reg* r);
cudaError_t launch_zz_phase(iqs_reg* r, int n_edges, const int32_t* edges, const double* w, double gamma);
cudaError_t launch_scale(iqs_reg* r, double s);

// ---- reduce.cu: results land in r->results[0..count) (device); the caller copies them.
cudaError_t launch_norm2(iqs_reg* r);
cudaError_t launch_probability(iqs_reg* r, int q);
cudaError_t launch_probabilities(iqs_reg* r);                    // n values
cudaError_t launch_expectation(iqs_reg* r, uint64_t xm, uint64_t zm);
cudaError_t launch_energy(iqs_reg* r, int n_edges, const int32_t* edges, const double* w);
cudaError_t launch_probabilities_raw(const void* data, int n, int dtype, cudaStream_t s, double* partials,
                                     double* results, unsigned* flag);

// ---- kgate.cu: dense k-qubit gates (k <= max_kq(dtype))
int max_kq(int dtype);
cudaError_t launch_kq(iqs_reg* r, int k, const int* qubits, const double* U);
// iqs_kq_set_variant: the variant and blocks per SM used for this register's
// dtype, arithmetic, k and target class from now on in this process.
void set_kq_choice(const iqs_reg* r, int k, const int* qubits, int variant, int per_sm);
// ---- kgate_tc.cu: complex128 k-qubit gates on the tensor cores (k = 2..4)
bool kq_tensor_supported(int k);
cudaError_t launch_kq_c128_tensor(iqs_reg* r, int k, const int* qubits, const double* U);

// ---- measure.cu: qubit-group marginals and sampling
int max_marginal_qubits();
size_t marginal_scratch_bytes(const iqs_reg* r, int k, const int* qubits);
cudaError_t launch_marginal(iqs_reg* r, int k, const int* qubits, double* out_dev, double* partials);
size_t sample_scratch_bytes(int n);
cudaError_t launch_sample(iqs_reg* r, uint64_t shots, const double* u_dev, unsigned long long* out_dev,
                          double* scratch);

// ---- abi.cu: record a failure message for iqs_last_error() and return ``s``.
iqs_status report(iqs_status s, const char* fmt, ...);
// True (once) when an injected fault of ``kind`` (1 allocation, 2 launch) fires.
bool fault_now(int kind);

}  // namespace iqs
