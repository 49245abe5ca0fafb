// C ABI (include/iqs.h): register lifecycle, argument checks, dispatch to the
// kernel launchers, and synchronous result delivery.  No call aborts or
// prints; failures return a status and leave a thread-local message.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include <algorithm>
#include <atomic>
#include <cstdlib>

#include "internal.h"

#include <nvtx3/nvToolsExt.h>

namespace {

std::atomic<uint64_t> g_launches{0};

// Host-side fault injection (iqs_inject_fault / IQS_FAULT): kind 1 = allocation,
// 2 = kernel launch; the fault fires on the (countdown + 1)-th event of that kind.
std::atomic<int> g_fault_kind{0};
std::atomic<int> g_fault_countdown{0};

struct FaultEnv {
  FaultEnv() {
    const char* v = std::getenv("IQS_FAULT");
    if (v == nullptr) return;
    int kind = 0;
    if (std::strncmp(v, "alloc", 5) == 0) kind = 1;
    else if (std::strncmp(v, "launch", 6) == 0) kind = 2;
    const char* colon = std::strchr(v, ':');
    g_fault_countdown = colon ? std::atoi(colon + 1) : 0;
    g_fault_kind = kind;
  }
} g_fault_env;

thread_local char g_err[512] = "";

iqs_status fail(iqs_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

iqs_status cuda_fail(cudaError_t e, const char* what) {
  cudaGetLastError();  // clear a sticky launch error where possible
  return fail(IQS_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CHECK_REG(r)                                                  \
  do {                                                                \
    if ((r) == nullptr) return fail(IQS_EINVAL, "register is NULL");  \
  } while (0)

// One NVTX range per ABI call, named after the call, so a profiler timeline
// shows which library call issued which kernels (a no-op without a profiler).
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
};
#define TRACE() TraceRange trace_range_(__func__)

// Apply the gates queued under iqs_set_fusion before anything else reads or
// changes the state.
iqs_status flush_pending(iqs_reg* r) {
  if (r->fmask == 0) return IQS_OK;
  if (iqs::fault_now(2)) return fail(IQS_ECUDA, "flush of queued gates: injected launch failure");
  const cudaError_t e = iqs::launch_fused(r);
  if (e != cudaSuccess) return fail(IQS_ECUDA, "flush of queued gates: %s", cudaGetErrorString(e));
  r->fmask = 0;
  return IQS_OK;
}

#define FLUSH(r)                                                            \
  do {                                                                      \
    iqs_status s_ = flush_pending(const_cast<iqs_reg*>(r));                 \
    if (s_ != IQS_OK) return s_;                                            \
  } while (0)

// A kernel-launching call: an armed launch fault fails it before anything is queued.
#define LAUNCH_TRY(expr, what)                                                              \
  do {                                                                                      \
    if (iqs::fault_now(2)) return fail(IQS_ECUDA, "%s: injected launch failure", what);    \
    cudaError_t e_ = (expr);                                                                \
    if (e_ != cudaSuccess) return cuda_fail(e_, what);                                      \
  } while (0)

#define CUDA_TRY(expr, what)                         \
  do {                                               \
    cudaError_t e_ = (expr);                         \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

iqs_status check_dtype(int dtype) {
  if (dtype != IQS_C64 && dtype != IQS_C128) return fail(IQS_EINVAL, "dtype must be IQS_C64 or IQS_C128");
  return IQS_OK;
}

iqs_status check_n(int n) {
  if (n < 1 || n > IQS_MAX_QUBITS) return fail(IQS_EINVAL, "number of qubits %d outside [1, %d]", n, IQS_MAX_QUBITS);
  return IQS_OK;
}

iqs_status alloc_scratch(iqs_reg* r) {
  using namespace iqs;
  if (cudaMalloc(&r->partials, sizeof(double) * kRedBlocks * kRedSlots) != cudaSuccess ||
      cudaMalloc(&r->results, sizeof(double) * kRedSlots) != cudaSuccess ||
      cudaMalloc(&r->flag, sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    return fail(IQS_ENOMEM, "cannot allocate reduction scratch");
  }
  if (cudaMallocHost(&r->host_results, sizeof(double) * kRedSlots) != cudaSuccess) {
    cudaGetLastError();
    return fail(IQS_ENOMEM, "cannot allocate pinned result buffer");
  }
  CUDA_TRY(cudaMemsetAsync(r->flag, 0, sizeof(unsigned), r->stream), "clear flag");
  return IQS_OK;
}

void free_reg(iqs_reg* r) {
  if (r->owns && r->data) cudaFree(r->data);
  if (r->partials) cudaFree(r->partials);
  if (r->results) cudaFree(r->results);
  if (r->flag) cudaFree(r->flag);
  if (r->host_results) cudaFreeHost(r->host_results);
  delete r;
}

iqs_status new_reg(int n, int dtype, void* ptr, bool owns, void* stream, iqs_reg** out) {
  if (out == nullptr) return fail(IQS_EINVAL, "out is NULL");
  *out = nullptr;
  iqs_status s = check_n(n);
  if (s != IQS_OK) return s;
  if ((s = check_dtype(dtype)) != IQS_OK) return s;
  iqs_reg* r = new (std::nothrow) iqs_reg();
  if (r == nullptr) return fail(IQS_ENOMEM, "host allocation failed");
  r->n = n;
  r->dtype = dtype;
  r->stream = (cudaStream_t)stream;
  cudaGetDevice(&r->device);
  if (iqs::fault_now(1)) {
    delete r;
    return fail(IQS_ENOMEM, "injected allocation failure");
  }
  if (owns) {
    const size_t bytes = (size_t)iqs::num_amps(r) * iqs::amp_bytes(r);
    if (cudaMalloc(&r->data, bytes) != cudaSuccess) {
      cudaGetLastError();
      delete r;
      return fail(IQS_ENOMEM, "cannot allocate %zu bytes for the state", bytes);
    }
    r->owns = true;
  } else {
    if (ptr == nullptr || ((uintptr_t)ptr & 15u)) {
      delete r;
      return fail(IQS_EINVAL, "device pointer is NULL or not 16-byte aligned");
    }
    r->data = ptr;
  }
  if ((s = alloc_scratch(r)) != IQS_OK) {
    free_reg(r);
    return s;
  }
  if (owns) {
    const cudaError_t e = iqs::launch_init_basis(r, 0);
    if (e != cudaSuccess) {
      free_reg(r);
      return cuda_fail(e, "initialise state");
    }
  }
  *out = r;
  return IQS_OK;
}

iqs_status read_results(iqs_reg* r, int count, double* out) {
  CUDA_TRY(cudaMemcpyAsync(r->host_results, r->results, sizeof(double) * count, cudaMemcpyDeviceToHost, r->stream),
           "copy results");
  CUDA_TRY(cudaStreamSynchronize(r->stream), "synchronise");
  std::memcpy(out, r->host_results, sizeof(double) * count);
  return IQS_OK;
}

iqs_status check_flag(iqs_reg* r) {
  unsigned f = 0;
  CUDA_TRY(cudaMemcpyAsync(&f, r->flag, sizeof(unsigned), cudaMemcpyDeviceToHost, r->stream), "read flag");
  CUDA_TRY(cudaStreamSynchronize(r->stream), "synchronise");
  if (f) {
    CUDA_TRY(cudaMemsetAsync(r->flag, 0, sizeof(unsigned), r->stream), "clear flag");
    if (f & 2u) return fail(IQS_ETIMEOUT, "a bounded wait of a tensor-core kernel gave up");
    return fail(IQS_ERANGE, "an amplitude with |a| >= 2^64, Inf or NaN was met by emulated complex128 arithmetic");
  }
  return IQS_OK;
}

iqs::Mat2 to_mat(const double* U) {
  iqs::Mat2 m;
  for (int k = 0; k < 4; ++k) {
    m.re[k] = U[2 * k];
    m.im[k] = U[2 * k + 1];
  }
  return m;
}

iqs_status check_edges(const iqs_reg* r, int n_edges, const int32_t* edges) {
  if (n_edges < 0 || n_edges > iqs::kMaxEdges) return fail(IQS_EINVAL, "n_edges %d outside [0, %d]", n_edges, iqs::kMaxEdges);
  if (n_edges > 0 && edges == nullptr) return fail(IQS_EINVAL, "edges is NULL");
  for (int e = 0; e < n_edges; ++e) {
    const int u = edges[2 * e], v = edges[2 * e + 1];
    if (u < 0 || u >= r->n || v < 0 || v >= r->n || u == v)
      return fail(IQS_EINVAL, "edge %d = (%d, %d) invalid for %d qubits", e, u, v, r->n);
  }
  return IQS_OK;
}

// k distinct qubits in [0, n).
iqs_status check_qubit_set(const iqs_reg* r, int k, const int* qubits) {
  uint64_t seen = 0;
  for (int j = 0; j < k; ++j) {
    const int q = qubits[j];
    if (q < 0 || q >= r->n) return fail(IQS_EINVAL, "qubit %d outside [0, %d)", q, r->n);
    if ((seen >> q) & 1ull) return fail(IQS_EINVAL, "qubit %d listed twice", q);
    seen |= 1ull << q;
  }
  return IQS_OK;
}

// Temporary device memory from the stream-ordered allocator, returned on the
// same stream (release(), or the destructor on an early error return).
struct DeviceScratch {
  cudaStream_t stream;
  void* ptr = nullptr;
  explicit DeviceScratch(cudaStream_t s) : stream(s) {}
  iqs_status get(size_t bytes) {
    if (iqs::fault_now(1)) return fail(IQS_ENOMEM, "injected allocation failure");
    if (cudaMallocAsync(&ptr, bytes < 16 ? 16 : bytes, stream) != cudaSuccess) {
      cudaGetLastError();
      ptr = nullptr;
      return fail(IQS_ENOMEM, "cannot allocate %zu bytes of scratch", bytes);
    }
    return IQS_OK;
  }
  iqs_status release() {
    if (ptr == nullptr) return IQS_OK;
    const cudaError_t e = cudaFreeAsync(ptr, stream);
    ptr = nullptr;
    return e == cudaSuccess ? IQS_OK : cuda_fail(e, "free scratch");
  }
  ~DeviceScratch() {
    if (ptr) cudaFreeAsync(ptr, stream);
  }
};

}  // namespace

void iqs::note_launches(int k) { g_launches.fetch_add((uint64_t)k); }

bool iqs::fault_now(int kind) {
  if (g_fault_kind.load() != kind) return false;
  if (g_fault_countdown.fetch_sub(1) > 0) return false;
  g_fault_kind = 0;
  g_fault_countdown = 0;
  return true;
}

iqs_status iqs::report(iqs_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

extern "C" {

iqs_status iqs_create(int n, int dtype, void* stream, iqs_reg** out) {
  TRACE();
  return new_reg(n, dtype, nullptr, true, stream, out);
}

iqs_status iqs_wrap(int n, int dtype, void* device_ptr, void* stream, iqs_reg** out) {
  TRACE();
  return new_reg(n, dtype, device_ptr, false, stream, out);
}

iqs_status iqs_destroy(iqs_reg* reg) {
  TRACE();
  if (reg == nullptr) return IQS_OK;
  flush_pending(reg);  // a borrowed buffer outlives the register: it gets the queued gates
  cudaStreamSynchronize(reg->stream);
  free_reg(reg);
  return IQS_OK;
}

iqs_status iqs_data(const iqs_reg* reg, void** device_ptr) {
  TRACE();
  CHECK_REG(reg);
  FLUSH(reg);
  if (device_ptr == nullptr) return fail(IQS_EINVAL, "out is NULL");
  *device_ptr = reg->data;
  return IQS_OK;
}

iqs_status iqs_info(const iqs_reg* reg, int* n, int* dtype) {
  TRACE();
  CHECK_REG(reg);
  if (n) *n = reg->n;
  if (dtype) *dtype = reg->dtype;
  return IQS_OK;
}

iqs_status iqs_set_stream(iqs_reg* reg, void* stream) {
  TRACE();
  CHECK_REG(reg);
  FLUSH(reg);
  reg->stream = (cudaStream_t)stream;
  return IQS_OK;
}

iqs_status iqs_set_math(iqs_reg* reg, int math) {
  TRACE();
  CHECK_REG(reg);
  FLUSH(reg);
  if (math != IQS_MATH_AUTO && math != IQS_MATH_EMULATED && math != IQS_MATH_NATIVE)
    return fail(IQS_EINVAL, "unknown math mode %d", math);
  reg->math = math;
  return IQS_OK;
}

iqs_status iqs_synchronize(iqs_reg* reg) {
  TRACE();
  CHECK_REG(reg);
  FLUSH(reg);
  return check_flag(reg);
}

iqs_status iqs_init_basis(iqs_reg* reg, uint64_t index) {
  TRACE();
  CHECK_REG(reg);
  reg->fmask = 0;  // the state is replaced: queued gates are void
  if (index >= iqs::num_amps(reg)) return fail(IQS_EINVAL, "basis index out of range");
  LAUNCH_TRY(iqs::launch_init_basis(reg, index), "init_basis");
  return IQS_OK;
}

iqs_status iqs_init_uniform(iqs_reg* reg) {
  TRACE();
  CHECK_REG(reg);
  reg->fmask = 0;  // the state is replaced: queued gates are void
  LAUNCH_TRY(iqs::launch_init_uniform(reg), "init_uniform");
  return IQS_OK;
}

iqs_status iqs_upload(iqs_reg* reg, const void* host, size_t bytes) {
  TRACE();
  CHECK_REG(reg);
  reg->fmask = 0;  // the state is replaced: queued gates are void
  if (host == nullptr || bytes != iqs::num_amps(reg) * iqs::amp_bytes(reg))
    return fail(IQS_EINVAL, "upload: NULL buffer or size %zu != state size", bytes);
  CUDA_TRY(cudaMemcpyAsync(reg->data, host, bytes, cudaMemcpyHostToDevice, reg->stream), "upload");
  CUDA_TRY(cudaStreamSynchronize(reg->stream), "upload sync");
  return IQS_OK;
}

iqs_status iqs_download(const iqs_reg* reg, void* host, size_t bytes) {
  TRACE();
  CHECK_REG(reg);
  FLUSH(reg);
  if (host == nullptr || bytes != iqs::num_amps(reg) * iqs::amp_bytes(reg))
    return fail(IQS_EINVAL, "download: NULL buffer or size %zu != state size", bytes);
  CUDA_TRY(cudaMemcpyAsync(host, reg->data, bytes, cudaMemcpyDeviceToHost, reg->stream), "download");
  CUDA_TRY(cudaStreamSynchronize(reg->stream), "download sync");
  return IQS_OK;
}

iqs_status iqs_copy_to_device(iqs_reg* reg, const void* host, uint64_t first, uint64_t count) {
  TRACE();
  CHECK_REG(reg);
  if (host == nullptr || first > iqs::num_amps(reg) || count > iqs::num_amps(reg) - first)
    return fail(IQS_EINVAL, "copy_to_device: NULL buffer or amplitudes [%llu, +%llu) outside the state",
                (unsigned long long)first, (unsigned long long)count);
  if (count == 0) return IQS_OK;
  reg->fmask = 0;  // part of the state is replaced: queued gates are void
  const size_t ab = iqs::amp_bytes(reg);
  CUDA_TRY(cudaMemcpyAsync((char*)reg->data + first * ab, host, count * ab, cudaMemcpyHostToDevice, reg->stream),
           "copy_to_device");
  return IQS_OK;
}

iqs_status iqs_copy_to_host(iqs_reg* reg, void* host, uint64_t first, uint64_t count) {
  TRACE();
  CHECK_REG(reg);
  FLUSH(reg);
  if (host == nullptr || first > iqs::num_amps(reg) || count > iqs::num_amps(reg) - first)
    return fail(IQS_EINVAL, "copy_to_host: NULL buffer or amplitudes [%llu, +%llu) outside the state",
                (unsigned long long)first, (unsigned long long)count);
  if (count == 0) return IQS_OK;
  const size_t ab = iqs::amp_bytes(reg);
  CUDA_TRY(cudaMemcpyAsync(host, (const char*)reg->data + first * ab, count * ab, cudaMemcpyDeviceToHost, reg->stream),
           "copy_to_host");
  return IQS_OK;
}

iqs_status iqs_apply_1q(iqs_reg* reg, int q, const double U[8]) {
  TRACE();
  CHECK_REG(reg);
  if (U == nullptr) return fail(IQS_EINVAL, "U is NULL");
  if (q < 0 || q >= reg->n) return fail(IQS_EINVAL, "qubit %d outside [0, %d)", q, reg->n);
  if (reg->fuse && q < iqs::fuse_bits(reg) && !(reg->dtype == IQS_C128 && reg->math == IQS_MATH_NATIVE)) {
    double* m = reg->fmat[q];
    if (!((reg->fmask >> q) & 1u)) {
      for (int k = 0; k < 8; ++k) m[k] = U[k];
    } else {  // m <- U m, FP64
      double t[8];
      for (int row = 0; row < 2; ++row)
        for (int col = 0; col < 2; ++col) {
          const double ar = U[2 * (2 * row)], ai = U[2 * (2 * row) + 1];
          const double br = U[2 * (2 * row + 1)], bi = U[2 * (2 * row + 1) + 1];
          const double cr = m[2 * col], ci = m[2 * col + 1];
          const double dr = m[2 * (2 + col)], di = m[2 * (2 + col) + 1];
          t[2 * (2 * row + col)] = ar * cr - ai * ci + br * dr - bi * di;
          t[2 * (2 * row + col) + 1] = ar * ci + ai * cr + br * di + bi * dr;
        }
      for (int k = 0; k < 8; ++k) m[k] = t[k];
    }
    reg->fmask |= 1u << q;
    return IQS_OK;
  }
  FLUSH(reg);
  LAUNCH_TRY(iqs::launch_1q(reg, q, to_mat(U)), "apply_1q");
  return IQS_OK;
}

iqs_status iqs_set_fusion(iqs_reg* reg, int on) {
  TRACE();
  CHECK_REG(reg);
  if (!on) FLUSH(reg);
  reg->fuse = on != 0;
  return IQS_OK;
}

iqs_status iqs_flush(iqs_reg* reg) {
  TRACE();
  CHECK_REG(reg);
  FLUSH(reg);
  return IQS_OK;
}

iqs_status iqs_apply_c1q(iqs_reg* reg, int c, int t, const double U[8]) {
  TRACE();
  CHECK_REG(reg);
  FLUSH(reg);
  if (U == nullptr) return fail(IQS_EINVAL, "U is NULL");
  if (c < 0 || c >= reg->n || t < 0 || t >= reg->n) return fail(IQS_EINVAL, "control/target outside [0, %d)", reg->n);
  if (c == t) return fail(IQS_EINVAL, "control and target are the same qubit (%d)", c);
  if (reg->n < 2) return fail(IQS_EINVAL, "a controlled gate needs 2 qubits");
  LAUNCH_TRY(iqs::launch_c1q(reg, c, t, to_mat(U)), "apply_c1q");
  return IQS_OK;
}

iqs_status iqs_apply_zz_phase(iqs_reg* reg, int n_edges, const int32_t* edges, const double* weights, double gamma) {
  TRACE();
  CHECK_REG(reg);
  FLUSH(reg);
  iqs_status s = check_edges(reg, n_edges, edges);
  if (s != IQS_OK) return s;
  if (!std::isfinite(gamma)) return fail(IQS_EINVAL, "gamma is not finite");
  if (weights)
    for (int e = 0; e < n_edges; ++e)
      if (!std::isfinite(weights[e])) return fail(IQS_EINVAL, "weight %d is not finite", e);
  LAUNCH_TRY(iqs::launch_zz_phase(reg, n_edges, edges, weights, gamma), "apply_zz_phase");
  return IQS_OK;
}

iqs_status iqs_norm2(iqs_reg* reg, double* out) {
  TRACE();
  CHECK_REG(reg);
  FLUSH(reg);
  if (out == nullptr) return fail(IQS_EINVAL, "out is NULL");
  LAUNCH_TRY(iqs::launch_norm2(reg), "norm2");
  iqs_status s = read_results(reg, 1, out);
  return s != IQS_OK ? s : check_flag(reg);
}

iqs_status iqs_probability(iqs_reg* reg, int q, double* out) {
  TRACE();
  CHECK_REG(reg);
  FLUSH(reg);
  if (out == nullptr) return fail(IQS_EINVAL, "out is NULL");
  if (q < 0 || q >= reg->n) return fail(IQS_EINVAL, "qubit %d outside [0, %d)", q, reg->n);
  LAUNCH_TRY(iqs::launch_probability(reg, q), "probability");
  iqs_status s = read_results(reg, 1, out);
  return s != IQS_OK ? s : check_flag(reg);
}

iqs_status iqs_probabilities(iqs_reg* reg, double* out) {
  TRACE();
  CHECK_REG(reg);
  FLUSH(reg);
  if (out == nullptr) return fail(IQS_EINVAL, "out is NULL");
  LAUNCH_TRY(iqs::launch_probabilities(reg), "probabilities");
  iqs_status s = read_results(reg, reg->n, out);
  return s != IQS_OK ? s : check_flag(reg);
}

iqs_status iqs_expectation_masks(iqs_reg* reg, uint64_t xmask, uint64_t zmask, double* out) {
  TRACE();
  CHECK_REG(reg);
  FLUSH(reg);
  if (out == nullptr) return fail(IQS_EINVAL, "out is NULL");
  const uint64_t all = reg->n >= 64 ? ~0ull : ((1ull << reg->n) - 1ull);
  if ((xmask | zmask) & ~all) return fail(IQS_EINVAL, "mask bits at or above n = %d", reg->n);
  LAUNCH_TRY(iqs::launch_expectation(reg, xmask, zmask), "expectation");
  double v;
  iqs_status s = read_results(reg, 1, &v);
  if (s != IQS_OK) return s;
  if (xmask != 0) {
    // pair sum times 2 * (sign from i^{nY}): nY = 0 -> +Re, 1 -> -Im, 2 -> -Re, 3 -> +Im
    const int nY = __builtin_popcountll(xmask & zmask) & 3;
    const double sgn = (nY == 0 || nY == 3) ? 1.0 : -1.0;
    v = 2.0 * sgn * v;
  }
  *out = v;
  return check_flag(reg);
}

iqs_status iqs_expectation(iqs_reg* reg, const char* pauli, double* out) {
  TRACE();
  CHECK_REG(reg);
  if (pauli == nullptr) return fail(IQS_EINVAL, "pauli is NULL");
  const size_t len = strnlen(pauli, IQS_MAX_QUBITS + 2);
  if ((int)len != reg->n) return fail(IQS_EINVAL, "Pauli string length %zu != n = %d", len, reg->n);
  uint64_t xm = 0, zm = 0;
  for (int k = 0; k < reg->n; ++k) {
    switch (pauli[k]) {
      case 'I': break;
      case 'X': xm |= 1ull << k; break;
      case 'Y': xm |= 1ull << k; zm |= 1ull << k; break;
      case 'Z': zm |= 1ull << k; break;
      default: return fail(IQS_EINVAL, "bad Pauli character '%c' at %d", pauli[k], k);
    }
  }
  return iqs_expectation_masks(reg, xm, zm, out);
}

iqs_status iqs_renormalize(iqs_reg* reg) {
  TRACE();
  CHECK_REG(reg);
  double nn;
  iqs_status s = iqs_norm2(reg, &nn);
  if (s != IQS_OK) return s;
  if (!(nn > 0.0) || !std::isfinite(nn)) return fail(IQS_EINVAL, "cannot renormalise a state of squared norm %g", nn);
  LAUNCH_TRY(iqs::launch_scale(reg, 1.0 / std::sqrt(nn)), "renormalize");
  return IQS_OK;
}

iqs_status iqs_energy_maxcut(iqs_reg* reg, int n_edges, const int32_t* edges, const double* weights, double* out) {
  TRACE();
  CHECK_REG(reg);
  FLUSH(reg);
  if (out == nullptr) return fail(IQS_EINVAL, "out is NULL");
  iqs_status s = check_edges(reg, n_edges, edges);
  if (s != IQS_OK) return s;
  double total = 0.0;
  for (int base = 0; base < n_edges; base += 255) {
    const int m = n_edges - base < 255 ? n_edges - base : 255;
    LAUNCH_TRY(iqs::launch_energy(reg, m, edges + 2 * base, weights ? weights + base : nullptr), "energy");
    double v;
    if ((s = read_results(reg, 1, &v)) != IQS_OK) return s;
    total += v;
  }
  *out = total;
  return check_flag(reg);
}

iqs_status iqs_apply_kq(iqs_reg* reg, int k, const int* qubits, const double* U) {
  TRACE();
  CHECK_REG(reg);
  FLUSH(reg);
  if (U == nullptr || qubits == nullptr) return fail(IQS_EINVAL, "qubits or U is NULL");
  const int kmax = iqs::max_kq(reg->dtype);
  if (k < 1 || k > kmax || k > reg->n) return fail(IQS_EINVAL, "k = %d outside [1, %d] for this register", k, kmax);
  iqs_status s = check_qubit_set(reg, k, qubits);
  if (s != IQS_OK) return s;
  const int entries = 2 << (2 * k);
  for (int i = 0; i < entries; ++i)
    if (!std::isfinite(U[i])) return fail(IQS_EINVAL, "U entry %d is not finite", i / 2);
  LAUNCH_TRY(iqs::launch_kq(reg, k, qubits, U), "apply_kq");
  return IQS_OK;
}

iqs_status iqs_kq_autotune(iqs_reg* reg, int k, const int* qubits, const double* U, double* best_ms, int* variant,
                           int* blocks_per_sm) {
  TRACE();
  CHECK_REG(reg);
  FLUSH(reg);
  if (U == nullptr || qubits == nullptr) return fail(IQS_EINVAL, "qubits or U is NULL");
  const int kmax = iqs::max_kq(reg->dtype);
  if (k < 1 || k > kmax || k > reg->n) return fail(IQS_EINVAL, "k = %d outside [1, %d] for this register", k, kmax);
  iqs_status s = check_qubit_set(reg, k, qubits);
  if (s != IQS_OK) return s;
  for (int i = 0; i < (2 << (2 * k)); ++i)
    if (!std::isfinite(U[i])) return fail(IQS_EINVAL, "U entry %d is not finite", i / 2);
  double ms = 0.0;
  int v = 0, ps = 0;
  LAUNCH_TRY(iqs::tune_kq(reg, k, qubits, U, &ms, &v, &ps), "kq_autotune");
  if (best_ms) *best_ms = ms;
  if (variant) *variant = v;
  if (blocks_per_sm) *blocks_per_sm = ps;
  return check_flag(reg);
}

iqs_status iqs_kq_set_variant(iqs_reg* reg, int k, const int* qubits, int variant, int blocks_per_sm) {
  TRACE();
  CHECK_REG(reg);
  if (qubits == nullptr) return fail(IQS_EINVAL, "qubits is NULL");
  const int kmax = iqs::max_kq(reg->dtype);
  if (k < 1 || k > kmax || k > reg->n) return fail(IQS_EINVAL, "k = %d outside [1, %d] for this register", k, kmax);
  iqs_status s = check_qubit_set(reg, k, qubits);
  if (s != IQS_OK) return s;
  if (variant < 0 || variant > 4) return fail(IQS_EINVAL, "variant %d outside [0, 4]", variant);
  if (blocks_per_sm < 1 || blocks_per_sm > 64) return fail(IQS_EINVAL, "blocks_per_sm %d outside [1, 64]", blocks_per_sm);
  iqs::set_kq_choice(reg, k, qubits, variant, blocks_per_sm);
  return IQS_OK;
}

iqs_status iqs_marginal(iqs_reg* reg, int k, const int* qubits, double* out) {
  TRACE();
  CHECK_REG(reg);
  FLUSH(reg);
  if (qubits == nullptr || out == nullptr) return fail(IQS_EINVAL, "qubits or out is NULL");
  const int kmax = std::min(reg->n, iqs::max_marginal_qubits());
  if (k < 1 || k > kmax) return fail(IQS_EINVAL, "k = %d outside [1, %d]", k, kmax);
  iqs_status s = check_qubit_set(reg, k, qubits);
  if (s != IQS_OK) return s;
  const size_t outs = (size_t)1 << k;
  const size_t pbytes = iqs::marginal_scratch_bytes(reg, k, qubits);
  DeviceScratch mem(reg->stream);
  if ((s = mem.get(sizeof(double) * outs + pbytes)) != IQS_OK) return s;
  double* out_dev = (double*)mem.ptr;
  double* partials = out_dev + outs;
  LAUNCH_TRY(iqs::launch_marginal(reg, k, qubits, out_dev, partials), "marginal");
  CUDA_TRY(cudaMemcpyAsync(out, out_dev, sizeof(double) * outs, cudaMemcpyDeviceToHost, reg->stream), "copy marginal");
  if ((s = mem.release()) != IQS_OK) return s;
  CUDA_TRY(cudaStreamSynchronize(reg->stream), "synchronise");
  return check_flag(reg);
}

iqs_status iqs_sample(iqs_reg* reg, uint64_t shots, const double* uniforms, uint64_t* out) {
  TRACE();
  CHECK_REG(reg);
  FLUSH(reg);
  if (shots == 0) return IQS_OK;
  if (uniforms == nullptr || out == nullptr) return fail(IQS_EINVAL, "uniforms or out is NULL");
  if (shots > (1ull << 32)) return fail(IQS_EINVAL, "at most 2^32 shots per call");
  for (uint64_t s = 0; s < shots; ++s)
    if (!(uniforms[s] >= 0.0 && uniforms[s] < 1.0)) return fail(IQS_EINVAL, "uniform %llu outside [0, 1)", (unsigned long long)s);
  const size_t sbytes = iqs::sample_scratch_bytes(reg->n);
  DeviceScratch mem(reg->stream);
  iqs_status st = mem.get(sbytes + 16 * (size_t)shots);
  if (st != IQS_OK) return st;
  double* scratch = (double*)mem.ptr;
  double* u_dev = (double*)((char*)mem.ptr + sbytes);
  unsigned long long* out_dev = (unsigned long long*)(u_dev + shots);
  CUDA_TRY(cudaMemcpyAsync(u_dev, uniforms, sizeof(double) * shots, cudaMemcpyHostToDevice, reg->stream), "copy uniforms");
  LAUNCH_TRY(iqs::launch_sample(reg, shots, u_dev, out_dev, scratch), "sample");
  CUDA_TRY(cudaMemcpyAsync(out, out_dev, sizeof(uint64_t) * shots, cudaMemcpyDeviceToHost, reg->stream), "copy samples");
  if ((st = mem.release()) != IQS_OK) return st;
  CUDA_TRY(cudaStreamSynchronize(reg->stream), "synchronise");
  if ((st = check_flag(reg)) != IQS_OK) return st;
  if (out[0] == ~0ull) return fail(IQS_EINVAL, "cannot sample a state of zero weight");
  return IQS_OK;
}

// State files: the 8 bytes "IQSSTATE", then uint32 version (1), n, dtype and
// a zero word, then the 2^n amplitudes as stored (interleaved re, im).
iqs_status iqs_save(iqs_reg* reg, const char* path) {
  TRACE();
  CHECK_REG(reg);
  FLUSH(reg);
  if (path == nullptr) return fail(IQS_EINVAL, "path is NULL");
  FILE* f = std::fopen(path, "wb");
  if (f == nullptr) return fail(IQS_EINVAL, "cannot open %s for writing", path);
  const uint32_t hdr[4] = {1u, (uint32_t)reg->n, (uint32_t)reg->dtype, 0u};
  bool ok = std::fwrite("IQSSTATE", 1, 8, f) == 8 && std::fwrite(hdr, sizeof(hdr), 1, f) == 1;
  const size_t total = iqs::num_amps(reg) * iqs::amp_bytes(reg), step = (size_t)64 << 20;
  void* buf = nullptr;
  if (ok && cudaMallocHost(&buf, std::min(total, step)) != cudaSuccess) {
    cudaGetLastError();
    std::fclose(f);
    return fail(IQS_ENOMEM, "save: no pinned staging buffer");
  }
  for (size_t off = 0; ok && off < total; off += step) {
    const size_t m = std::min(step, total - off);
    ok = cudaMemcpyAsync(buf, (const char*)reg->data + off, m, cudaMemcpyDeviceToHost, reg->stream) == cudaSuccess &&
         cudaStreamSynchronize(reg->stream) == cudaSuccess && std::fwrite(buf, 1, m, f) == m;
  }
  if (buf) cudaFreeHost(buf);
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) return fail(IQS_ECUDA, "save to %s failed", path);
  return IQS_OK;
}

iqs_status iqs_load(iqs_reg* reg, const char* path) {
  TRACE();
  CHECK_REG(reg);
  if (path == nullptr) return fail(IQS_EINVAL, "path is NULL");
  FILE* f = std::fopen(path, "rb");
  if (f == nullptr) return fail(IQS_EINVAL, "cannot open %s", path);
  char magic[8];
  uint32_t hdr[4];
  if (std::fread(magic, 1, 8, f) != 8 || std::memcmp(magic, "IQSSTATE", 8) != 0 || std::fread(hdr, sizeof(hdr), 1, f) != 1 ||
      hdr[0] != 1u) {
    std::fclose(f);
    return fail(IQS_EINVAL, "%s is not a state file", path);
  }
  if ((int)hdr[1] != reg->n || (int)hdr[2] != reg->dtype) {
    std::fclose(f);
    return fail(IQS_EINVAL, "%s holds %u qubits of dtype %u; the register has %d of dtype %d", path, hdr[1], hdr[2],
                reg->n, reg->dtype);
  }
  reg->fmask = 0;  // the state is replaced: queued gates are void
  const size_t total = iqs::num_amps(reg) * iqs::amp_bytes(reg), step = (size_t)64 << 20;
  void* buf = nullptr;
  if (cudaMallocHost(&buf, std::min(total, step)) != cudaSuccess) {
    cudaGetLastError();
    std::fclose(f);
    return fail(IQS_ENOMEM, "load: no pinned staging buffer");
  }
  bool ok = true;
  for (size_t off = 0; ok && off < total; off += step) {
    const size_t m = std::min(step, total - off);
    ok = std::fread(buf, 1, m, f) == m &&
         cudaMemcpyAsync((char*)reg->data + off, buf, m, cudaMemcpyHostToDevice, reg->stream) == cudaSuccess &&
         cudaStreamSynchronize(reg->stream) == cudaSuccess;
  }
  cudaFreeHost(buf);
  std::fclose(f);
  if (!ok) return fail(IQS_EINVAL, "%s is truncated or could not be copied", path);
  return IQS_OK;
}

const char* iqs_last_error(void) { return g_err; }

const char* iqs_version(void) { return "iqs-gb300 0.1.0 (sm_103a)"; }

uint64_t iqs_kernel_launches(void) { return g_launches.load(); }

iqs_status iqs_inject_fault(int kind, int after) {
  TRACE();
  if (kind < 0 || kind > 2 || after < 0) return fail(IQS_EINVAL, "fault kind must be 0, 1 or 2 and after >= 0");
  g_fault_countdown = after;
  g_fault_kind = kind;
  return IQS_OK;
}

}  // extern "C"
