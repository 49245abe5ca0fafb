// Allocation-free variant of the all-qubit probability reduction
// (iqs_probabilities_noalloc in include/iqs.h).
//
// Some callers cannot call cudaMalloc: a serving process whose allocator owns
// all device memory up front, a real-time loop that forbids allocation after
// start-up, or host code that must not touch the CUDA allocator at all.  They
// can use this entry point with their own state and output buffers: its
// scratch (the per-block partial sums of the reduction and one out-of-range
// flag) lives in a file-scope static device array instead of memory allocated
// per register.
//
// Facts a caller needs:
//   - Scratch size is fixed: kScratchDoubles doubles (about 320 KiB).  Every
//     GPU that loads this library holds that array until the process exits.
//   - The kernel grid is fixed (kRedBlocks blocks), so the scratch bound does
//     not depend on the state size; the accepted state sizes are n in
//     [1, IQS_MAX_QUBITS] qubits, and anything else is rejected with
//     IQS_EINVAL before any work is queued.
//   - Host code cannot use the array's name as a device address.  The first
//     call on each device looks the address up with cudaGetSymbolAddress (with
//     that device current) and caches it; that first call should therefore
//     come before any stream capture on that device.
//   - Every call on a device shares the same array, and the array keeps the
//     last call's contents.  The partial sums are fully rewritten by each call
//     before they are read; the flag, which must start at zero, is cleared at
//     the start of each call.  Calls that overlap on the GPU (different
//     streams, no ordering between them) race on the array and give wrong
//     results; order them on one stream or with events.
//   - No call here allocates: no cudaMalloc, cudaFree or allocating library
//     routine.
#include <cmath>
#include <mutex>

#include "internal.h"

namespace {

using iqs::kRedBlocks;
using iqs::kRedSlots;

// partial sums (kRedBlocks x kRedSlots), then one 8-byte slot for the flag
constexpr size_t kPartialDoubles = (size_t)kRedBlocks * kRedSlots;
constexpr size_t kScratchDoubles = kPartialDoubles + 1;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (looked up once per device).
cudaError_t scratch_address(int dev, double** out) {
  std::lock_guard<std::mutex> lock(g_mutex);
  if (g_addr[dev] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

// An out-of-range complex128 amplitude (|a| >= 2^64, Inf, NaN) turns every output into NaN.
__global__ void k_flag_to_nan(const unsigned* flag, double* out, int n) {
  if (*flag && (int)threadIdx.x < n) out[threadIdx.x] = __longlong_as_double(0x7ff8000000000000ll);
}

}  // namespace

extern "C" iqs_status iqs_probabilities_noalloc(const void* state, int n, int dtype, void* stream, double* out) {
  if (dtype != IQS_C64 && dtype != IQS_C128) return iqs::report(IQS_EINVAL, "dtype must be IQS_C64 or IQS_C128");
  if (n < 1 || n > IQS_MAX_QUBITS)
    return iqs::report(IQS_EINVAL,
                       "n = %d outside [1, %d]: the static scratch of iqs_probabilities_noalloc holds %d x %d "
                       "partial sums, enough for at most %d qubits",
                       n, IQS_MAX_QUBITS, kRedBlocks, kRedSlots, IQS_MAX_QUBITS);
  if (state == nullptr || ((uintptr_t)state & 15u)) return iqs::report(IQS_EINVAL, "state is NULL or not 16-byte aligned");
  if (out == nullptr || ((uintptr_t)out & 7u)) return iqs::report(IQS_EINVAL, "out is NULL or not 8-byte aligned");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return iqs::report(IQS_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return iqs::report(IQS_EINTERNAL, "device %d beyond the %d supported", dev, kMaxDevices);
  double* scratch = nullptr;
  if ((e = scratch_address(dev, &scratch)) != cudaSuccess)
    return iqs::report(IQS_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
  cudaStream_t s = (cudaStream_t)stream;
  unsigned* flag = reinterpret_cast<unsigned*>(scratch + kPartialDoubles);
  if ((e = cudaMemsetAsync(flag, 0, sizeof(unsigned), s)) != cudaSuccess)
    return iqs::report(IQS_ECUDA, "clear flag: %s", cudaGetErrorString(e));
  if ((e = iqs::launch_probabilities_raw(state, n, dtype, s, scratch, out, flag)) != cudaSuccess)
    return iqs::report(IQS_ECUDA, "probabilities_noalloc: %s", cudaGetErrorString(e));
  k_flag_to_nan<<<1, 64, 0, s>>>(flag, out, n);
  if ((e = iqs::launched(1)) != cudaSuccess)
    return iqs::report(IQS_ECUDA, "probabilities_noalloc flag check: %s", cudaGetErrorString(e));
  return IQS_OK;
}
