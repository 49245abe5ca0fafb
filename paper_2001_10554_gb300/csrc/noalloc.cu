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
//     that device current) and caches it, together with the unique id of the
//     CUDA context it belongs to; that first call should therefore come before
//     any stream capture on that device.  A later call whose current context
//     has another id (the context was destroyed and created again, e.g. by
//     cudaDeviceReset) looks the address up again instead of using a stale
//     one; the first call after such a reset should again precede any capture.
//   - Every call on a device shares the same array, and the array keeps the
//     last call's contents.  The partial sums are fully rewritten by each call
//     before they are read; the flag, which must start at zero, is cleared at
//     the start of each call.  Calls that overlap on the GPU (different
//     streams, no ordering between them) race on the array and give wrong
//     results; order them on one stream or with events.
//   - No call here allocates: no cudaMalloc, cudaFree or allocating library
//     routine.
#include <cuda.h>  // CUcontext and CUresult types; driver functions are resolved through the runtime

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

struct ScratchAddress {
  double* addr = nullptr;
  bool ctx_known = false;       // whether ctx_id identifies the context addr belongs to
  unsigned long long ctx_id = 0;
};
ScratchAddress g_addr[kMaxDevices];

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// Unique id (for the life of the process) of the calling thread's current
// context; false when there is none yet or the driver cannot tell.
bool current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult r;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &r) == cudaSuccess &&
        r == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &r) == cudaSuccess &&
        r == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(p);
  });
  if (get_current == nullptr || get_id == nullptr) return false;
  CUcontext c = nullptr;
  if (get_current(&c) != CUDA_SUCCESS || c == nullptr) return false;
  return get_id(c, id) == CUDA_SUCCESS;
}

// Device address of g_noalloc_scratch in the current context of device
// ``dev``: cached per device and looked up again when the context changed
// (or cannot be identified).
cudaError_t scratch_address(int dev, double** out) {
  std::lock_guard<std::mutex> lock(g_mutex);
  ScratchAddress& c = g_addr[dev];
  unsigned long long id = 0;
  if (c.addr != nullptr && c.ctx_known && current_context_id(&id) && id == c.ctx_id) {
    *out = c.addr;
    return cudaSuccess;
  }
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  c.addr = static_cast<double*>(p);  // the lookup has made the device's context current
  c.ctx_known = current_context_id(&c.ctx_id);
  *out = c.addr;
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
