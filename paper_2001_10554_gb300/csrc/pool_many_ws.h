// The multi-circuit pool workspace (iqs_pool_many in include/iqs.h), shared
// by the brick-circuit engines (pool_many.cu) and the gate-list engine
// (pool_ops.cu).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "iqs.h"

struct iqs_pool_many {
  int dtype = IQS_C64;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  uint64_t timeout_ns = 2000000000ull;  // 2 s per wait
  int debug_never = 0;
  // device buffers (grown on demand)
  void* arena = nullptr;
  size_t arena_bytes = 0;
  void* blob = nullptr;  // params, tables, jobs, counters, partials, outputs
  size_t blob_bytes = 0;
  int engine = 0;         // 0 auto (cluster-resident for complex64 when every state fits), 1 persistent, 2 cluster
  void* mats = nullptr;   // fused matrices of the cluster-resident path
  size_t mats_bytes = 0;
  void* ops_buf = nullptr;  // gate-list engine: programs, matrices, states, results (one buffer, grown)
  size_t ops_bytes = 0;
};
