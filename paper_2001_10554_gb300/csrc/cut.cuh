// Max-Cut cut count C(x) = sum_{(u,v) in E} (x_u XOR x_v) (Section 4: H_MaxCut
// counts the edges cut by the bipartition x).
#pragma once

#include <cstdint>

namespace iqs {

// Edge list as kernel parameter (at most 255 edges per launch; longer lists
// are applied in chunks): vertex indices fit in a byte (n <= 34).
constexpr int kEdgeChunk = 255;
struct EdgesU8 {
  int m;  // number of edges, <= kEdgeChunk
  uint8_t u[kEdgeChunk + 1];
  uint8_t v[kEdgeChunk + 1];
};

// Unweighted cut count of basis state x.  Every lane reads the same edge at
// the same time, so the parameter-bank loads broadcast.
template <class X>
__device__ __forceinline__ int cut_count(X x, const EdgesU8& E) {
  int c = 0;
#pragma unroll 4
  for (int e = 0; e < E.m; ++e) c += (int)(((x >> E.u[e]) ^ (x >> E.v[e])) & 1);
  return c;
}

}  // namespace iqs
