// Block-wide scan used by the planning kernels (one CTA of up to 1024 threads).
#pragma once

#include <stdint.h>

namespace schulze {

// Scans of up to this many entries run in a dynamic shared-memory buffer
// (208 KB: the launch opts in above the 48 KB default); longer ones in place
// in global memory.
constexpr int32_t kScanSmem = 53248;

// Block-wide exclusive scan of v[0..len) (uint32) in place; returns the total.
// Every thread of the block must call it; part holds >= 32 words. Thread t
// sums a contiguous run of v, the runs are scanned with warp shuffles and
// one pass over the warp totals, then each thread rewrites its run.
__device__ inline uint32_t block_exclusive_scan(uint32_t* v, int32_t len, uint32_t* part) {
  const int T = blockDim.x, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int per = (len + T - 1) / T;
  const int b = min(len, threadIdx.x * per), e = min(len, b + per);
  uint32_t s = 0;
  for (int c = b; c < e; ++c) s += v[c];
  uint32_t x = s;  // inclusive scan within the warp
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) part[wid] = x;
  __syncthreads();
  if (wid == 0) {
    const int nw = T >> 5;
    uint32_t w = lane < nw ? part[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) part[lane] = w;  // inclusive warp totals
  }
  __syncthreads();
  uint32_t run = (wid ? part[wid - 1] : 0u) + x - s;
  for (int c = b; c < e; ++c) {
    const uint32_t y = v[c];
    v[c] = run;
    run += y;
  }
  const uint32_t total = part[(T >> 5) - 1];
  __syncthreads();
  return total;
}

}  // namespace schulze
