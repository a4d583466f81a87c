// Block-wide scan used by the planning kernels (one CTA of up to 1024 threads).
#pragma once

#include <stdint.h>

namespace schulze {

// Scans of up to this many entries run in a dynamic shared-memory buffer
// (208 KB: the launch opts in above the 48 KB default); longer ones in place
// in global memory.
constexpr int32_t kScanSmem = 53248;

// Block-wide exclusive scan of v[0..len) (uint32) in place; returns the total.
// Every thread of the block must call it; part holds >= 33 words. Warp w
// owns the contiguous segment [w * seg, (w + 1) * seg): its lanes read 32
// consecutive words at a time (no shared-memory bank conflicts), a first
// pass sums the segment, one warp scans the segment totals, and a second
// pass scans each run of 32 with warp shuffles, carrying the running sum.
__device__ inline uint32_t block_exclusive_scan(uint32_t* v, int32_t len, uint32_t* part) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int32_t seg = (len + nw - 1) / nw;
  const int32_t b = min(len, wid * seg), e = min(len, b + seg);
  uint32_t s = 0;
  for (int32_t c = b + lane; c < e; c += 32) s += v[c];
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
  if (lane == 0) part[wid] = s;
  __syncthreads();
  if (wid == 0) {
    const uint32_t x = lane < nw ? part[lane] : 0u;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane < nw) part[lane] = inc - x;  // exclusive prefix of each segment
    if (lane == 31) part[32] = inc;        // the total
  }
  __syncthreads();
  uint32_t carry = part[wid];
  for (int32_t c0 = b; c0 < e; c0 += 32) {
    const int32_t c = c0 + lane;
    const uint32_t x = c < e ? v[c] : 0u;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
      if (lane >= o) inc += y;
    }
    if (c < e) v[c] = carry + inc - x;
    carry += __shfl_sync(0xFFFFFFFFu, inc, 31);
  }
  const uint32_t total = part[32];
  __syncthreads();
  return total;
}

}  // namespace schulze
