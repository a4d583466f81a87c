// Counting a < b on two 16-bit lanes at once, for lane values below 2^15:
// with the guard bit (bit 15 of each lane) set in a, the difference
// (a | guard) - b lies in [1, 2^16 - 1] in each lane, so no borrow crosses
// the lanes, and its bit 15 is set exactly when a >= b. Three integer
// instructions per pair of lanes (subtract, shift, and-not, add), against
// about five for a packed compare followed by a packed subtract.
#pragma once

#include <stdint.h>

namespace schulze {

constexpr uint32_t kGuard2 = 0x80008000u;  // bit 15 of both 16-bit lanes

// acc's lanes += [a < b] for each lane; a_guarded = a | kGuard2.
__device__ __forceinline__ uint32_t count_lt2(uint32_t acc, uint32_t a_guarded, uint32_t b) {
  return acc + ((~(a_guarded - b) >> 15) & 0x00010001u);
}

}  // namespace schulze
