// (max, min) tile routines shared by the single-election closure and the
// batched elections: the diagonal-tile Floyd-Warshall and the 64 x 64 x 64
// tile update X = max(X, A (x) B). Each runs on a group of 128 threads that
// synchronise through `Bar`: the whole block, or one named barrier per group
// when a block runs several groups side by side.
#pragma once

#include <type_traits>

#include "internal.cuh"

namespace schulze {
namespace tiles {

constexpr int kB = 64;         // block / tile size
constexpr int kThreads = 128;  // threads of one tile group
constexpr int kRM = 8;         // rows per thread in a tile update
constexpr int kRN = 4;         // columns per thread in a tile update
constexpr int kTX = kB / kRN;  // 16 column groups x 8 row groups = 128 threads

// All threads of the block.
struct BlockBarrier {
  __device__ __forceinline__ void sync() const { __syncthreads(); }
  __device__ __forceinline__ bool sync_or(bool p) const { return __syncthreads_or(p) != 0; }
};

// Named barrier `id` (1..15) over the 128 threads of one group.
struct GroupBarrier {
  int id;
  __device__ __forceinline__ void sync() const { asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory"); }
  __device__ __forceinline__ bool sync_or(bool p) const {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred pi, po;\n\tsetp.ne.u32 pi, %1, 0;\n\t"
        "bar.red.or.pred po, %2, 128, pi;\n\tselp.u32 %0, 1, 0, po;\n\t}"
        : "=r"(r)
        : "r"(uint32_t(p)), "r"(id)
        : "memory");
    return r != 0;
  }
};

// Closes the diagonal tile (r, r) in place by plain Floyd-Warshall over its
// 64 vertices. Thread t keeps row t / 2, columns 32 (t % 2) .. + 31 in
// registers; at step k the two owners of row k publish it through shared
// memory and p[i][k] comes from the thread itself or its neighbour lane.
// Row k and column k do not change during step k (min(x, y) <= x). The
// tile's diagonal may pick up cycle widths; it never changes an off-diagonal
// entry and is zeroed on output. Returns whether the tile holds a nonzero.
template <typename E, class Bar>
__device__ bool diag_closure_local(E* __restrict__ W, int32_t ld, int32_t r, int32_t (*rowbuf)[kB], int tid,
                                   const Bar& bar) {
  const int i = tid >> 1, half = tid & 1;
  E* base = W + (int64_t(r) * kB + i) * ld + int64_t(r) * kB + half * 32;
  int32_t v[32];
  if (sizeof(E) == 2) {
    const uint4* src = reinterpret_cast<const uint4*>(base);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint4 x = __ldcg(src + q);
      const uint32_t w4[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        v[8 * q + 2 * h] = int32_t(int16_t(w4[h] & 0xFFFFu));
        v[8 * q + 2 * h + 1] = int32_t(int16_t(w4[h] >> 16));
      }
    }
  } else {
    const int4* src = reinterpret_cast<const int4*>(base);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      int4 x = __ldcg(src + q);
      v[4 * q] = x.x, v[4 * q + 1] = x.y, v[4 * q + 2] = x.z, v[4 * q + 3] = x.w;
    }
  }
#pragma unroll
  for (int k = 0; k < kB; ++k) {
    int32_t* rb = rowbuf[k & 1];
    if (i == k) {
#pragma unroll
      for (int c = 0; c < 32; c += 4)
        *reinterpret_cast<int4*>(&rb[half * 32 + c]) = make_int4(v[c], v[c + 1], v[c + 2], v[c + 3]);
    }
    bar.sync();
    const int32_t mine = v[k & 31];
    const int32_t other = __shfl_xor_sync(0xFFFFFFFFu, mine, 1);
    const int32_t a = ((k >> 5) == half) ? mine : other;  // p[i][k]
#pragma unroll
    for (int c = 0; c < 32; c += 4) {
      int4 b = *reinterpret_cast<const int4*>(&rb[half * 32 + c]);
      v[c] = max(v[c], min(a, b.x));
      v[c + 1] = max(v[c + 1], min(a, b.y));
      v[c + 2] = max(v[c + 2], min(a, b.z));
      v[c + 3] = max(v[c + 3], min(a, b.w));
    }
  }
  int32_t any = 0;
  if (sizeof(E) == 2) {
    uint4* dst = reinterpret_cast<uint4*>(base);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint32_t w4[4];
#pragma unroll
      for (int h = 0; h < 4; ++h)
        w4[h] = (uint32_t(v[8 * q + 2 * h]) & 0xFFFFu) | (uint32_t(v[8 * q + 2 * h + 1]) << 16);
      __stcg(dst + q, make_uint4(w4[0], w4[1], w4[2], w4[3]));
      any |= int32_t(w4[0] | w4[1] | w4[2] | w4[3]);
    }
  } else {
    int4* dst = reinterpret_cast<int4*>(base);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      __stcg(dst + q, make_int4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]));
      any |= v[4 * q] | v[4 * q + 1] | v[4 * q + 2] | v[4 * q + 3];
    }
  }
  return any != 0;
}

// The closure above, then one barrier that also reports whether the tile
// holds a nonzero anywhere. The _local form leaves that barrier to the
// caller (it returns this thread's part of the answer).
template <typename E, class Bar>
__device__ bool diag_closure(E* __restrict__ W, int32_t ld, int32_t r, int32_t (*rowbuf)[kB], int tid,
                             const Bar& bar) {
  return bar.sync_or(diag_closure_local<E>(W, ld, r, rowbuf, tid, bar));
}

// Shared-memory operand layouts of one tile update.
struct SmemS32 {
  int32_t A[kB][kB];  // A[k][i] = W(ti, r)[i][k] (transposed)
  int32_t B[kB][kB];  // B[k][j] = W(r, tj)[k][j]
};
struct SmemS16 {
  uint32_t A[kB][kB];  // A[k][i] = W(ti, r)[i][k] in both 16-bit halves
  uint16_t B[kB][kB];  // B[k][j]
};

// Which min/max unit an int32 update of the micro-tile runs on (kMix):
// 0 all integer; 1 every second entry on the fp32 unit; 2 the mins on the
// fp32 unit and the three-input max on the integer unit; 3 a third of the
// entries integer, the rest fp32; 4 two thirds integer. The fp32 forms read
// the same bits (fmin_bits): exact for every count below 0x7F800000.
#ifndef SCHULZE_S32_MIX
#define SCHULZE_S32_MIX 0
#endif
constexpr int kS32Mix = SCHULZE_S32_MIX;

template <int kMix, int kE>
__device__ __forceinline__ int32_t update2_s32(int32_t c, int32_t a0, int32_t b0, int32_t a1, int32_t b1) {
  const uint32_t uc = uint32_t(c), ua0 = uint32_t(a0), ub0 = uint32_t(b0), ua1 = uint32_t(a1), ub1 = uint32_t(b1);
  constexpr bool kInt = kMix == 0 || (kMix == 1 && (kE & 1) == 0) || (kMix == 3 && kE % 3 == 0) ||
                        (kMix == 4 && kE % 3 != 0);
  if (kMix == 2) return int32_t(imax3_bits(uc, fmin_bits(ua0, ub0), fmin_bits(ua1, ub1)));
  if (kInt) return __vimax3_s32(c, min(a0, b0), min(a1, b1));
  return int32_t(fmax3_bits(uc, fmin_bits(ua0, ub0), fmin_bits(ua1, ub1)));
}

// X(ti, tj) = max(X, W(ti, r) (x) W(r, tj)), int32 lanes. Returns whether
// the updated tile holds a nonzero. kMix: see update2_s32 (0 whenever a
// count may reach 0x7F800000).
template <int kMix, class Bar>
__device__ bool tile_update_s32_local(int32_t* __restrict__ W, int32_t ld, int32_t ti, int32_t tj, int32_t r,
                                      SmemS32& sm, int tid, const Bar& bar) {
  const int tx = tid % kTX, ty = tid / kTX;
  const int32_t* Ag = W + int64_t(ti) * kB * ld + int64_t(r) * kB;
  const int32_t* Bg = W + int64_t(r) * kB * ld + int64_t(tj) * kB;
  int32_t* Cg = W + int64_t(ti) * kB * ld + int64_t(tj) * kB;
  {  // A: row i = tid % 64, 32 consecutive k from (tid / 64) * 32
    const int i = tid % kB, k0 = (tid / kB) * 32;
    const int4* src = reinterpret_cast<const int4*>(Ag + int64_t(i) * ld + k0);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      int4 v = __ldcg(src + q);
      sm.A[k0 + 4 * q + 0][i] = v.x;
      sm.A[k0 + 4 * q + 1][i] = v.y;
      sm.A[k0 + 4 * q + 2][i] = v.z;
      sm.A[k0 + 4 * q + 3][i] = v.w;
    }
  }
  for (int t = tid; t < kB * kB / 4; t += kThreads) {  // B: straight copy
    int k = t / 16, c4 = t % 16;
    int4 v = __ldcg(reinterpret_cast<const int4*>(Bg + int64_t(k) * ld) + c4);
    *reinterpret_cast<int4*>(&sm.B[k][c4 * 4]) = v;
  }
  int32_t acc[kRM][kRN];
#pragma unroll
  for (int rr = 0; rr < kRM; ++rr) {
    int4 v = __ldcg(reinterpret_cast<const int4*>(Cg + int64_t(ty * kRM + rr) * ld + tx * kRN));
    acc[rr][0] = v.x, acc[rr][1] = v.y, acc[rr][2] = v.z, acc[rr][3] = v.w;
  }
  bar.sync();
  // two k-steps per three-input max: max(c, min(a, b), min(a', b'))
#pragma unroll 2
  for (int k = 0; k < kB; k += 2) {
    int32_t a[2][8], bb[2][4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      int4 a0 = *reinterpret_cast<const int4*>(&sm.A[k + h][ty * kRM]);
      int4 a1 = *reinterpret_cast<const int4*>(&sm.A[k + h][ty * kRM + 4]);
      int4 b = *reinterpret_cast<const int4*>(&sm.B[k + h][tx * kRN]);
      a[h][0] = a0.x, a[h][1] = a0.y, a[h][2] = a0.z, a[h][3] = a0.w;
      a[h][4] = a1.x, a[h][5] = a1.y, a[h][6] = a1.z, a[h][7] = a1.w;
      bb[h][0] = b.x, bb[h][1] = b.y, bb[h][2] = b.z, bb[h][3] = b.w;
    }
    auto row = [&](auto rrc) {
      constexpr int rr = decltype(rrc)::value;
      acc[rr][0] = update2_s32<kMix, rr * kRN + 0>(acc[rr][0], a[0][rr], bb[0][0], a[1][rr], bb[1][0]);
      acc[rr][1] = update2_s32<kMix, rr * kRN + 1>(acc[rr][1], a[0][rr], bb[0][1], a[1][rr], bb[1][1]);
      acc[rr][2] = update2_s32<kMix, rr * kRN + 2>(acc[rr][2], a[0][rr], bb[0][2], a[1][rr], bb[1][2]);
      acc[rr][3] = update2_s32<kMix, rr * kRN + 3>(acc[rr][3], a[0][rr], bb[0][3], a[1][rr], bb[1][3]);
    };
    static_assert(kRM == 8 && kRN == 4, "micro-tile shape");
    row(std::integral_constant<int, 0>{}), row(std::integral_constant<int, 1>{});
    row(std::integral_constant<int, 2>{}), row(std::integral_constant<int, 3>{});
    row(std::integral_constant<int, 4>{}), row(std::integral_constant<int, 5>{});
    row(std::integral_constant<int, 6>{}), row(std::integral_constant<int, 7>{});
  }
  int32_t any = 0;
#pragma unroll
  for (int rr = 0; rr < kRM; ++rr) {
    int4 v = make_int4(acc[rr][0], acc[rr][1], acc[rr][2], acc[rr][3]);
    __stcg(reinterpret_cast<int4*>(Cg + int64_t(ty * kRM + rr) * ld + tx * kRN), v);
    any |= v.x | v.y | v.z | v.w;
  }
  return any != 0;  // the caller's barrier also frees the shared operands
}

// X(ti, tj) = max(X, W(ti, r) (x) W(r, tj)), two 16-bit lanes per word.
template <class Bar>
__device__ bool tile_update_s16_local(int16_t* __restrict__ W, int32_t ld, int32_t ti, int32_t tj, int32_t r,
                                      SmemS16& sm, int tid, const Bar& bar) {
  const int tx = tid % kTX, ty = tid / kTX;
  const int16_t* Ag = W + int64_t(ti) * kB * ld + int64_t(r) * kB;
  const int16_t* Bg = W + int64_t(r) * kB * ld + int64_t(tj) * kB;
  int16_t* Cg = W + int64_t(ti) * kB * ld + int64_t(tj) * kB;
  {
    const int i = tid % kB, k0 = (tid / kB) * 32;
    const uint4* src = reinterpret_cast<const uint4*>(Ag + int64_t(i) * ld + k0);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint4 v = __ldcg(src + q);
      const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        uint32_t lo = w4[h] & 0xFFFFu, hi = w4[h] >> 16;
        sm.A[k0 + 8 * q + 2 * h][i] = lo | (lo << 16);
        sm.A[k0 + 8 * q + 2 * h + 1][i] = hi | (hi << 16);
      }
    }
  }
  for (int t = tid; t < kB * kB / 8; t += kThreads) {
    int k = t / 8, c8 = t % 8;
    uint4 v = __ldcg(reinterpret_cast<const uint4*>(Bg + int64_t(k) * ld) + c8);
    *reinterpret_cast<uint4*>(&sm.B[k][c8 * 8]) = v;
  }
  uint32_t acc[kRM][kRN / 2];
#pragma unroll
  for (int rr = 0; rr < kRM; ++rr) {
    uint2 v = __ldcg(reinterpret_cast<const uint2*>(Cg + int64_t(ty * kRM + rr) * ld + tx * kRN));
    acc[rr][0] = v.x, acc[rr][1] = v.y;
  }
  bar.sync();
#pragma unroll 2
  for (int k = 0; k < kB; k += 2) {
    uint32_t a[2][8], b[2][2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      uint4 a0 = *reinterpret_cast<const uint4*>(&sm.A[k + h][ty * kRM]);
      uint4 a1 = *reinterpret_cast<const uint4*>(&sm.A[k + h][ty * kRM + 4]);
      uint2 bv = *reinterpret_cast<const uint2*>(&sm.B[k + h][tx * kRN]);
      a[h][0] = a0.x, a[h][1] = a0.y, a[h][2] = a0.z, a[h][3] = a0.w;
      a[h][4] = a1.x, a[h][5] = a1.y, a[h][6] = a1.z, a[h][7] = a1.w;
      b[h][0] = bv.x, b[h][1] = bv.y;
    }
#pragma unroll
    for (int rr = 0; rr < kRM; ++rr)
#pragma unroll
      for (int w = 0; w < 2; ++w)
        acc[rr][w] = __vimax3_s16x2(acc[rr][w], __vmins2(a[0][rr], b[0][w]), __vmins2(a[1][rr], b[1][w]));
  }
  uint32_t any = 0;
#pragma unroll
  for (int rr = 0; rr < kRM; ++rr) {
    __stcg(reinterpret_cast<uint2*>(Cg + int64_t(ty * kRM + rr) * ld + tx * kRN), make_uint2(acc[rr][0], acc[rr][1]));
    any |= acc[rr][0] | acc[rr][1];
  }
  return any != 0u;
}

// Tile update by lane format; kMix (int32 only) as for tile_update_s32_local.
// update() ends with the barrier that also reports whether the updated tile
// holds a nonzero (and frees the shared operands); update_local() leaves
// that barrier to the caller and returns this thread's part of the answer.
template <typename E, int kMix = 0>
struct Ops;
template <int kMix>
struct Ops<int32_t, kMix> {
  using Smem = SmemS32;
  template <class Bar>
  static __device__ bool update_local(int32_t* W, int32_t ld, int32_t ti, int32_t tj, int32_t r, Smem& sm, int tid,
                                      const Bar& bar) {
    return tile_update_s32_local<kMix>(W, ld, ti, tj, r, sm, tid, bar);
  }
  template <class Bar>
  static __device__ bool update(int32_t* W, int32_t ld, int32_t ti, int32_t tj, int32_t r, Smem& sm, int tid,
                                const Bar& bar) {
    return bar.sync_or(update_local(W, ld, ti, tj, r, sm, tid, bar));
  }
};
template <int kMix>
struct Ops<int16_t, kMix> {
  using Smem = SmemS16;
  template <class Bar>
  static __device__ bool update_local(int16_t* W, int32_t ld, int32_t ti, int32_t tj, int32_t r, Smem& sm, int tid,
                                      const Bar& bar) {
    return tile_update_s16_local(W, ld, ti, tj, r, sm, tid, bar);
  }
  template <class Bar>
  static __device__ bool update(int16_t* W, int32_t ld, int32_t ti, int32_t tj, int32_t r, Smem& sm, int tid,
                                const Bar& bar) {
    return bar.sync_or(update_local(W, ld, ti, tj, r, sm, tid, bar));
  }
};

}  // namespace tiles
}  // namespace schulze
