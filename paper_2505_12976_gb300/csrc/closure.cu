// Widest paths, all pairs (Sect. 2.1 definition; Sect. 4 "straightforward
// algorithm" computing p(a, b) for every pair), as a blocked Floyd-Warshall
// in the (max, min) semiring.
//
// Edge weights are winning votes, w[i][j] = d[i][j] if d[i][j] > d[j][i]
// else 0, packed into a zero-padded square workspace W (int16 when every
// count fits in 15 bits, else int32). The closure runs on W in rounds of
// B = 64 candidates: round r
//   1. closes the diagonal tile (r, r) by plain Floyd-Warshall,
//   2. updates the row and column panels: X = max(X, A (x) B) with A or B
//      the closed diagonal tile,
//   3. updates every other tile (i, j): X = max(X, W(i, r) (x) W(r, j)),
// where (x) is the (max, min) product. Widths only grow and every value
// written is the width of a real path, so the order of the updates inside a
// phase does not matter and the result is the exact closure.
#include <algorithm>

#include "internal.cuh"

namespace schulze {
namespace {

constexpr int kB = 64;        // block / tile size
constexpr int kThreads = 128; // threads per tile CTA
constexpr int kRM = 8;        // rows per thread
constexpr int kRN = 4;        // columns per thread
constexpr int kTX = kB / kRN; // 16 column groups
// rows: 8 groups of 8 -> 8 * 16 = 128 threads

// ---------------------------------------------------------------- pack

// W[i][j] = d[i][j] if d[i][j] > d[j][i] else 0 (i != j, both < m), 0 elsewhere.
template <typename E>
__global__ void pack_kernel(const int32_t* __restrict__ d, int32_t m, int32_t mp, int64_t bound, E* __restrict__ W,
                            int32_t* status) {
  __shared__ int32_t s[32][33];
  const int32_t bi = blockIdx.y * 32, bj = blockIdx.x * 32;
  // s = d[bj.., bi..] (the transposed block)
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int32_t i = bj + r, j = bi + threadIdx.x;
    s[r][threadIdx.x] = (i < m && j < m) ? d[int64_t(i) * m + j] : 0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int32_t i = bi + r, j = bj + threadIdx.x;
    int32_t out = 0;
    if (i < m && j < m) {
      int32_t a = d[int64_t(i) * m + j];
      int32_t b = s[threadIdx.x][r];  // d[j][i]
      if (a < 0 || int64_t(a) > bound) set_status(status, SCHULZE_EDATA);
      if (i != j && a > b) out = a;
    }
    if (i < mp && j < mp) W[int64_t(i) * mp + j] = E(out);
  }
}

// p[i][j] = W[i][j] for i, j < m (unpadded int32 output).
template <typename E>
__global__ void widen_kernel(const E* __restrict__ W, int32_t mp, int32_t m, int32_t* __restrict__ p) {
  const int64_t total = int64_t(m) * m;
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
    int64_t i = t / m, j = t % m;
    p[t] = i == j ? 0 : int32_t(W[i * mp + j]);
  }
}

// ------------------------------------------------------ tile routines

// Closes the diagonal tile (r, r) in place: plain Floyd-Warshall over its
// 64 vertices, 1024 threads with 4 independent entries each. Row k and
// column k do not change during step k (min(x, y) <= x), so one barrier per
// step suffices. The diagonal of the tile is left at whatever cycle width it
// reaches: it never changes an off-diagonal entry and is zeroed on output.
constexpr int kDiagThreads = 1024;
template <typename E>
__device__ void diag_closure(E* __restrict__ W, int32_t ld, int32_t r, int32_t* __restrict__ s /*[64][65]*/) {
  const int64_t base = int64_t(r) * kB * ld + int64_t(r) * kB;
  for (int t = threadIdx.x; t < kB * kB; t += kDiagThreads) {
    int i = t / kB, j = t % kB;
    s[i * (kB + 1) + j] = int32_t(__ldcg(&W[base + int64_t(i) * ld + j]));
  }
  __syncthreads();
  const int i = threadIdx.x / 16, j0 = threadIdx.x % 16;  // columns j0 + 16 q
  int32_t* row = s + i * (kB + 1);
  for (int k = 0; k < kB; ++k) {
    const int32_t a = row[k];
    const int32_t* rk = s + k * (kB + 1);
    int32_t v[4], b[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      v[q] = row[j0 + 16 * q];
      b[q] = rk[j0 + 16 * q];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) row[j0 + 16 * q] = max(v[q], min(a, b[q]));
    __syncthreads();
  }
  for (int t = threadIdx.x; t < kB * kB; t += kDiagThreads) {
    int ii = t / kB, jj = t % kB;
    __stcg(&W[base + int64_t(ii) * ld + jj], E(s[ii * (kB + 1) + jj]));
  }
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

// X(ti, tj) = max(X, W(ti, r) (x) W(r, tj)), int32 lanes.
__device__ void tile_update_s32(int32_t* __restrict__ W, int32_t ld, int32_t ti, int32_t tj, int32_t r,
                                SmemS32& sm) {
  const int tid = threadIdx.x;
  const int tx = tid % kTX, ty = tid / kTX;
  const int32_t* Ag = W + int64_t(ti) * kB * ld + int64_t(r) * kB;
  const int32_t* Bg = W + int64_t(r) * kB * ld + int64_t(tj) * kB;
  int32_t* Cg = W + int64_t(ti) * kB * ld + int64_t(tj) * kB;
  // A: row i = tid % 64, 32 consecutive k from (tid / 64) * 32
  {
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
  // B: straight copy, 16 int4 per row
  for (int t = tid; t < kB * kB / 4; t += kThreads) {
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
  __syncthreads();
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
#pragma unroll
    for (int rr = 0; rr < kRM; ++rr)
#pragma unroll
      for (int cc = 0; cc < kRN; ++cc)
        acc[rr][cc] = __vimax3_s32(acc[rr][cc], min(a[0][rr], bb[0][cc]), min(a[1][rr], bb[1][cc]));
  }
#pragma unroll
  for (int rr = 0; rr < kRM; ++rr) {
    int4 v = make_int4(acc[rr][0], acc[rr][1], acc[rr][2], acc[rr][3]);
    __stcg(reinterpret_cast<int4*>(Cg + int64_t(ty * kRM + rr) * ld + tx * kRN), v);
  }
  __syncthreads();  // shared operands are reused by the next call
}

// X(ti, tj) = max(X, W(ti, r) (x) W(r, tj)), two 16-bit lanes per word.
__device__ void tile_update_s16(int16_t* __restrict__ W, int32_t ld, int32_t ti, int32_t tj, int32_t r,
                                SmemS16& sm) {
  const int tid = threadIdx.x;
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
  __syncthreads();
  // two k-steps per three-input max: max(c, min(a, b), min(a', b'))
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
#pragma unroll
  for (int rr = 0; rr < kRM; ++rr)
    __stcg(reinterpret_cast<uint2*>(Cg + int64_t(ty * kRM + rr) * ld + tx * kRN), make_uint2(acc[rr][0], acc[rr][1]));
  __syncthreads();
}

template <typename E>
struct Ops;
template <>
struct Ops<int32_t> {
  using Smem = SmemS32;
  static __device__ void update(int32_t* W, int32_t ld, int32_t ti, int32_t tj, int32_t r, Smem& sm) {
    tile_update_s32(W, ld, ti, tj, r, sm);
  }
};
template <>
struct Ops<int16_t> {
  using Smem = SmemS16;
  static __device__ void update(int16_t* W, int32_t ld, int32_t ti, int32_t tj, int32_t r, Smem& sm) {
    tile_update_s16(W, ld, ti, tj, r, sm);
  }
};

// ------------------------------------------------- per-phase kernels

template <typename E>
__global__ void __launch_bounds__(kDiagThreads) phase1_kernel(E* W, int32_t ld, int32_t r) {
  __shared__ int32_t s[kB * (kB + 1)];
  diag_closure<E>(W, ld, r, s);
}

// blockIdx.x < nb - 1: row panel tile (r, j); else column panel tile (i, r).
template <typename E>
__global__ void __launch_bounds__(kThreads) phase2_kernel(E* W, int32_t ld, int32_t r, int32_t nb) {
  __shared__ __align__(16) typename Ops<E>::Smem sm;
  int32_t t = blockIdx.x;
  if (t < nb - 1) {
    int32_t j = t + (t >= r);
    Ops<E>::update(W, ld, r, j, r, sm);
  } else {
    t -= nb - 1;
    int32_t i = t + (t >= r);
    Ops<E>::update(W, ld, i, r, r, sm);
  }
}

template <typename E>
__global__ void __launch_bounds__(kThreads) phase3_kernel(E* W, int32_t ld, int32_t r, int32_t nb) {
  __shared__ __align__(16) typename Ops<E>::Smem sm;
  int32_t t = blockIdx.x;
  int32_t i = t / (nb - 1), j = t % (nb - 1);
  i += (i >= r);
  j += (j >= r);
  Ops<E>::update(W, ld, i, j, r, sm);
}

template <typename E>
int run_closure(schulze_ctx* ctx, const int32_t* d, int32_t m, int64_t bound, int32_t* p, void* ws,
                cudaStream_t stream) {
  const int32_t mp = int32_t(align_up(size_t(m), kB));
  const int32_t nb = mp / kB;
  E* W = static_cast<E*>(ws);
  const double mm = double(m) * double(m);
  const double tile3 = double(kB) * kB * kB;
  {
    Launch L(ctx, stream, "closure_pack", mm * (8.0 + sizeof(E)));
    dim3 g(mp / 32, mp / 32), b(32, 8);
    pack_kernel<E><<<g, b, 0, stream>>>(d, m, mp, bound, W, ctx->status);
  }
  for (int32_t r = 0; r < nb; ++r) {
    {
      Launch L(ctx, stream, "closure_diag", tile3);
      phase1_kernel<E><<<1, kDiagThreads, 0, stream>>>(W, mp, r);
    }
    if (nb > 1) {
      {
        Launch L(ctx, stream, "closure_panels", 2.0 * (nb - 1) * tile3);
        phase2_kernel<E><<<2 * (nb - 1), kThreads, 0, stream>>>(W, mp, r, nb);
      }
      {
        Launch L(ctx, stream, "closure_tiles", double(nb - 1) * (nb - 1) * tile3);
        phase3_kernel<E><<<(nb - 1) * (nb - 1), kThreads, 0, stream>>>(W, mp, r, nb);
      }
    }
  }
  {
    Launch L(ctx, stream, "closure_widen", mm * (4.0 + sizeof(E)));
    int sms = ctx->sm_count > 0 ? ctx->sm_count : 148;
    int64_t total = int64_t(m) * m;
    int blocks = int(std::min<int64_t>((total + 255) / 256, int64_t(sms) * 32));
    widen_kernel<E><<<blocks, 256, 0, stream>>>(W, mp, m, p);
  }
  return check_launch();
}

}  // namespace

size_t closure_workspace_bytes(int32_t m, int64_t bound, uint32_t flags) {
  size_t mp = align_up(size_t(m), kB);
  return mp * mp * (use_s16(bound, flags) ? 2 : 4) + 4096;
}

int closure_launch(schulze_ctx* ctx, const int32_t* d, int32_t m, int64_t bound, int32_t* p, uint32_t flags,
                   void* ws, cudaStream_t stream) {
  if (use_s16(bound, flags)) return run_closure<int16_t>(ctx, d, m, bound, p, ws, stream);
  return run_closure<int32_t>(ctx, d, m, bound, p, ws, stream);
}

}  // namespace schulze
