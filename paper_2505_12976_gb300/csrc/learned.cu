// Learned winner proposal with exact certification.
//
// The paper has no learned component; this is an engineering addition that
// keeps the Schulze winners exact. A small MLP scores candidates from 16
// features of the tally (some of them quantities the paper uses: Copeland
// wins and losses of the dominance relation, Sect. 2.1, and the loser filter
// of Sect. 4). The best-scored candidates are then CERTIFIED with the
// definitions of Sect. 2.1: c is a winner iff p(c, j) >= p(j, c) for all j,
// with p(c, .) and p(., c) computed by single-source / single-sink widest
// paths (the deterministic form of the wide-path questions of Sect. 3). If
// no proposal certifies, the full closure decides.
//
// Structure used by certification: a candidate without outgoing edges
// ("cold") ends every path it is on, so widest paths between the others
// ("warm") only go through warm candidates, p(cold, .) = 0, and a cold
// candidate is a winner iff it has no incoming edge either.
#include <math.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "internal.cuh"

namespace schulze {
namespace {

constexpr int kNF = 16;  // features per candidate
constexpr int kH = 64;   // hidden width
constexpr int kNP = 5313;
constexpr int kOffW1 = 0, kOffB1 = 1024, kOffW2 = 1088, kOffB2 = 5184, kOffW3 = 5248, kOffB3 = 5312;
constexpr int32_t kCertifyMaxWarm = 2048;  // larger warm sets go straight to the closure
constexpr int kMaxProposals = 8;
constexpr int kMaxTies = 16;

// ------------------------------------------------------------ features

struct Acc {  // per-candidate accumulators of the features pass
  int32_t* wins;
  int32_t* losses;
  unsigned long long* rowsum;
  unsigned long long* colsum;
  int32_t* maxw_out;
  int32_t* maxw_in;
  unsigned long long* sumw_out;
  unsigned long long* sumw_in;
  int32_t* min_margin;
  int32_t* max_margin;
  int32_t* max_drow;
};

// The accumulators of the features pass and the rank counters (one launch
// instead of a kernel and two memsets).
__global__ void acc_init_kernel(Acc a, int32_t m, int32_t* __restrict__ cnt14, int32_t* __restrict__ cnt15) {
  for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) {
    cnt14[c] = cnt15[c] = 0;
    a.wins[c] = a.losses[c] = 0;
    a.rowsum[c] = a.colsum[c] = a.sumw_out[c] = a.sumw_in[c] = 0ull;
    a.maxw_out[c] = a.maxw_in[c] = a.max_drow[c] = 0;
    a.min_margin[c] = INT32_MAX;
    a.max_margin[c] = INT32_MIN;
  }
}

__device__ __forceinline__ int32_t warp_max(int32_t v) {
  for (int o = 16; o; o >>= 1) v = max(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
  return v;
}

// Row statistics without per-tile atomics: a CTA takes a strip of kFR rows
// 32 s .. 32 s + 31 against the columns of one chunk (kFChunks chunks, in
// the order of features_cta), tile by tile (kFC columns): d[i][j] and the
// transposed d[j][i] copied into shared memory with cp.async, kFStages - 1
// tiles in flight while one is counted. Thread t takes row t / 8 and the
// columns 32 s + 4 (t % 8) .. +3 of every 32-column slab s of each tile
// (16-byte reads of the row tile, one word of the transposed tile per
// column; both free of bank conflicts), keeping its statistics in
// registers, its sums as partials over a tile (entries of d are counts in
// [0, n]) added into 64-bit totals after each tile. The eight threads of a row combine them with
// shuffles at the end and one adds them to the candidate's accumulators
// (ties follow from wins and losses). Tiles holding no diagonal entry and
// no padding skip the per-entry checks. Every entry is read twice (as d[i][j]
// for row i and as d[i][j] for row j's column).
#ifndef SCHULZE_FEAT_SLABS
#define SCHULZE_FEAT_SLABS 4
#endif
// 32-column slabs per tile (even): four, with two stages, measured 3% faster
// for the whole features call than two slabs with three stages (m = 8192)
constexpr int kFSlabs = SCHULZE_FEAT_SLABS;
constexpr int kFR = 32, kFC = 32 * kFSlabs, kFChunks = 8;
constexpr int kFXL = kFC + 4;  // row tile stride: 16-byte aligned rows
constexpr int kFYL = kFR + 1;  // transposed tile stride

__device__ __forceinline__ void cp_async4(int32_t* dst, const int32_t* src, bool ok) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(src), "r"(ok ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async16(int32_t* dst, const int32_t* src, bool ok) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(src), "r"(ok ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Tiles in flight per CTA: kFStages buffers of both tiles in dynamic shared
// memory, kFStages - 1 tiles copied ahead of the one being counted.
#ifndef SCHULZE_FEAT_STAGES
#define SCHULZE_FEAT_STAGES 2
#endif
constexpr int kFStages = SCHULZE_FEAT_STAGES;
constexpr int kFStageWords = kFR * kFXL + kFC * kFYL;
constexpr size_t kFSmem = size_t(kFStages) * kFStageWords * 4;
constexpr int kFMinBlocks = int((227 * 1024) / (kFSmem + 1024)) < 4 ? int((227 * 1024) / (kFSmem + 1024)) : 4;

// The CTA's (strip, chunk) from its place in the launch: strips are grouped
// by the chunk that holds their rows as columns (S strips a group), and
// the CTAs of (row group g, chunk c) follow right after those of (c, g), so
// that the transposed tiles one set reads were just read by the other and
// are still in L2.
__device__ void features_cta(int32_t nstrips, int32_t S, int32_t* strip, int32_t* chunk) {
  int32_t L = blockIdx.x;
  for (int32_t g = 0; g < kFChunks; ++g)
    for (int32_t c = g; c < kFChunks; ++c)
      for (int side = 0; side < (c == g ? 1 : 2); ++side) {
        const int32_t rg = side ? c : g, ch = side ? g : c;
        const int32_t cnt = max(0, min(S, nstrips - rg * S));
        if (L < cnt) {
          *strip = rg * S + L, *chunk = ch;
          return;
        }
        L -= cnt;
      }
  *strip = nstrips, *chunk = 0;  // not reached: the grid has nstrips * kFChunks CTAs
}

__device__ __forceinline__ uint32_t prmt(uint32_t x, uint32_t y, uint32_t sel) {
  uint32_t r;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(x), "r"(y), "r"(sel));
  return r;
}

// Feature statistics modes, by the ballot count n (entries of d lie in [0, n]):
// kFPacked (n <= 32766): tiles without diagonal entries or padding are
//   counted two entries per instruction, as 16-bit lanes. With a guard bit
//   set in each lane, (a | G) - b holds 2^15 + a - b per lane without a
//   borrow across lanes (a, b < 2^15): its bit 15 is set iff a >= b, and the
//   biased margins keep their order for unsigned 16-bit min / max. Masks of
//   the guard bits count wins and losses, and lane sums (two-lane dot
//   products with weights 1, 1) add entries and masked entries into 32-bit
//   partials; a mask widened from a lane's sign bit (prmt) selects the
//   winning edges. Biased lanes lie in [2, 2^16 - 2], so the initial values
//   2^16 - 1 (minimum) and 0 (maximum) mark "no entry".
// kFNarrow (4 kFSlabs n < 2^32): 32-bit partial sums per tile (4 kFSlabs
//   entries a thread), one entry at a time.
// kFWide: 64-bit sums per entry (a tile's entries could overflow a 32-bit
//   partial).
// kVec: rows of d start on 16-byte boundaries (m % 4 == 0, d aligned), so
// the copies move four entries at a time.
constexpr int kFPacked = 0, kFNarrow = 1, kFWide = 2;

template <bool kVec, int kMode>
__global__ void __launch_bounds__(256, kFMinBlocks) features_pass_kernel(const int32_t* __restrict__ d, int32_t m, Acc a) {
  using Part = typename std::conditional<kMode == kFWide, unsigned long long, uint32_t>::type;
  extern __shared__ __align__(16) int32_t fsm[];
  // stage b: x = d[i][j] (kFR rows of kFXL), then y = d[j][i] (kFC rows: of
  // kFYL words, or with kVec of 32 words whose 16-byte quads are permuted by
  // the row, so that both the 16-byte copies and the column reads below
  // avoid bank conflicts)
  auto X = [&](int b) { return reinterpret_cast<int32_t(*)[kFXL]>(fsm + b * kFStageWords); };
  auto Yp = [&](int b) { return fsm + b * kFStageWords + kFR * kFXL; };
  auto yat = [&](int b, int c, int rr) -> int32_t* {  // &y[c][rr]
    return kVec ? Yp(b) + c * 32 + ((((rr >> 2) ^ ((c >> 2) & 7)) << 2) | (rr & 3)) : Yp(b) + c * kFYL + rr;
  };
  __shared__ int32_t s_place[2];
  const int32_t ntile = (m + kFC - 1) / kFC, per = (ntile + kFChunks - 1) / kFChunks;
  if (threadIdx.x == 0) features_cta((m + kFR - 1) / kFR, per * (kFC / kFR), &s_place[0], &s_place[1]);
  __syncthreads();
  const int32_t I = s_place[0] * kFR;
  const int32_t t0 = s_place[1] * per, t1 = min(ntile, t0 + per);
  if (I >= m || t0 >= t1) return;
  const int r = threadIdx.x >> 3, q = threadIdx.x & 7;
  const int32_t i = I + r;
  int32_t win = 0, loss = 0, mx_wo = 0, mx_wi = 0, mx_d = 0, mn_mg = INT32_MAX, mx_mg = INT32_MIN;
  unsigned long long s_row = 0, s_col = 0, s_wo = 0, s_wi = 0;
  auto issue = [&](int32_t J, int b) {
    if (kVec) {
#pragma unroll
      for (int u = 0; u < kFR * kFC / 1024; ++u) {  // x: 32 rows x kFC / 4 quads
        const int e = threadIdx.x + 256 * u, rr = e / (kFC / 4), cc = (e % (kFC / 4)) * 4;
        const bool ok = I + rr < m && J + cc < m;
        cp_async16(&X(b)[rr][cc], ok ? d + int64_t(I + rr) * m + J + cc : d, ok);
      }
#pragma unroll
      for (int u = 0; u < kFR * kFC / 1024; ++u) {  // y: kFC rows (candidates J + yr) x 8 quads (I + 4 qd ..)
        const int e = threadIdx.x + 256 * u, yr = e >> 3, qd = e & 7;
        const bool ok = J + yr < m && I + 4 * qd < m;
        cp_async16(yat(b, yr, 4 * qd), ok ? d + int64_t(J + yr) * m + I + 4 * qd : d, ok);
      }
    } else {
#pragma unroll
      for (int u = 0; u < kFR * kFC / 256; ++u) {  // x: 32 rows x kFC columns
        const int e = threadIdx.x + 256 * u, rr = e / kFC, cc = e % kFC;
        const bool ok = I + rr < m && J + cc < m;
        cp_async4(&X(b)[rr][cc], ok ? d + int64_t(I + rr) * m + J + cc : d, ok);
      }
#pragma unroll
      for (int u = 0; u < kFR * kFC / 256; ++u) {  // y: kFC rows (candidates J + yr) x 32 columns (I + yc)
        const int e = threadIdx.x + 256 * u, yr = e >> 5, yc = e & 31;
        const bool ok = J + yr < m && I + yc < m;
        cp_async4(yat(b, yr, yc), ok ? d + int64_t(J + yr) * m + I + yc : d, ok);
      }
    }
    cp_async_commit();
  };
  Part p_row = 0, p_col = 0, p_wo = 0, p_wi = 0;
  // packed lanes (kFPacked): biased margin min / max, largest entry, largest
  // winning edge out / in, and wins / losses counted in units of 2^15
  constexpr uint32_t G = 0x80008000u;
  uint32_t mn2 = 0xFFFFFFFFu, mx2 = 0u, mxd2 = 0u, mxwo2 = 0u, mxwi2 = 0u, wacc = 0u, lacc = 0u;
  auto count = [&](int32_t a_, int32_t b_) {
    const int32_t diff = a_ - b_;
    p_row += Part(a_), p_col += Part(b_);
    mx_d = max(mx_d, a_);
    mn_mg = min(mn_mg, diff), mx_mg = max(mx_mg, diff);
    const bool w = diff > 0, l = diff < 0;
    win += w, loss += l;
    const int32_t wo = w ? a_ : 0, wi = l ? b_ : 0;
    p_wo += Part(wo), p_wi += Part(wi);
    mx_wo = max(mx_wo, wo), mx_wi = max(mx_wi, wi);
  };
  for (int st = 0; st < kFStages - 1; ++st) {
    if (t0 + st < t1) issue((t0 + st) * kFC, st);
    else cp_async_commit();  // empty groups keep the wait below uniform
  }
  for (int32_t tile = t0; tile < t1; ++tile) {
    const int32_t J = tile * kFC;
    const int kk = tile - t0, b = kk % kFStages;
    cp_async_wait<kFStages - 2>();  // this thread's copies of this tile have landed
    __syncthreads();                // everyone's have, and the previous tile is counted
    if (tile + kFStages - 1 < t1) issue((tile + kFStages - 1) * kFC, (kk + kFStages - 1) % kFStages);
    else cp_async_commit();
    if (i >= m) continue;
    p_row = p_col = p_wo = p_wi = 0;
    const bool clean = J + kFC <= m && (J >= I + kFR || I >= J + kFC);  // no diagonal entry, no padding
#pragma unroll
    for (int sp = 0; sp < kFSlabs; sp += 2) {  // columns 32 sp + 4 q .. +3 and 32 (sp + 1) + 4 q .. +3
      int32_t dij[8], dji[8];
      {
        const int4 lo = *reinterpret_cast<const int4*>(&X(b)[r][32 * sp + 4 * q]);
        const int4 hi = *reinterpret_cast<const int4*>(&X(b)[r][32 * sp + 32 + 4 * q]);
        dij[0] = lo.x, dij[1] = lo.y, dij[2] = lo.z, dij[3] = lo.w;
        dij[4] = hi.x, dij[5] = hi.y, dij[6] = hi.z, dij[7] = hi.w;
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) dji[k] = *yat(b, 32 * sp + (k >> 2) * 32 + 4 * q + (k & 3), r);
      if (clean) {
        if (kMode == kFPacked) {
#pragma unroll
          for (int k = 0; k < 8; k += 4) {  // two lane pairs at a time (three-input min / max)
            uint32_t av[2], bv[2], dA[2], wo[2], wi[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              av[h] = prmt(uint32_t(dij[k + 2 * h]), uint32_t(dij[k + 2 * h + 1]), 0x5410u);  // d[i][j], d[i][j+1]
              bv[h] = prmt(uint32_t(dji[k + 2 * h]), uint32_t(dji[k + 2 * h + 1]), 0x5410u);  // d[j][i], d[j+1][i]
              dA[h] = (av[h] | G) - bv[h];                    // 2^15 + a - b per lane
              const uint32_t dB = (bv[h] | G) - av[h];        // 2^15 + b - a
              const uint32_t wb = ~dB & G, lb = ~dA[h] & G;  // a > b, a < b
              wacc = __dp2a_lo(wb, 0x0101u, wacc), lacc = __dp2a_lo(lb, 0x0101u, lacc);
              wo[h] = av[h] & prmt(wb, 0u, 0xBB99u), wi[h] = bv[h] & prmt(lb, 0u, 0xBB99u);
              p_row = __dp2a_lo(av[h], 0x0101u, p_row), p_col = __dp2a_lo(bv[h], 0x0101u, p_col);
              p_wo = __dp2a_lo(wo[h], 0x0101u, p_wo), p_wi = __dp2a_lo(wi[h], 0x0101u, p_wi);
            }
            mn2 = __vimin3_u16x2(mn2, dA[0], dA[1]), mx2 = __vimax3_u16x2(mx2, dA[0], dA[1]);
            mxd2 = __vimax3_u16x2(mxd2, av[0], av[1]);
            mxwo2 = __vimax3_u16x2(mxwo2, wo[0], wo[1]), mxwi2 = __vimax3_u16x2(mxwi2, wi[0], wi[1]);
          }
        } else {
#pragma unroll
          for (int k = 0; k < 8; ++k) count(dij[k], dji[k]);
        }
      } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int32_t j = J + 32 * sp + (k >> 2) * 32 + 4 * q + (k & 3);
          if (j < m && j != i) count(dij[k], dji[k]);
        }
      }
    }
    s_row += p_row, s_col += p_col, s_wo += p_wo, s_wi += p_wi;
  }
  if (kMode == kFPacked) {  // fold the lanes into the per-entry statistics
    win += int32_t(wacc >> 15), loss += int32_t(lacc >> 15);
    const int32_t mnb = min(int32_t(mn2 & 0xFFFFu), int32_t(mn2 >> 16));
    const int32_t mxb = max(int32_t(mx2 & 0xFFFFu), int32_t(mx2 >> 16));
    if (mnb != 0xFFFF) mn_mg = min(mn_mg, mnb - 0x8000);
    if (mxb != 0) mx_mg = max(mx_mg, mxb - 0x8000);
    mx_d = max(mx_d, max(int32_t(mxd2 & 0xFFFFu), int32_t(mxd2 >> 16)));
    mx_wo = max(mx_wo, max(int32_t(mxwo2 & 0xFFFFu), int32_t(mxwo2 >> 16)));
    mx_wi = max(mx_wi, max(int32_t(mxwi2 & 0xFFFFu), int32_t(mxwi2 >> 16)));
  }
#pragma unroll
  for (int o = 1; o <= 4; o <<= 1) {
    win += __shfl_xor_sync(0xFFFFFFFFu, win, o);
    loss += __shfl_xor_sync(0xFFFFFFFFu, loss, o);
    s_row += __shfl_xor_sync(0xFFFFFFFFu, s_row, o);
    s_col += __shfl_xor_sync(0xFFFFFFFFu, s_col, o);
    s_wo += __shfl_xor_sync(0xFFFFFFFFu, s_wo, o);
    s_wi += __shfl_xor_sync(0xFFFFFFFFu, s_wi, o);
    mx_wo = max(mx_wo, __shfl_xor_sync(0xFFFFFFFFu, mx_wo, o));
    mx_wi = max(mx_wi, __shfl_xor_sync(0xFFFFFFFFu, mx_wi, o));
    mx_d = max(mx_d, __shfl_xor_sync(0xFFFFFFFFu, mx_d, o));
    mn_mg = min(mn_mg, __shfl_xor_sync(0xFFFFFFFFu, mn_mg, o));
    mx_mg = max(mx_mg, __shfl_xor_sync(0xFFFFFFFFu, mx_mg, o));
  }
  if (q == 0 && i < m) {
    if (win) atomicAdd(&a.wins[i], win);
    if (loss) atomicAdd(&a.losses[i], loss);
    if (s_row) atomicAdd(&a.rowsum[i], s_row);
    if (s_col) atomicAdd(&a.colsum[i], s_col);
    if (s_wo) atomicAdd(&a.sumw_out[i], s_wo);
    if (s_wi) atomicAdd(&a.sumw_in[i], s_wi);
    if (mx_wo) atomicMax(&a.maxw_out[i], mx_wo);
    if (mx_wi) atomicMax(&a.maxw_in[i], mx_wi);
    if (mx_d) atomicMax(&a.max_drow[i], mx_d);
    if (mn_mg != INT32_MAX) atomicMin(&a.min_margin[i], mn_mg);
    if (mx_mg != INT32_MIN) atomicMax(&a.max_margin[i], mx_mg);
  }
}

// f[c][0..13] from the accumulators; ranks (14, 15) are counted afterwards.
__global__ void features_finalize_kernel(Acc a, int32_t m, int64_t n, float* __restrict__ feat) {
  const double nn = double(n > 0 ? n : 1), mm = double(m > 1 ? m - 1 : 1);
  const double inv_m = 1.0 / mm, inv_n = 1.0 / nn, inv_nm = 1.0 / (nn * mm);  // FP64 divides are slow
  for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) {
    float* f = feat + int64_t(c) * kNF;
    if (m < 2) {
      for (int q = 0; q < kNF; ++q) f[q] = 0.f;
      continue;
    }
    const int32_t wn = a.wins[c], ls = a.losses[c], mo = a.maxw_out[c], mi = a.maxw_in[c];
    f[0] = float(double(wn) * inv_m);
    f[1] = float(double(ls) * inv_m);
    f[2] = float(double(int64_t(m - 1) - wn - ls) * inv_m);  // every other candidate: win, loss or tie
    f[3] = float(double(a.rowsum[c]) * inv_nm);
    f[4] = float(double(a.colsum[c]) * inv_nm);
    f[5] = float(double(mo) * inv_n);
    f[6] = float(double(mi) * inv_n);
    f[7] = mi > mo ? 1.f : 0.f;
    f[8] = float(double(mo - mi) * inv_n);
    f[9] = float(double(a.sumw_out[c]) * inv_nm);
    f[10] = float(double(a.sumw_in[c]) * inv_nm);
    f[11] = float(double(a.min_margin[c]) * inv_n);
    f[12] = float(double(a.max_margin[c]) * inv_n);
    f[13] = float(double(a.max_drow[c]) * inv_n);
    f[14] = f[15] = 0.f;  // the ranks, filled in afterwards
  }
}

// f[c][14] = #{j: rowsum[j] > rowsum[c]} / (m-1); f[c][15] likewise for
// wins - losses. CTA (s, cb, z) ranks by the row sums (z = 0) or by wins -
// losses (z = 1): it maps the keys of candidates kRankChunk s .. + kRankChunk
// - 1 to unsigned integers in the same order (row sum + 1; wins - losses +
// 2^31), all above the padding value 0, sorts them into descending order with
// a bitonic network in shared memory, then counts for each candidate c of
// block cb the keys of the chunk above its own by binary search; the counts
// of the chunks are added atomically.
constexpr int kRankChunk = 1024;
__global__ void __launch_bounds__(kRankChunk / 2) features_rank_kernel(Acc a, int32_t m, int32_t* __restrict__ cnt14,
                                                                       int32_t* __restrict__ cnt15) {
  __shared__ unsigned long long ks[kRankChunk];
  const bool by_row = blockIdx.z == 0;
  auto key = [&](int32_t c) -> unsigned long long {
    return by_row ? a.rowsum[c] + 1ull
                  : (unsigned long long)(int64_t(a.wins[c]) - a.losses[c] + (int64_t(1) << 31));
  };
  const int32_t j0 = blockIdx.x * kRankChunk;
  for (int t = threadIdx.x; t < kRankChunk; t += blockDim.x) ks[t] = j0 + t < m ? key(j0 + t) : 0ull;
  __syncthreads();
  for (int k = 2; k <= kRankChunk; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      const int t = threadIdx.x, i = 2 * t - (t & (j - 1)), l = i + j;  // i has bit j clear
      const unsigned long long x = ks[i], y = ks[l];
      if ((x < y) == ((i & k) == 0)) ks[i] = y, ks[l] = x;  // descending where bit k of i is clear
      __syncthreads();
    }
  int32_t* cnt = by_row ? cnt14 : cnt15;
  const int32_t c1 = min(m, int32_t(blockIdx.y + 1) * kRankChunk);
  for (int32_t c = blockIdx.y * kRankChunk + threadIdx.x; c < c1; c += blockDim.x) {
    const unsigned long long x = key(c);
    int lo = 0, hi = kRankChunk;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (ks[mid] > x) lo = mid + 1;
      else hi = mid;
    }
    if (lo) atomicAdd(&cnt[c], lo);
  }
}

__global__ void features_rank_finalize_kernel(const int32_t* __restrict__ cnt14, const int32_t* __restrict__ cnt15,
                                              int32_t m, float* __restrict__ feat) {
  const double inv_m = 1.0 / double(m > 1 ? m - 1 : 1);
  for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) {
    if (m < 2) continue;
    feat[int64_t(c) * kNF + 14] = float(double(cnt14[c]) * inv_m);
    feat[int64_t(c) * kNF + 15] = float(double(cnt15[c]) * inv_m);
  }
}

// ----------------------------------------------------------------- MLP

// Forward pass, one thread per candidate; parameters staged in shared
// memory. h1, h2 (ReLU outputs) are stored when given (training). Launched
// with kMlpThreads per CTA so that a list of a few thousand candidates
// spreads over most SMs; every thread reads the same weight at a time
// (a broadcast), four weights per 16-byte load, each sum taken in the
// parameters' order.
constexpr int kMlpThreads = 64;
__global__ void __launch_bounds__(256) mlp_forward_kernel(const float* __restrict__ theta,
                                                          const float* __restrict__ feat, int32_t N,
                                                          float* __restrict__ score, float* __restrict__ h1out,
                                                          float* __restrict__ h2out) {
  __shared__ __align__(16) float p[kNP + 3];
  // stage the parameters with eight loads in flight per thread (16-byte
  // loads when the caller's array is 16-byte aligned)
  if ((reinterpret_cast<uintptr_t>(theta) & 15u) == 0) {
    const float4* t4 = reinterpret_cast<const float4*>(theta);
    float4* p4 = reinterpret_cast<float4*>(p);
    constexpr int kN4 = kNP / 4;
    for (int t0 = threadIdx.x; t0 < kN4; t0 += 8 * blockDim.x) {
      float4 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int t = t0 + u * blockDim.x;
        if (t < kN4) v[u] = __ldg(t4 + t);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int t = t0 + u * blockDim.x;
        if (t < kN4) p4[t] = v[u];
      }
    }
    for (int t = 4 * kN4 + threadIdx.x; t < kNP; t += blockDim.x) p[t] = theta[t];
  } else {
    for (int t0 = threadIdx.x; t0 < kNP; t0 += 8 * blockDim.x) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int t = t0 + u * blockDim.x;
        if (t < kNP) v[u] = __ldg(theta + t);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int t = t0 + u * blockDim.x;
        if (t < kNP) p[t] = v[u];
      }
    }
  }
  __syncthreads();
  const int32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  float x[kNF];
#pragma unroll
  for (int q = 0; q < kNF; ++q) x[q] = feat[int64_t(c) * kNF + q];
  float h1[kH];
  static_assert(kOffW1 % 4 == 0 && kOffW2 % 4 == 0 && kNF % 4 == 0 && kH % 4 == 0, "16-byte weight rows");
#pragma unroll
  for (int o = 0; o < kH; ++o) {
    float s = p[kOffB1 + o];
    const float4* w = reinterpret_cast<const float4*>(p + kOffW1 + o * kNF);
#pragma unroll
    for (int q4 = 0; q4 < kNF / 4; ++q4) {
      const float4 v = w[q4];
      s = fmaf(v.x, x[4 * q4], s), s = fmaf(v.y, x[4 * q4 + 1], s);
      s = fmaf(v.z, x[4 * q4 + 2], s), s = fmaf(v.w, x[4 * q4 + 3], s);
    }
    h1[o] = fmaxf(s, 0.f);
  }
  float out = p[kOffB3];
  // four outputs at a time: their sums are independent chains that hide
  // each other's latency (each sum still runs in the parameters' order)
#pragma unroll 4
  for (int o = 0; o < kH; ++o) {
    float s = p[kOffB2 + o];
    const float4* w = reinterpret_cast<const float4*>(p + kOffW2 + o * kH);
#pragma unroll
    for (int q4 = 0; q4 < kH / 4; ++q4) {
      const float4 v = w[q4];
      s = fmaf(v.x, h1[4 * q4], s), s = fmaf(v.y, h1[4 * q4 + 1], s);
      s = fmaf(v.z, h1[4 * q4 + 2], s), s = fmaf(v.w, h1[4 * q4 + 3], s);
    }
    const float h = fmaxf(s, 0.f);
    if (h2out) h2out[int64_t(c) * kH + o] = h;
    out = fmaf(p[kOffW3 + o], h, out);
  }
  if (h1out) {
#pragma unroll
    for (int q = 0; q < kH; ++q) h1out[int64_t(c) * kH + q] = h1[q];
  }
  score[c] = out;
}

// Listwise softmax cross-entropy of one election (segment) per CTA: target
// mass 1/|winners| on each winner. ds[c] = (softmax_c - t_c) / nseg; the
// segment's loss goes to seg_loss[e].
__global__ void __launch_bounds__(256) mlp_loss_kernel(const float* __restrict__ score,
                                                       const int32_t* __restrict__ label,
                                                       const int32_t* __restrict__ seg_off, int32_t nseg,
                                                       float* __restrict__ ds, float* __restrict__ seg_loss) {
  __shared__ float red[256];
  __shared__ int32_t redi[256];
  const int32_t e = blockIdx.x;
  const int32_t a = seg_off[e], b = seg_off[e + 1];
  float mx = -INFINITY;
  int32_t nw = 0;
  for (int32_t c = a + threadIdx.x; c < b; c += blockDim.x) {
    mx = fmaxf(mx, score[c]);
    nw += label[c] != 0;
  }
  red[threadIdx.x] = mx;
  redi[threadIdx.x] = nw;
  __syncthreads();
  for (int o = blockDim.x / 2; o; o >>= 1) {
    if (threadIdx.x < o) {
      red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + o]);
      redi[threadIdx.x] += redi[threadIdx.x + o];
    }
    __syncthreads();
  }
  mx = red[0];
  nw = max(redi[0], 1);
  __syncthreads();
  float se = 0.f;
  for (int32_t c = a + threadIdx.x; c < b; c += blockDim.x) se += expf(score[c] - mx);
  red[threadIdx.x] = se;
  __syncthreads();
  for (int o = blockDim.x / 2; o; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  const float lse = mx + logf(red[0]);
  __syncthreads();
  float l = 0.f;
  const float inv_e = 1.f / float(nseg), inv_w = 1.f / float(nw);
  for (int32_t c = a + threadIdx.x; c < b; c += blockDim.x) {
    const float logp = score[c] - lse;
    const float t = label[c] ? inv_w : 0.f;
    l -= t * logp;
    ds[c] = (expf(logp) - t) * inv_e;
  }
  red[threadIdx.x] = l;
  __syncthreads();
  for (int o = blockDim.x / 2; o; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) seg_loss[e] = red[0];
}

constexpr int kChunk = 64;  // candidates per backward CTA

// Backward over a chunk of kChunk candidates: dh2, dh1 per candidate, then
// this chunk's sum of every parameter gradient into partial[chunk][kNP].
struct BackwardSmem {
  float W2[kH * kH], W3[kH];
  float sx[kChunk][kNF], sh1[kChunk][kH + 1], sh2[kChunk][kH + 1], sd2[kChunk][kH + 1], sd1[kChunk][kH + 1];
  float sds[kChunk];
};

__global__ void __launch_bounds__(256) mlp_backward_kernel(const float* __restrict__ theta,
                                                           const float* __restrict__ feat,
                                                           const float* __restrict__ h1g, const float* __restrict__ h2g,
                                                           const float* __restrict__ ds, int32_t N,
                                                           float* __restrict__ partial) {
  extern __shared__ __align__(16) unsigned char bw_raw[];
  BackwardSmem& S = *reinterpret_cast<BackwardSmem*>(bw_raw);
  float* W2 = S.W2;
  float* W3 = S.W3;
  auto& sx = S.sx;
  auto& sh1 = S.sh1;
  auto& sh2 = S.sh2;
  auto& sd2 = S.sd2;
  auto& sd1 = S.sd1;
  float* sds = S.sds;
  const int32_t c0 = blockIdx.x * kChunk;
  const int nc = min(kChunk, N - c0);
  for (int t = threadIdx.x; t < kH * kH; t += blockDim.x) W2[t] = theta[kOffW2 + t];
  for (int t = threadIdx.x; t < kH; t += blockDim.x) W3[t] = theta[kOffW3 + t];
  for (int t = threadIdx.x; t < kChunk * kH; t += blockDim.x) {
    const int r = t / kH, q = t % kH;
    sh1[r][q] = r < nc ? h1g[int64_t(c0 + r) * kH + q] : 0.f;
    sh2[r][q] = r < nc ? h2g[int64_t(c0 + r) * kH + q] : 0.f;
  }
  for (int t = threadIdx.x; t < kChunk * kNF; t += blockDim.x) {
    const int r = t / kNF, q = t % kNF;
    sx[r][q] = r < nc ? feat[int64_t(c0 + r) * kNF + q] : 0.f;
  }
  for (int t = threadIdx.x; t < kChunk; t += blockDim.x) sds[t] = t < nc ? ds[c0 + t] : 0.f;
  __syncthreads();
  // dh2[r][o] = ds_r * W3[o] * [h2 > 0]
  for (int t = threadIdx.x; t < kChunk * kH; t += blockDim.x) {
    const int r = t / kH, o = t % kH;
    sd2[r][o] = sh2[r][o] > 0.f ? sds[r] * W3[o] : 0.f;
  }
  __syncthreads();
  // dh1[r][q] = sum_o W2[o][q] dh2[r][o] * [h1 > 0]
  for (int t = threadIdx.x; t < kChunk * kH; t += blockDim.x) {
    const int r = t / kH, q = t % kH;
    float s = 0.f;
    for (int o = 0; o < kH; ++o) s = fmaf(W2[o * kH + q], sd2[r][o], s);
    sd1[r][q] = sh1[r][q] > 0.f ? s : 0.f;
  }
  __syncthreads();
  float* out = partial + int64_t(blockIdx.x) * kNP;
  for (int t = threadIdx.x; t < kNP; t += blockDim.x) {
    float g = 0.f;
    if (t < kOffB1) {  // W1[o][q]: sum_r dh1[r][o] x[r][q]
      const int o = t / kNF, q = t % kNF;
      for (int r = 0; r < kChunk; ++r) g = fmaf(sd1[r][o], sx[r][q], g);
    } else if (t < kOffW2) {
      const int o = t - kOffB1;
      for (int r = 0; r < kChunk; ++r) g += sd1[r][o];
    } else if (t < kOffB2) {  // W2[o][q]: sum_r dh2[r][o] h1[r][q]
      const int o = (t - kOffW2) / kH, q = (t - kOffW2) % kH;
      for (int r = 0; r < kChunk; ++r) g = fmaf(sd2[r][o], sh1[r][q], g);
    } else if (t < kOffW3) {
      const int o = t - kOffB2;
      for (int r = 0; r < kChunk; ++r) g += sd2[r][o];
    } else if (t < kOffB3) {  // W3[o]: sum_r ds_r h2[r][o]
      const int o = t - kOffW3;
      for (int r = 0; r < kChunk; ++r) g = fmaf(sds[r], sh2[r][o], g);
    } else {
      for (int r = 0; r < kChunk; ++r) g += sds[r];
    }
    out[t] = g;
  }
}

// grad[t] = sum over chunks of partial[chunk][t], in chunk order; loss =
// sum of the segment losses / nseg. Deterministic.
__global__ void mlp_reduce_kernel(const float* __restrict__ partial, int32_t nchunks, const float* __restrict__ seg_loss,
                                  int32_t nseg, float* __restrict__ grad, float* __restrict__ loss) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < kNP) {
    float g = 0.f;
    for (int32_t c = 0; c < nchunks; ++c) g += partial[int64_t(c) * kNP + t];
    grad[t] = g;
  }
  if (t == 0 && loss) {
    float l = 0.f;
    for (int32_t e = 0; e < nseg; ++e) l += seg_loss[e];
    *loss = l / float(nseg);
  }
}

// Adam (Kingma and Ba, 2015), 1-based step.
__global__ void adam_kernel(float* __restrict__ theta, float* __restrict__ m1, float* __restrict__ m2,
                            const float* __restrict__ grad, int64_t step, float lr, float b1, float b2, float eps) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= kNP) return;
  const float g = grad[t];
  const float a = b1 * m1[t] + (1.f - b1) * g;
  const float v = b2 * m2[t] + (1.f - b2) * g * g;
  m1[t] = a;
  m2[t] = v;
  const float mh = a / (1.f - powf(b1, float(step)));
  const float vh = v / (1.f - powf(b2, float(step)));
  theta[t] -= lr * mh / (sqrtf(vh) + eps);
}

// --------------------------------------------------------- proposals

// (s, c) ranks before (s2, c2): higher score, then smaller id
__device__ __forceinline__ bool ranks_before(float s, int32_t c, float s2, int32_t c2) {
  return s > s2 || (s == s2 && c < c2);
}

// Pops the head of a sorted register list (static indices only).
__device__ __forceinline__ void pop_head(float (&ls)[kMaxProposals], int32_t (&li)[kMaxProposals]) {
#pragma unroll
  for (int q = 0; q + 1 < kMaxProposals; ++q) ls[q] = ls[q + 1], li[q] = li[q + 1];
  ls[kMaxProposals - 1] = -INFINITY, li[kMaxProposals - 1] = INT32_MAX;
}

// Repeated warp-wide selection of the best list head: the `top` best of the
// 32 lanes' sorted lists, in order (lane 0 holds them in bs/bi per round).
__device__ __forceinline__ void warp_merge(float (&ls)[kMaxProposals], int32_t (&li)[kMaxProposals], int32_t top,
                                           float* out_s, int32_t* out_i) {
  for (int r = 0; r < top; ++r) {
    float bs = ls[0];
    int32_t bi = li[0];
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const float s2 = __shfl_xor_sync(0xFFFFFFFFu, bs, o);
      const int32_t i2 = __shfl_xor_sync(0xFFFFFFFFu, bi, o);
      if (ranks_before(s2, i2, bs, bi)) bs = s2, bi = i2;
    }
    if (bi != INT32_MAX && li[0] == bi) pop_head(ls, li);  // ids are unique: one lane pops
    if ((threadIdx.x & 31) == 0) out_s[r] = bs, out_i[r] = bi;
  }
}

// The `top` best scores (ties: smaller id first), -1 past the candidates;
// one CTA: each thread keeps the best `top` of its scores in registers,
// each warp merges its lanes' lists, warp 0 merges the warps'.
__device__ void topk_body(const float* __restrict__ score, int32_t m, int32_t top, int32_t* __restrict__ out) {
  __shared__ float ws[32][kMaxProposals];
  __shared__ int32_t wi[32][kMaxProposals];
  float ls[kMaxProposals];
  int32_t li[kMaxProposals];
#pragma unroll
  for (int q = 0; q < kMaxProposals; ++q) ls[q] = -INFINITY, li[q] = INT32_MAX;
  for (int32_t c = threadIdx.x; c < m; c += blockDim.x) {
    float s = score[c];
    int32_t id = c;
#pragma unroll
    for (int q = 0; q < kMaxProposals; ++q)  // insertion: the displaced entry moves down
      if (ranks_before(s, id, ls[q], li[q])) {
        const float ts = ls[q];
        const int32_t ti = li[q];
        ls[q] = s, li[q] = id, s = ts, id = ti;
      }
  }
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  warp_merge(ls, li, top, ws[wid], wi[wid]);
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int q = 0; q < kMaxProposals; ++q) {
      const bool ok = lane < nwarps && q < top;
      ls[q] = ok ? ws[lane][q] : -INFINITY;
      li[q] = ok ? wi[lane][q] : INT32_MAX;
    }
    __shared__ float fs[kMaxProposals];
    __shared__ int32_t fi[kMaxProposals];
    warp_merge(ls, li, top, fs, fi);
    __syncwarp();
    if (lane < top) out[lane] = fi[lane] == INT32_MAX ? -1 : fi[lane];
  }
}

// Copeland score wins - losses as a non-learned proposer.
__global__ void copeland_score_kernel(Acc a, int32_t m, float* __restrict__ score) {
  for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x)
    score[c] = float(a.wins[c] - a.losses[c]);
}

// ------------------------------------------------------- certification

// warm[a] = a-th candidate with an outgoing edge (wins > 0), in id order;
// slot[c] = its index or -1. One CTA.
__device__ void warm_list_body(const int32_t* __restrict__ wins, int32_t m, int32_t* __restrict__ warm,
                               int32_t* __restrict__ slot, int32_t* __restrict__ nwarm) {
  __shared__ int32_t part[1024];
  const int T = blockDim.x;
  const int per = (m + T - 1) / T;
  const int b = threadIdx.x * per, e = min(m, b + per);
  int32_t s = 0;
  for (int c = b; c < e; ++c) s += wins[c] > 0;
  part[threadIdx.x] = s;
  __syncthreads();
  for (int o = 1; o < T; o <<= 1) {
    int32_t x = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += x;
    __syncthreads();
  }
  int32_t pos = threadIdx.x ? part[threadIdx.x - 1] : 0;
  for (int c = b; c < e; ++c) {
    if (wins[c] > 0) {
      warm[pos] = c;
      slot[c] = pos++;
    } else {
      slot[c] = -1;
    }
  }
  if (threadIdx.x == T - 1) *nwarm = part[T - 1];
}

__global__ void __launch_bounds__(1024) warm_list_kernel(const int32_t* __restrict__ wins, int32_t m,
                                                         int32_t* __restrict__ warm, int32_t* __restrict__ slot,
                                                         int32_t* __restrict__ nwarm) {
  warm_list_body(wins, m, warm, slot, nwarm);
}

// The proposals and the warm list in one launch (CTA 0 and CTA 1 side by
// side): the two single-CTA passes of schulze_winners_fast depend on
// different inputs (the scores; the wins of the features pass).
__global__ void __launch_bounds__(1024) propose_kernel(const float* __restrict__ score, int32_t m, int32_t top,
                                                       int32_t* __restrict__ out, const int32_t* __restrict__ wins,
                                                       int32_t* __restrict__ warm, int32_t* __restrict__ slot,
                                                       int32_t* __restrict__ nwarm) {
  if (blockIdx.x == 0)
    topk_body(score, m, top, out);
  else
    warm_list_body(wins, m, warm, slot, nwarm);
}

// Ww[a][b] = w(warm[a], warm[b]) and Wt[b][a] = the same (winning votes).
__global__ void warm_pack_kernel(const int32_t* __restrict__ d, int32_t m, const int32_t* __restrict__ warm,
                                 const int32_t* __restrict__ nwarm, int32_t* __restrict__ Ww, int32_t* __restrict__ Wt) {
  const int32_t nw = *nwarm;
  if (nw > kCertifyMaxWarm) return;
  const int64_t total = int64_t(nw) * nw;
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
    const int32_t a = int32_t(t / nw), b = int32_t(t % nw);
    const int32_t i = warm[a], j = warm[b];
    int32_t w = 0;
    if (i != j) {
      const int32_t x = d[int64_t(i) * m + j], y = d[int64_t(j) * m + i];
      w = x > y ? x : 0;
    }
    Ww[t] = w;
    Wt[int64_t(b) * nw + a] = w;
  }
}

// Widest paths from (dir 0) or to (dir 1) warm candidate `s` inside the warm
// subgraph, by (max, min) Bellman-Ford rounds until nothing changes (at most
// nw rounds). x lives in shared memory; warp per target, lanes over sources.
// dir 0: x[b] = max(x[b], max_a min(x[a], w[a][b])) reads Wt row b;
// dir 1: x[b] = max(x[b], max_a min(w[b][a], x[a])) reads Ww row b.
// x[s] is the empty path (+inf). Returns the number of rounds.
__device__ int32_t widest_warm(const int32_t* __restrict__ Ww, const int32_t* __restrict__ Wt, int32_t nw, int32_t s,
                               int dir, int32_t* __restrict__ x) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int32_t* M = dir == 0 ? Wt : Ww;
  for (int32_t b = threadIdx.x; b < nw; b += blockDim.x)
    x[b] = b == s ? INT32_MAX : (dir == 0 ? Ww[int64_t(s) * nw + b] : Ww[int64_t(b) * nw + s]);
  __syncthreads();
  int32_t rounds = 0;
  for (;;) {
    ++rounds;
    int changed = 0;
    for (int32_t b = wid; b < nw; b += nwarps) {
      const int32_t* row = M + int64_t(b) * nw;
      int32_t best = 0;
      for (int32_t a = lane; a < nw; a += 32) best = max(best, min(x[a], row[a]));
      best = warp_max(best);
      if (lane == 0 && b != s && best > x[b]) {
        x[b] = best;  // monotone: reading old or new values elsewhere is still a valid lower bound
        changed = 1;
      }
    }
    if (!__syncthreads_or(changed) || rounds > nw + 1) break;
  }
  return rounds;
}

// Certification, one CTA of 1024 threads. Proposals are tried in order;
// the first c with p(c, j) >= p(j, c) for every warm j is a winner (for cold
// j, p(j, c) = 0). The other winners are the warm candidates tied with c
// (each certified in turn) and the cold candidates without incoming edges.
// res: [0] 1 if the winner set is exact, 0 if the closure must decide;
// [1] index of the certified proposal (-1 none); [2] ties checked;
// [3] Bellman-Ford rounds.
__global__ void __launch_bounds__(1024) certify_kernel(const int32_t* __restrict__ Ww, const int32_t* __restrict__ Wt,
                                                       const int32_t* __restrict__ nwarm_p,
                                                       const int32_t* __restrict__ warm,
                                                       const int32_t* __restrict__ slot,
                                                       const int32_t* __restrict__ losses, int32_t m,
                                                       const int32_t* __restrict__ cand, int32_t ncand,
                                                       int32_t* __restrict__ fwd, int32_t* __restrict__ bwd,
                                                       int32_t* __restrict__ winners, int32_t* __restrict__ res) {
  __shared__ int32_t s_ok, s_ties[kMaxTies], s_nties, s_overflow;
  const int32_t nw = *nwarm_p;
  for (int32_t c = threadIdx.x; c < m; c += blockDim.x) winners[c] = 0;
  if (threadIdx.x == 0) res[0] = 0, res[1] = -1, res[2] = 0, res[3] = 0;
  __syncthreads();
  if (nw > kCertifyMaxWarm) return;  // closure decides
  if (nw == 0) {  // no edges at all: every candidate is a winner, so the first proposal certifies
    for (int32_t c = threadIdx.x; c < m; c += blockDim.x) winners[c] = 1;
    if (threadIdx.x == 0) res[0] = 1, res[1] = ncand > 0 ? 0 : -1;
    return;
  }
  int32_t rounds = 0;
  int32_t found = -1;
  for (int32_t p = 0; p < ncand && found < 0; ++p) {
    const int32_t c = cand[p];
    if (c < 0 || c >= m || slot[c] < 0) continue;  // cold proposals cannot be certified this way
    const int32_t s = slot[c];
    rounds += widest_warm(Ww, Wt, nw, s, 0, fwd);
    rounds += widest_warm(Ww, Wt, nw, s, 1, bwd);
    if (threadIdx.x == 0) s_ok = 1;
    __syncthreads();
    for (int32_t b = threadIdx.x; b < nw; b += blockDim.x)
      if (b != s && fwd[b] < bwd[b]) s_ok = 0;
    __syncthreads();
    if (s_ok) found = p;
    __syncthreads();
  }
  if (found < 0) {
    if (threadIdx.x == 0) res[3] = rounds;
    return;
  }
  const int32_t c = cand[found], s = slot[c];
  // ties with c among the warm candidates
  if (threadIdx.x == 0) s_nties = 0, s_overflow = 0;
  __syncthreads();
  for (int32_t b = threadIdx.x; b < nw; b += blockDim.x) {
    if (b != s && fwd[b] == bwd[b]) {
      const int32_t q = atomicAdd(&s_nties, 1);
      if (q < kMaxTies) s_ties[q] = b;
      else s_overflow = 1;
    }
  }
  __syncthreads();
  if (s_overflow) {
    if (threadIdx.x == 0) res[1] = found, res[3] = rounds;
    return;  // too many ties: the closure decides
  }
  const int32_t nt = s_nties;
  // cold candidates without incoming edges are winners too
  for (int32_t j = threadIdx.x; j < m; j += blockDim.x)
    if (slot[j] < 0 && losses[j] == 0) winners[j] = 1;
  if (threadIdx.x == 0) winners[c] = 1;
  for (int32_t t = 0; t < nt; ++t) {
    const int32_t sb = s_ties[t];
    rounds += widest_warm(Ww, Wt, nw, sb, 0, fwd);
    rounds += widest_warm(Ww, Wt, nw, sb, 1, bwd);
    if (threadIdx.x == 0) s_ok = 1;
    __syncthreads();
    for (int32_t b = threadIdx.x; b < nw; b += blockDim.x)
      if (b != sb && fwd[b] < bwd[b]) s_ok = 0;
    __syncthreads();
    if (s_ok && threadIdx.x == 0) winners[warm[sb]] = 1;
    __syncthreads();
  }
  if (threadIdx.x == 0) res[0] = 1, res[1] = found, res[2] = nt, res[3] = rounds;
}

struct LearnedWs {
  Acc acc;
  int32_t *cnt14, *cnt15;
  float* score;
  int32_t *cand, *warm, *slot, *nwarm, *Ww, *Wt, *res;
};

size_t learned_ws_bytes(int32_t m) {
  size_t b = 0;
  b += 12 * align_up(size_t(m) * 8, 256);
  b += 4 * align_up(size_t(m) * 4, 256);
  b += 2 * align_up(size_t(std::min<int32_t>(m, kCertifyMaxWarm)) * size_t(std::min<int32_t>(m, kCertifyMaxWarm)) * 4,
                    256);
  return b + 8192;
}

LearnedWs carve_learned(void* ws, int32_t m) {
  Carver cv(ws);
  LearnedWs w;
  w.acc.wins = cv.take<int32_t>(m);
  w.acc.losses = cv.take<int32_t>(m);
  w.acc.rowsum = cv.take<unsigned long long>(m);
  w.acc.colsum = cv.take<unsigned long long>(m);
  w.acc.maxw_out = cv.take<int32_t>(m);
  w.acc.maxw_in = cv.take<int32_t>(m);
  w.acc.sumw_out = cv.take<unsigned long long>(m);
  w.acc.sumw_in = cv.take<unsigned long long>(m);
  w.acc.min_margin = cv.take<int32_t>(m);
  w.acc.max_margin = cv.take<int32_t>(m);
  w.acc.max_drow = cv.take<int32_t>(m);
  w.cnt14 = cv.take<int32_t>(m);
  w.cnt15 = cv.take<int32_t>(m);
  w.score = cv.take<float>(m);
  w.slot = cv.take<int32_t>(m);
  w.warm = cv.take<int32_t>(m);
  w.cand = cv.take<int32_t>(kMaxProposals);
  w.nwarm = cv.take<int32_t>(1);
  w.res = cv.take<int32_t>(4);
  const size_t cw = size_t(std::min<int32_t>(m, kCertifyMaxWarm));
  w.Ww = cv.take<int32_t>(cw * cw);
  w.Wt = cv.take<int32_t>(cw * cw);
  return w;
}

int features_into(schulze_ctx* ctx, const int32_t* d, int32_t m, int64_t n, float* feat, const LearnedWs& w,
                  cudaStream_t stream) {
  const int g = std::max(1, std::min((m + 255) / 256, 1024));
  {
    Launch L(ctx, stream, "learn_features_init", double(m) * 64.0);
    acc_init_kernel<<<g, 256, 0, stream>>>(w.acc, m, w.cnt14, w.cnt15);
  }
  {
    Launch L(ctx, stream, "learn_features", double(m) * double(m) * 4.0);
    const unsigned grid = unsigned((m + kFR - 1) / kFR) * kFChunks;
    const bool vec = m % 4 == 0 && reinterpret_cast<uintptr_t>(d) % 16 == 0;
    const int mode = n <= 32766 ? kFPacked : n < (int64_t(1) << 32) / (4 * kFSlabs) ? kFNarrow : kFWide;
    auto kern = vec ? (mode == kFPacked   ? features_pass_kernel<true, kFPacked>
                       : mode == kFNarrow ? features_pass_kernel<true, kFNarrow>
                                          : features_pass_kernel<true, kFWide>)
                    : (mode == kFPacked   ? features_pass_kernel<false, kFPacked>
                       : mode == kFNarrow ? features_pass_kernel<false, kFNarrow>
                                          : features_pass_kernel<false, kFWide>);
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kFSmem));
    kern<<<grid, 256, kFSmem, stream>>>(d, m, w.acc);
  }
  {
    Launch L(ctx, stream, "learn_features_finalize", double(m) * kNF * 4.0);
    features_finalize_kernel<<<(m + 63) / 64, 64, 0, stream>>>(w.acc, m, n, feat);
  }
  {
    Launch L(ctx, stream, "learn_feature_ranks", double(m) * 16.0);
    const unsigned nch = unsigned((m + kRankChunk - 1) / kRankChunk);
    features_rank_kernel<<<dim3(nch, nch, 2), kRankChunk / 2, 0, stream>>>(w.acc, m, w.cnt14, w.cnt15);
    features_rank_finalize_kernel<<<(m + 63) / 64, 64, 0, stream>>>(w.cnt14, w.cnt15, m, feat);
  }
  return check_launch();
}

int certify_launch(schulze_ctx* ctx, const int32_t* d, int32_t m, const int32_t* cand, int32_t ncand,
                   int32_t* winners, int32_t* res, const LearnedWs& w, int32_t* fwd, int32_t* bwd,
                   cudaStream_t stream, bool warm_listed = false) {
  if (!warm_listed) {
    Launch L(ctx, stream, "certify_warm_list", double(m) * 8.0);
    warm_list_kernel<<<1, 1024, 0, stream>>>(w.acc.wins, m, w.warm, w.slot, w.nwarm);
  }
  {
    const int64_t cw = std::min<int32_t>(m, kCertifyMaxWarm);
    const int blocks = int(std::max<int64_t>(1, std::min<int64_t>((cw * cw + 255) / 256, 4096)));
    Launch L(ctx, stream, "certify_warm_pack", double(cw) * double(cw) * 16.0);
    warm_pack_kernel<<<blocks, 256, 0, stream>>>(d, m, w.warm, w.nwarm, w.Ww, w.Wt);
  }
  {
    Launch L(ctx, stream, "certify_paths", 0.0);
    certify_kernel<<<1, 1024, 0, stream>>>(w.Ww, w.Wt, w.nwarm, w.warm, w.slot, w.acc.losses, m, cand, ncand, fwd,
                                           bwd, winners, res);
  }
  return check_launch();
}

}  // namespace
}  // namespace schulze

using namespace schulze;

extern "C" {

int schulze_features(schulze_ctx* ctx, const int32_t* d, int32_t m, int64_t n, float* feat, schulze_stream_t stream) {
  AbiRange abi_range("schulze_features");
  if (!ctx || !d || !feat || m < 1 || m > kMaxM || n < 0) return SCHULZE_EINVAL;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return SCHULZE_ECUDA;
  if (int rc = ensure_workspace(ctx, learned_ws_bytes(m), stream)) return rc;
  const LearnedWs w = carve_learned(ctx->ws.base, m);
  return features_into(ctx, d, m, n, feat, w, stream);
}

int schulze_mlp_forward(schulze_ctx* ctx, const float* params, const float* feat, int32_t N, float* score,
                        schulze_stream_t stream) {
  AbiRange abi_range("schulze_mlp_forward");
  if (!ctx || !params || !feat || !score || N < 0) return SCHULZE_EINVAL;
  if (N == 0) return SCHULZE_OK;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return SCHULZE_ECUDA;
  Launch L(ctx, stream, "mlp_forward", double(N) * 5248.0 * 2.0);
  mlp_forward_kernel<<<(N + kMlpThreads - 1) / kMlpThreads, kMlpThreads, 0, stream>>>(params, feat, N, score, nullptr,
                                                                                        nullptr);
  return check_launch();
}

int schulze_mlp_train_step(schulze_ctx* ctx, float* params, float* adam_m, float* adam_v, int64_t step,
                           const float* feat, const int32_t* label, const int32_t* seg_off, int32_t nseg, int32_t N,
                           float lr, float* loss, float* grad, schulze_stream_t stream) {
  AbiRange abi_range("schulze_mlp_train_step");
  if (!ctx || !params || !adam_m || !adam_v || step < 1 || !feat || !label || !seg_off || nseg < 1 || N < 1 ||
      !(lr >= 0.f))
    return SCHULZE_EINVAL;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return SCHULZE_ECUDA;
  const int32_t nchunks = (N + kChunk - 1) / kChunk;
  const size_t need = align_up(size_t(N) * 4, 256) * 2 + 2 * align_up(size_t(N) * kH * 4, 256) +
                      align_up(size_t(nchunks) * kNP * 4, 256) + align_up(size_t(nseg) * 4, 256) +
                      align_up(size_t(kNP) * 4, 256) + 4096;
  if (int rc = ensure_workspace(ctx, need, stream)) return rc;
  Carver cv(ctx->ws.base);
  float* score = cv.take<float>(N);
  float* ds = cv.take<float>(N);
  float* h1 = cv.take<float>(size_t(N) * kH);
  float* h2 = cv.take<float>(size_t(N) * kH);
  float* partial = cv.take<float>(size_t(nchunks) * kNP);
  float* seg_loss = cv.take<float>(nseg);
  float* g = grad ? grad : cv.take<float>(kNP);
  {
    Launch L(ctx, stream, "mlp_train_forward", double(N) * 5248.0 * 2.0);
    mlp_forward_kernel<<<(N + kMlpThreads - 1) / kMlpThreads, kMlpThreads, 0, stream>>>(params, feat, N, score, h1, h2);
  }
  {
    Launch L(ctx, stream, "mlp_train_loss", double(N) * 8.0);
    mlp_loss_kernel<<<nseg, 256, 0, stream>>>(score, label, seg_off, nseg, ds, seg_loss);
  }
  {
    Launch L(ctx, stream, "mlp_train_backward", double(N) * 5248.0 * 4.0);
    cudaFuncSetAttribute(mlp_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         int(sizeof(BackwardSmem)));
    mlp_backward_kernel<<<nchunks, 256, sizeof(BackwardSmem), stream>>>(params, feat, h1, h2, ds, N, partial);
    mlp_reduce_kernel<<<(kNP + 255) / 256, 256, 0, stream>>>(partial, nchunks, seg_loss, nseg, g, loss);
  }
  {
    Launch L(ctx, stream, "mlp_train_adam", double(kNP) * 16.0);
    adam_kernel<<<(kNP + 255) / 256, 256, 0, stream>>>(params, adam_m, adam_v, g, step, lr, 0.9f, 0.999f, 1e-8f);
  }
  return check_launch();
}

int schulze_certify(schulze_ctx* ctx, const int32_t* d, int32_t m, int64_t n, const int32_t* cand, int32_t ncand,
                    int32_t* winners, int32_t* result, schulze_stream_t stream) {
  AbiRange abi_range("schulze_certify");
  if (!ctx || !d || !cand || !winners || !result || m < 1 || m > kMaxM || n < 0 || ncand < 0 ||
      ncand > kMaxProposals)
    return SCHULZE_EINVAL;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return SCHULZE_ECUDA;
  const size_t need = learned_ws_bytes(m) + align_up(size_t(m) * kNF * 4, 256) + 2 * align_up(size_t(m) * 4, 256);
  if (int rc = ensure_workspace(ctx, need, stream)) return rc;
  const LearnedWs w = carve_learned(ctx->ws.base, m);
  Carver cv(static_cast<char*>(ctx->ws.base) + learned_ws_bytes(m));
  float* feat = cv.take<float>(size_t(m) * kNF);
  int32_t* fwd = cv.take<int32_t>(m);
  int32_t* bwd = cv.take<int32_t>(m);
  if (int rc = features_into(ctx, d, m, n, feat, w, stream)) return rc;  // wins / losses for the warm set
  return certify_launch(ctx, d, m, cand, ncand, winners, result, w, fwd, bwd, stream);
}

int schulze_winners_fast(schulze_ctx* ctx, const int32_t* d, int32_t m, int64_t n, const float* params, int32_t top,
                         int32_t* winners, int32_t* stats, schulze_stream_t stream) {
  AbiRange abi_range("schulze_winners_fast");
  if (!ctx || !d || !winners || m < 1 || m > kMaxM || n < 0 || top < 1 || top > kMaxProposals) return SCHULZE_EINVAL;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return SCHULZE_ECUDA;
  const size_t lw = learned_ws_bytes(m);
  const size_t need = lw + align_up(size_t(m) * kNF * 4, 256) + 2 * align_up(size_t(m) * 4, 256) + 4096;
  if (int rc = ensure_workspace(ctx, need, stream)) return rc;
  const LearnedWs w = carve_learned(ctx->ws.base, m);
  Carver cv(static_cast<char*>(ctx->ws.base) + lw);
  float* feat = cv.take<float>(size_t(m) * kNF);
  int32_t* fwd = cv.take<int32_t>(m);
  int32_t* bwd = cv.take<int32_t>(m);
  if (int rc = features_into(ctx, d, m, n, feat, w, stream)) return rc;
  {
    Launch L(ctx, stream, "proposal_scores", double(m) * 5248.0 * 2.0);
    if (params)
      mlp_forward_kernel<<<(m + kMlpThreads - 1) / kMlpThreads, kMlpThreads, 0, stream>>>(params, feat, m, w.score,
                                                                                          nullptr, nullptr);
    else
      copeland_score_kernel<<<std::max(1, std::min((m + 255) / 256, 1024)), 256, 0, stream>>>(w.acc, m, w.score);
  }
  {
    Launch L(ctx, stream, "proposal_topk", double(m) * 4.0);  // and the warm list
    propose_kernel<<<2, 1024, 0, stream>>>(w.score, m, std::min(top, m), w.cand, w.acc.wins, w.warm, w.slot,
                                          w.nwarm);
  }
  if (int rc = certify_launch(ctx, d, m, w.cand, std::min(top, m), winners, w.res, w, fwd, bwd, stream, true))
    return rc;
  int32_t res[4] = {0, -1, 0, 0};
  int32_t nwarm = 0;
  if (cudaMemcpyAsync(res, w.res, sizeof(res), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaMemcpyAsync(&nwarm, w.nwarm, sizeof(nwarm), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess)
    return SCHULZE_ECUDA;
  int32_t fallback = 0;
  if (!res[0] && nwarm > kCertifyMaxWarm) {
    // a warm set too large for the certification CTA (dense profiles): the
    // paper's propagation (Alg. 1-4) decides exactly, with O(m^2) passes
    // per round instead of the closure's O(nw^3)
    fallback = 2;
    if (int rc = ensure_workspace(ctx, propagation_workspace_bytes(m), stream)) return rc;
    int32_t ps[2] = {0, 0};
    if (int rc = winners_propagation_launch(ctx, d, m, false, winners, ps, ctx->ws.base, stream)) return rc;
  } else if (!res[0]) {
    // no proposal certified (or too many ties): the full closure decides,
    // on workspace memory after the certification data
    fallback = 1;
    const size_t mm4 = align_up(size_t(m) * size_t(m) * 4, 256);
    const size_t stage = std::max(closure_workspace_bytes(m, n, 0), extract_workspace_bytes(m));
    if (int rc = ensure_workspace(ctx, mm4 + stage + 4096, stream)) return rc;
    Carver c2(ctx->ws.base);
    int32_t* p = c2.take<int32_t>(size_t(m) * size_t(m));
    void* rest = c2.take<char>(0);
    if (int rc = closure_launch(ctx, d, m, n, p, 0, rest, stream)) return rc;
    if (int rc = extract_launch(ctx, p, m, winners, nullptr, nullptr, rest, stream)) return rc;
  }
  if (stats) {
    stats[0] = res[0] ? res[1] : -1;  // proposal index that certified
    stats[1] = fallback;
    stats[2] = res[2];  // ties checked
    stats[3] = res[3];  // Bellman-Ford rounds
  }
  return SCHULZE_OK;
}

}  // extern "C"
