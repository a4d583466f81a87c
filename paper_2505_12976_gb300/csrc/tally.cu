// Pairwise tally: d[i][j] = number of ballots that prefer i to j (Sect. 2.1).
//
// Two exact kernels, chosen by cost:
//  * dense  (position compare, O(n m^2)): ballots are turned into position
//    rows pos[v][c] (unlisted = k) and every (i, j) tile counts
//    pos[v][i] < pos[v][j] with packed 16-bit SIMD compares;
//  * sparse (pair count, O(n k^2)): d[i][j] = cnt[i] - C[i][j], where cnt[i]
//    is the number of ballots listing i and C[i][j] the number listing j
//    above i. C vanishes outside A x A, A the set of listed candidates.
//    - compact form (|A| small): each CTA counts C over A x A for its slice
//      of the ballots in a private shared-memory matrix, while d is filled
//      as if C were zero in one streaming pass; a second kernel sums the
//      slices and fixes the A x A entries of d;
//    - grouped form: ballot entries are grouped by candidate (counting
//      sort), and each CTA owns a block of rows of d, counts C for them in
//      shared memory and writes the rows of d once.
//    Which form runs is decided on the device once |A| is known.
#include <algorithm>

#include "count.cuh"
#include "internal.cuh"

namespace schulze {
namespace {

constexpr int kWarp = 32;
constexpr int32_t kLocalHistMax = 16384;  // candidates counted in shared memory per CTA
// compact pair count: |A| limits (16-bit packed / 32-bit counters), CTAs, threads
constexpr int32_t kCompactMaxPacked = 256;
constexpr int32_t kCompactMaxWide = 224;
constexpr int kCompactMaxCtas = 160;
constexpr int kCompactThreads = 1024;
constexpr uint16_t kNoSlot = 0xFFFFu;

// ------------------------------------------------------------------ dense

constexpr int kDenseVoters = 32;  // ballots staged in shared memory per step
constexpr int kMaxVoterChunk = 32768;  // 16-bit lane counters never overflow

// pos[v][c] for v in [v0, v0 + nv): position of c in ballot v, k if unlisted.
// One warp per ballot. Out-of-range ids and repeated ids set EDATA.
__global__ void pos_build_kernel(const int32_t* __restrict__ ranks, int64_t v0, int64_t nv, int32_t m, int32_t k,
                                 int32_t ldp, uint16_t* __restrict__ pos, int32_t* status) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t w = warp; w < nv; w += nwarps) {
    const int32_t* row = ranks + (v0 + w) * k;
    uint16_t* prow = pos + w * ldp;
    for (int32_t c = lane; c < ldp; c += kWarp) prow[c] = uint16_t(k);
    __syncwarp();
    for (int32_t q = lane; q < k; q += kWarp) {
      int32_t c = row[q];
      if (c >= 0 && c < m)
        prow[c] = uint16_t(q);
      else
        set_status(status, SCHULZE_EDATA);
    }
    __syncwarp();
    // a repeated id keeps only one of its positions: the other one sees it
    for (int32_t q = lane; q < k; q += kWarp) {
      int32_t c = row[q];
      if (c >= 0 && c < m && prow[c] != uint16_t(q)) set_status(status, SCHULZE_EDATA);
    }
    __syncwarp();
  }
}

// Weak orders in position form: pos[v][c] for v in [v0, v0 + nv) copied from
// the caller's int32 positions (smaller is better, equal is tied) into the
// 16-bit rows; a position outside [0, 65534] sets EDATA, one above 32767
// sets *wide. Padding columns (c >= m) hold 0x7FFF; their counts are never
// written.
__global__ void pos_copy_kernel(const int32_t* __restrict__ src, int64_t v0, int64_t nv, int32_t m, int32_t ldp,
                                uint16_t* __restrict__ pos, int32_t* status, int32_t* __restrict__ wide) {
  const int64_t total = nv * ldp;
  bool bad = false, big = false;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t w = e / ldp;
    const int32_t c = int32_t(e - w * ldp);
    uint16_t v = 0x7FFFu;
    if (c < m) {
      const int32_t x = src[(v0 + w) * m + c];
      bad |= x < 0 || x > 65534;
      big |= x > 32767;
      v = uint16_t(x < 0 ? 0 : (x > 65534 ? 65534 : x));
    }
    pos[e] = v;
  }
  if (bad) set_status(status, SCHULZE_EDATA);
  if (big) *wide = 1;  // positions need the 16-bit compare
}

// One CTA counts a TILE x TILE block of d over a chunk of ballots.
// Thread micro-tile RM x RN (RN even); lanes of a 32-bit word hold two
// adjacent j columns; the row operand is duplicated into both halves.
// Positions below 2^15 (guard_ok, and no wide position flagged in *wide)
// are compared with count_lt2, others with a packed 16-bit compare.
template <int TILE, int RM, int RN>
__global__ void __launch_bounds__((TILE / RM) * (TILE / RN))
    dense_tally_kernel(const uint16_t* __restrict__ pos, int32_t ldp, int64_t nv, int32_t m, int32_t nbt,
                       int32_t vchunk, int upper_only, int add, int guard_ok, const int32_t* __restrict__ wide,
                       int32_t* __restrict__ d) {
  const bool guard = guard_ok && !(wide && *wide);
  const uint32_t gbits = guard ? kGuard2 : 0u;
  constexpr int TX = TILE / RN, TY = TILE / RM, NT = TX * TY, WN = RN / 2;
  __shared__ __align__(16) uint32_t sI[kDenseVoters][TILE];      // row positions, duplicated
  __shared__ __align__(16) uint16_t sJ[kDenseVoters][TILE];      // column positions
  int32_t tile = blockIdx.x, bi, bj;
  if (upper_only) {  // enumerate bi <= bj
    bi = 0;
    int32_t rem = tile;
    while (rem >= nbt - bi) {
      rem -= nbt - bi;
      ++bi;
    }
    bj = bi + rem;
  } else {
    bi = tile / nbt;
    bj = tile % nbt;
  }
  const int32_t I0 = bi * TILE, J0 = bj * TILE;
  const int64_t vb = int64_t(blockIdx.y) * vchunk;
  const int64_t ve = min(nv, vb + vchunk);
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  uint32_t acc[RM][WN];
#pragma unroll
  for (int r = 0; r < RM; ++r)
#pragma unroll
    for (int w = 0; w < WN; ++w) acc[r][w] = 0u;

  for (int64_t v0 = vb; v0 < ve; v0 += kDenseVoters) {
    const int nvs = int(ve - v0 < kDenseVoters ? ve - v0 : int64_t(kDenseVoters));
    __syncthreads();
    for (int t = threadIdx.x; t < kDenseVoters * TILE; t += NT) {
      int vv = t / TILE, c = t % TILE;
      uint32_t pi = 0x7FFFu, pj = 0u;  // padding never counts: pi is not below pj
      if (vv < nvs) {
        const uint16_t* prow = pos + (v0 + vv) * ldp;
        pi = prow[I0 + c];
        pj = prow[J0 + c];
      }
      sI[vv][c] = pi | (pi << 16) | gbits;
      sJ[vv][c] = uint16_t(pj);
    }
    __syncthreads();
    for (int vv = 0; vv < nvs; ++vv) {
      uint32_t a[RM], b[WN];
#pragma unroll
      for (int r = 0; r < RM; r += 4) {
        uint4 t4 = *reinterpret_cast<const uint4*>(&sI[vv][ty * RM + r]);
        a[r] = t4.x, a[r + 1] = t4.y, a[r + 2] = t4.z, a[r + 3] = t4.w;
      }
#pragma unroll
      for (int w = 0; w < WN; w += 2) {
        uint2 t2 = *reinterpret_cast<const uint2*>(&sJ[vv][tx * RN + 2 * w]);
        b[w] = t2.x, b[w + 1] = t2.y;
      }
      if (guard) {
#pragma unroll
        for (int r = 0; r < RM; ++r)
#pragma unroll
          for (int w = 0; w < WN; ++w) acc[r][w] = count_lt2(acc[r][w], a[r], b[w]);
      } else {
#pragma unroll
        for (int r = 0; r < RM; ++r)
#pragma unroll
          for (int w = 0; w < WN; ++w) acc[r][w] = __vsub2(acc[r][w], __vcmpltu2(a[r], b[w]));
      }
    }
  }
  // lanes -> int32 counts (added atomically when several CTAs share a tile)
#pragma unroll
  for (int r = 0; r < RM; ++r) {
    int32_t i = I0 + ty * RM + r;
    if (i >= m) continue;
#pragma unroll
    for (int w = 0; w < WN; ++w) {
      int32_t j = J0 + tx * RN + 2 * w;
      int32_t lo = int32_t(acc[r][w] & 0xFFFFu), hi = int32_t(acc[r][w] >> 16);
      int32_t* dst = d + int64_t(i) * m + j;
      if (j < m) {
        if (add) atomicAdd(dst, lo); else dst[0] = lo;
      }
      if (j + 1 < m) {
        if (add) atomicAdd(dst + 1, hi); else dst[1] = hi;
      }
    }
  }
}

// Full rankings: d[j][i] = n - d[i][j]. Fills the strictly lower tiles from
// the upper ones (tiles of size TILE; the diagonal tiles are complete).
__global__ void mirror_kernel(int32_t* __restrict__ d, int32_t m, int32_t tile, int64_t n) {
  __shared__ int32_t s[32][33];
  const int32_t bi = blockIdx.y * 32, bj = blockIdx.x * 32;  // source block (rows bi.., cols bj..), bi < bj tile
  if ((bi / tile) >= (bj / tile)) return;  // only blocks inside strictly upper tiles
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int32_t i = bi + r, j = bj + threadIdx.x;
    s[r][threadIdx.x] = (i < m && j < m) ? d[int64_t(i) * m + j] : 0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int32_t i = bj + r, j = bi + threadIdx.x;  // destination (row in bj block, col in bi block)
    if (i < m && j < m) d[int64_t(i) * m + j] = int32_t(n) - s[threadIdx.x][r];
  }
}

// ----------------------------------------------------------------- sparse

// cnt[c] += 1 for every listed c; checks ids (range, repeats within a
// ballot via a per-warp bitmap in shared memory). One warp per ballot. With
// kLocal the CTA first counts in a shared-memory histogram and adds it to
// cnt once per candidate at the end (popular candidates would otherwise
// serialise on one global counter).
template <bool kLocal>
__global__ void sparse_count_kernel(const int32_t* __restrict__ ranks, int64_t n, int32_t m, int32_t k,
                                    int32_t* __restrict__ cnt, int32_t* status) {
  pdl_enter();
  extern __shared__ uint32_t smem_count[];  // [m] histogram if kLocal, then warps_per_block * words
  const int words = (m + 31) / 32;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint32_t* hist = smem_count;
  uint32_t* bm = smem_count + (kLocal ? m : 0) + wib * words;
  if (kLocal) {
    for (int32_t c = threadIdx.x; c < m; c += blockDim.x) hist[c] = 0u;
  }
  for (int t = lane; t < words; t += kWarp) bm[t] = 0u;
  __syncthreads();
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  if (k <= 32) {
    // ballots of at most 32 positions: a lane per position, the next two
    // ballots' ids in flight while this one is checked and counted
    auto id = [&](int64_t u) { return (u < n && lane < k) ? ranks[u * k + lane] : -1; };
    int32_t x0 = id(warp), x1 = id(warp + nwarps);
    const bool pa = lane < k;
    for (int64_t v = warp; v < n; v += nwarps) {
      const int32_t ca = x0;
      x0 = x1;
      x1 = id(v + 2 * nwarps);
      const bool oka = pa && ca >= 0 && ca < m;
      const uint32_t bita = 1u << (ca & 31);
      const uint32_t olda = oka ? atomicOr(&bm[ca >> 5], bita) : 0u;
      const bool fa = oka && !(olda & bita);  // first occurrence
      if (pa && !fa) set_status(status, SCHULZE_EDATA);  // out of range or repeated
      if (fa) {
        if (kLocal)
          atomicAdd(&hist[ca], 1u);
        else
          atomicAdd(&cnt[ca], 1);
      }
      __syncwarp();
      if (oka) bm[ca >> 5] = 0u;  // clear what this ballot set
      __syncwarp();
    }
  } else if (k <= 64) {
    // ballots of at most 64 positions: a lane holds positions lane and
    // lane + 32 in registers (also for clearing the bitmap), and the next
    // ballot's ids are loaded while this one is checked and counted
    auto ids = [&](int64_t u, int32_t& a, int32_t& b) {
      a = (u < n && lane < k) ? ranks[u * k + lane] : -1;
      b = (u < n && lane + 32 < k) ? ranks[u * k + lane + 32] : -1;
    };
    int32_t xa, xb;
    ids(warp, xa, xb);
    for (int64_t v = warp; v < n; v += nwarps) {
      const int32_t ca = xa, cb = xb;
      ids(v + nwarps, xa, xb);
      const bool pa = lane < k, pb = lane + 32 < k;
      const bool oka = pa && ca >= 0 && ca < m, okb = pb && cb >= 0 && cb < m;
      const uint32_t bita = 1u << (ca & 31), bitb = 1u << (cb & 31);
      const uint32_t olda = oka ? atomicOr(&bm[ca >> 5], bita) : 0u;
      const uint32_t oldb = okb ? atomicOr(&bm[cb >> 5], bitb) : 0u;
      const bool fa = oka && !(olda & bita), fb = okb && !(oldb & bitb);  // first occurrences
      if ((pa && !fa) || (pb && !fb)) set_status(status, SCHULZE_EDATA);  // out of range or repeated
      if (kLocal) {
        if (fa) atomicAdd(&hist[ca], 1u);
        if (fb) atomicAdd(&hist[cb], 1u);
      } else {
        if (fa) atomicAdd(&cnt[ca], 1);
        if (fb) atomicAdd(&cnt[cb], 1);
      }
      __syncwarp();
      if (oka) bm[ca >> 5] = 0u;  // clear what this ballot set
      if (okb) bm[cb >> 5] = 0u;
      __syncwarp();
    }
  } else
  for (int64_t v = warp; v < n; v += nwarps) {
    const int32_t* row = ranks + v * k;
    for (int32_t q0 = 0; q0 < k; q0 += kWarp) {
      int32_t q = q0 + lane;
      bool act = q < k;
      int32_t c = act ? row[q] : -1;
      bool ok = act && c >= 0 && c < m;
      if (act && !ok) set_status(status, SCHULZE_EDATA);
      if (ok) {
        uint32_t bit = 1u << (c & 31);
        uint32_t old = atomicOr(&bm[c >> 5], bit);
        if (old & bit)
          set_status(status, SCHULZE_EDATA);
        else if (kLocal)
          atomicAdd(&hist[c], 1u);
        else
          atomicAdd(&cnt[c], 1);
      }
    }
    __syncwarp();
    for (int32_t q = lane; q < k; q += kWarp) {  // clear what this ballot set
      int32_t c = row[q];
      if (c >= 0 && c < m) bm[c >> 5] = 0u;
    }
    __syncwarp();
  }
  if (kLocal) {
    __syncthreads();
    for (int32_t c = threadIdx.x; c < m; c += blockDim.x)
      if (hist[c]) atomicAdd(&cnt[c], int32_t(hist[c]));
  }
}

// Plans the sparse tally on the device, in two passes over tiles of
// kPlanTile candidates (one CTA per tile, a thread per candidate):
//  * off[c] / cursor[c]: start of candidate c's entries (exclusive scan of cnt);
//  * ord: the order in which the grouped form's rows kernel takes the rows
//    (longest first, by floor(log2(cnt)));
//  * slot[c]: index of c among the listed candidates (-1 if unlisted), act
//    the inverse, meta[0] = |A| and meta[1] = 1 when the compact form runs
//    (|A| <= compact_max). For the compact form the slots follow decreasing
//    cnt (ties by id): ballots drawn around a common order then list, in
//    their first positions, candidates whose slots lie close together, and
//    the pair counts of one position land in distinct shared-memory banks
//    (each slot of a 16-bit-packed row takes its own word in the first half
//    of the slots, see compact_pairs_kernel).
// The first pass sums each tile (listed candidates, entries, units of the
// heavy rows, rows per length bucket) into agg; the second combines the
// sums of the tiles before its own with its local scans and writes its
// candidates' entries of every table directly.
constexpr int kPlanTile = 1024;
constexpr int kAggWords = 40;  // listed, entries, heavy units, 34 bucket counts (padded)
constexpr int kBuckets = 34;   // 33: heavy (more than S entries); 1 .. 32: floor(log2(cnt)) + 1; 0: unlisted

__device__ __forceinline__ int plan_bucket(int32_t x, uint32_t S) {
  return uint32_t(x) > S ? 33 : (x > 0 ? 32 - __clz(x) : 0);
}

// ctr[key] += 1 for every lane, aggregated over the lanes with the same key
// (all 32 lanes call it); returns the old value plus the lane's rank among them
__device__ __forceinline__ uint32_t warp_bump(uint32_t* ctr, int key) {
  const int lane = threadIdx.x & 31;
  const uint32_t peers = __match_any_sync(0xFFFFFFFFu, key);
  const int leader = __ffs(peers) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(&ctr[key], uint32_t(__popc(peers)));
  return __shfl_sync(0xFFFFFFFFu, base, leader) + uint32_t(__popc(peers & ((1u << lane) - 1u)));
}

// sum over the block (kPlanTile threads) of v; valid in every thread
__device__ __forceinline__ uint32_t plan_block_sum(uint32_t v, uint32_t* ws) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  __syncthreads();  // ws free
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  uint32_t t = ws[threadIdx.x & 31];
#pragma unroll
  for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
  return t;
}

// exclusive scans over the block (kPlanTile threads, in thread order) of a and b
__device__ __forceinline__ void plan_block_scan2(uint32_t a, uint32_t b, uint32_t& ea, uint32_t& eb,
                                                 uint32_t (*ws)[32]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t ia = a, ib = b;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t ya = __shfl_up_sync(0xFFFFFFFFu, ia, o), yb = __shfl_up_sync(0xFFFFFFFFu, ib, o);
    if (lane >= o) ia += ya, ib += yb;
  }
  __syncthreads();  // ws free
  if (lane == 31) ws[0][wid] = ia, ws[1][wid] = ib;
  __syncthreads();
  if (wid == 0) {
    const uint32_t xa = ws[0][lane], xb = ws[1][lane];
    uint32_t sa = xa, sb = xb;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t ya = __shfl_up_sync(0xFFFFFFFFu, sa, o), yb = __shfl_up_sync(0xFFFFFFFFu, sb, o);
      if (lane >= o) sa += ya, sb += yb;
    }
    ws[0][lane] = sa - xa, ws[1][lane] = sb - xb;
  }
  __syncthreads();
  ea = ws[0][wid] + ia - a, eb = ws[1][wid] + ib - b;
}

__global__ void __launch_bounds__(kPlanTile) plan_tiles_kernel(const int32_t* __restrict__ cnt, int32_t m, uint32_t S,
                                                               uint32_t* __restrict__ agg) {
  pdl_enter();
  __shared__ uint32_t sb[kBuckets + 1];  // + a slot for the threads past m
  __shared__ uint32_t ws[32];
  if (threadIdx.x <= kBuckets) sb[threadIdx.x] = 0u;
  __syncthreads();
  const int32_t c = int32_t(blockIdx.x) * kPlanTile + int32_t(threadIdx.x);
  const int32_t x = c < m ? cnt[c] : 0;
  const int bk = c < m ? plan_bucket(x, S) : kBuckets;
  warp_bump(sb, bk);
  uint32_t* a = agg + size_t(blockIdx.x) * kAggWords;
  const uint32_t listed = plan_block_sum(x > 0 ? 1u : 0u, ws);
  const uint32_t entries = plan_block_sum(uint32_t(x), ws);
  const uint32_t units = plan_block_sum(bk == 33 ? (uint32_t(x) + S - 1) / S : 0u, ws);
  if (threadIdx.x == 0) a[0] = listed, a[1] = entries, a[2] = units;
  if (threadIdx.x < kBuckets) a[3 + threadIdx.x] = sb[threadIdx.x];
}

__global__ void __launch_bounds__(kPlanTile)
    plan_place_kernel(const int32_t* __restrict__ cnt, int32_t m, const uint32_t* __restrict__ agg, int32_t tiles,
                      uint32_t S, int32_t hcap, uint32_t* __restrict__ off, uint32_t* __restrict__ cursor,
                      int32_t* __restrict__ ord, int2* __restrict__ utab, int32_t* __restrict__ gmeta,
                      int32_t compact_max, int32_t* __restrict__ slot, int32_t* __restrict__ act,
                      int32_t* __restrict__ meta, int32_t* __restrict__ hint, int32_t* __restrict__ hint_valid) {
  pdl_enter();
  constexpr int kQ = 3 + kBuckets;   // quantities summed per tile
  __shared__ uint32_t before[kQ];    // over the tiles before this one
  __shared__ uint32_t all[kQ];       // over every tile
  __shared__ uint32_t bcur[kBuckets + 1];  // this tile's next ord position per bucket (+ a slot past m)
  __shared__ uint32_t ws[2][32];
  __shared__ uint32_t hnu[kPlanTile];  // units of this tile's heavy rows, by their order in ord
  const int32_t tile = int32_t(blockIdx.x);
  if (threadIdx.x < kQ) {
    uint32_t bf = 0, al = 0;
    for (int32_t t = 0; t < tiles; ++t) {
      const uint32_t v = agg[size_t(t) * kAggWords + threadIdx.x];
      bf += t < tile ? v : 0u;
      al += v;
    }
    before[threadIdx.x] = bf, all[threadIdx.x] = al;
  }
  __syncthreads();
  if (threadIdx.x == 0) {  // bucket starts: heavy rows first, then decreasing length
    uint32_t run = 0;
    for (int bk = kBuckets - 1; bk >= 0; --bk) {
      bcur[bk] = run + before[3 + bk];
      run += all[3 + bk];
    }
    bcur[kBuckets] = 0u;
  }
  const int32_t c = tile * kPlanTile + int32_t(threadIdx.x);
  const bool in = c < m;
  const int32_t x = in ? cnt[c] : 0;
  const bool listed = x > 0;
  uint32_t fl, ol;  // listed candidates and entries before c within the tile
  plan_block_scan2(listed ? 1u : 0u, uint32_t(x), fl, ol, ws);  // (its barriers also publish bcur)
  const uint32_t na = all[0], total = all[1];
  const uint32_t f = before[0] + fl;
  const bool compact = int32_t(na) <= compact_max;
  if (in) {
    if (hint) {
      // warm-first relabeling: listed c keeps rank f, unlisted c follows all
      // listed ones in id order
      const uint32_t nw = listed ? f : na + (uint32_t(c) - f);
      hint[m + int64_t(nw)] = c, hint[2 * int64_t(m) + c] = int32_t(nw), hint[c] = listed ? 1 : 0;
    }
    if (!compact) {
      slot[c] = listed ? int32_t(f) : -1;
      if (listed) act[f] = c;
    } else if (!listed) {
      slot[c] = -1;
    }
  }
  if (tile == 0 && threadIdx.x == 0) {
    meta[0] = int32_t(na), meta[1] = compact ? 1 : 0;
    if (hint) *hint_valid = na < uint32_t(m) ? 1 : 0, hint[3 * int64_t(m)] = int32_t(na);
  }
  if (compact) {
    // the compact form needs no grouping plan, only its slot order: CTA 0
    // collects the listed candidates and ranks them by (count desc, id asc)
    if (tile != 0) return;
    static_assert(kCompactMaxPacked >= kCompactMaxWide && kCompactMaxPacked * 4 <= kPlanTile, "4 threads per slot");
    __shared__ int32_t lid[kCompactMaxPacked];
    __shared__ int32_t lcnt[kCompactMaxPacked];
    __shared__ uint32_t nl;
    if (threadIdx.x == 0) nl = 0u;
    __syncthreads();
    for (int32_t c0 = 0; c0 < m; c0 += kPlanTile) {
      const int32_t cc = c0 + int32_t(threadIdx.x);
      const int32_t xc = cc < m ? cnt[cc] : 0;
      const bool lc = xc > 0;
      const uint32_t mask = __ballot_sync(0xFFFFFFFFu, lc);
      uint32_t base = 0;
      if ((threadIdx.x & 31) == 0 && mask) base = atomicAdd(&nl, uint32_t(__popc(mask)));
      base = __shfl_sync(0xFFFFFFFFu, base, 0);
      if (lc) {
        const uint32_t pos = base + uint32_t(__popc(mask & ((1u << (threadIdx.x & 31)) - 1u)));
        lid[pos] = cc, lcnt[pos] = xc;  // pos < na <= compact_max
      }
    }
    __syncthreads();
    const int32_t sl = int32_t(threadIdx.x >> 2), q = int32_t(threadIdx.x & 3);
    const bool own = sl < int32_t(na);
    const int32_t ci = own ? lid[sl] : 0, xi = own ? lcnt[sl] : 0;
    int32_t r = 0;  // listed candidates ahead of ci: larger count, or equal count and smaller id
#pragma unroll 8
    for (int32_t j = q; j < int32_t(na); j += 4) r += (lcnt[j] > xi || (lcnt[j] == xi && lid[j] < ci)) ? 1 : 0;
    r += __shfl_xor_sync(0xFFFFFFFFu, r, 1);
    r += __shfl_xor_sync(0xFFFFFFFFu, r, 2);
    if (own && q == 0) slot[ci] = r, act[r] = ci;
    return;
  }
  // grouped form: each candidate's entries start at off[c]. The rows kernel
  // takes its work from one queue: first the units of the heavy rows (more
  // than S entries; the first hcap of them in ord, each cut into units of S
  // entries, utab[u] = (index in ord, part)), then the other rows one by
  // one, in the order ord[]: heavy rows first, then by decreasing
  // floor(log2(cnt)), so that long rows start early and do not end the
  // kernel late. gmeta = {heavy rows split, units}.
  if (in) {
    const uint32_t o = before[1] + ol;
    off[c] = o, cursor[c] = o;
  }
  if (tile == 0 && threadIdx.x == 0) off[m] = total;
  const uint32_t hpre = bcur[33];  // this tile's first heavy row in ord (read before the bumps below)
  __syncthreads();
  const int bk = in ? plan_bucket(x, S) : kBuckets;
  const uint32_t t = warp_bump(bcur, bk);  // c's position in ord
  if (in) ord[t] = c;
  const uint32_t heavy = all[3 + 33], hs = min(heavy, uint32_t(hcap));
  const uint32_t nu = bk == 33 ? (uint32_t(x) + S - 1) / S : 0u;
  if (bk == 33) hnu[t - hpre] = nu;
  __syncthreads();
  const uint32_t htile = bcur[33] - hpre;  // this tile's heavy rows
  if (threadIdx.x < 32) {  // exclusive scan of hnu[0 .. htile) in place
    uint32_t carry = 0;
    for (uint32_t i0 = 0; i0 < htile; i0 += 32) {
      const uint32_t i = i0 + threadIdx.x;
      const uint32_t v = i < htile ? hnu[i] : 0u;
      uint32_t inc = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (int(threadIdx.x) >= o) inc += y;
      }
      if (i < htile) hnu[i] = carry + inc - v;
      carry += __shfl_sync(0xFFFFFFFFu, inc, 31);
    }
  }
  __syncthreads();
  if (bk == 33 && t < hs) {
    // the heavy rows before this tile's all lie below the cap when this one does
    const uint32_t u0 = before[2] + hnu[t - hpre];
    for (uint32_t q = 0; q < nu; ++q) utab[u0 + q] = make_int2(int32_t(t), int32_t(q));
    if (t == hs - 1 && heavy > hs) gmeta[1] = int32_t(u0 + nu);  // the cap cuts the heavy rows here
  }
  if (tile == 0 && threadIdx.x == 0) {
    gmeta[0] = int32_t(hs);
    if (heavy <= hs)
      gmeta[1] = int32_t(all[2]);  // every heavy row split
    else if (hs == 0)
      gmeta[1] = 0;
  }
}

// entries grouped by candidate: entries[cursor[c]++] = v * k + q. With kLocal
// (m <= kLocalHistMax, 1024 threads) each CTA takes a contiguous chunk of
// entries in rounds of kScatterHeld entries per thread (all their loads in
// flight at once): it counts the round per candidate in shared memory,
// reserves each candidate's slots with one global atomic (every thread
// issues all of its candidates' atomics before it uses their results; the
// returned base becomes the candidate's shared-memory cursor) and places
// the entries, reading the round's ids again (from L2).
constexpr int kScatterHeld = 28;
constexpr int kScatterThreads = 1024;
constexpr int kScatterResv = kLocalHistMax / kScatterThreads;  // candidates per thread in the reservations
static_assert(kLocalHistMax % (2 * kScatterThreads) == 0, "whole reservations per thread, in two halves");

template <bool kLocal>
__global__ void __launch_bounds__(1024) sparse_scatter_kernel(const int32_t* __restrict__ ranks, uint32_t total, int32_t m,
                                      uint32_t* __restrict__ cursor, uint32_t* __restrict__ entries,
                                      const int32_t* __restrict__ meta, const int32_t* __restrict__ gmeta,
                                      int32_t* __restrict__ hacc, uint32_t* __restrict__ hdone) {
  pdl_enter_early();
  if (meta[1]) return;  // compact form
  {
    // the split rows' accumulators and unit counters start at zero (the
    // rows kernel runs after this one)
    int4* h4 = reinterpret_cast<int4*>(hacc);  // 256-byte aligned rows of (m + 3) & ~3 words
    const int64_t hw4 = int64_t(gmeta[0]) * ((m + 3) / 4);
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < hw4; t += int64_t(gridDim.x) * blockDim.x)
      h4[t] = make_int4(0, 0, 0, 0);
    for (int32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < gmeta[0]; t += gridDim.x * blockDim.x) hdone[t] = 0u;
  }
  if (!kLocal) {
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
      int32_t c = ranks[e];
      if (c < 0 || c >= m) continue;  // already reported by the count pass
      uint32_t slot = atomicAdd(&cursor[c], 1u);
      entries[slot] = e;
    }
    return;
  }
  extern __shared__ uint32_t smem_scatter[];  // hist[m], cur[m]
  uint32_t* hist = smem_scatter;
  uint32_t* cur = smem_scatter + m;
  const uint32_t chunk = (total + gridDim.x - 1) / gridDim.x;
  const uint32_t e0 = min(total, blockIdx.x * chunk), e1 = min(total, e0 + chunk);
  for (int32_t c = threadIdx.x; c < m; c += blockDim.x) hist[c] = 0u;
  __syncthreads();
  constexpr uint32_t kRound = uint32_t(kScatterHeld) * kScatterThreads;
  for (uint32_t r0 = e0; r0 < e1; r0 += kRound) {
    {
      int32_t cv[kScatterHeld];
#pragma unroll
      for (int h = 0; h < kScatterHeld; ++h) {
        const uint32_t e = r0 + threadIdx.x + uint32_t(h) * kScatterThreads;
        cv[h] = e < e1 ? ranks[e] : -1;
      }
#pragma unroll
      for (int h = 0; h < kScatterHeld; ++h)
        if (cv[h] >= 0 && cv[h] < m) atomicAdd(&hist[cv[h]], 1u);
    }
    __syncthreads();
#pragma unroll
    for (int i0 = 0; i0 < kScatterResv; i0 += kScatterResv / 2) {  // two halves: eight atomics in flight
      uint32_t hv[kScatterResv / 2], bv[kScatterResv / 2];
#pragma unroll
      for (int i = 0; i < kScatterResv / 2; ++i) {
        const int32_t c = int32_t(threadIdx.x) + (i0 + i) * kScatterThreads;
        hv[i] = c < m ? hist[c] : 0u;
      }
#pragma unroll
      for (int i = 0; i < kScatterResv / 2; ++i)
        bv[i] = hv[i] ? atomicAdd(&cursor[int32_t(threadIdx.x) + (i0 + i) * kScatterThreads], hv[i]) : 0u;
#pragma unroll
      for (int i = 0; i < kScatterResv / 2; ++i) {
        const int32_t c = int32_t(threadIdx.x) + (i0 + i) * kScatterThreads;
        if (hv[i]) cur[c] = bv[i], hist[c] = 0u;
      }
    }
    __syncthreads();
    {
      int32_t cv[kScatterHeld];
#pragma unroll
      for (int h = 0; h < kScatterHeld; ++h) {
        const uint32_t e = r0 + threadIdx.x + uint32_t(h) * kScatterThreads;
        cv[h] = e < e1 ? __ldcg(ranks + e) : -1;
      }
#pragma unroll
      for (int h = 0; h < kScatterHeld; ++h)
        if (cv[h] >= 0 && cv[h] < m)
          entries[atomicAdd(&cur[cv[h]], 1u)] = r0 + threadIdx.x + uint32_t(h) * kScatterThreads;
    }
    __syncthreads();  // cur is read before the next round's reservations overwrite it
  }
}

// Grouped form: d[r][j] = cnt[r] - C[r][j] row by row, each row written
// once with streaming stores. C[r][.] is counted in shared memory as 16-bit
// counters, two columns per word (column j in the low half of word j / 2
// when j is even). The entries (v, q) of row r come from the grouping
// (entries[off[r] .. off[r+1]) hold v * k + q); each adds 1 to C[r][j] for
// every j listed above position q in ballot v. A counter never exceeds the
// entries counted into it (at most S <= 65535 per unit).
// A persistent CTA takes work from one queue (see plan_place_kernel):
//  * a unit of a heavy row (more than S entries) counts its slice of the
//    entries and adds its nonzero counters into the row's int32 accumulator
//    in global memory (L2-resident, reductions without return); the unit
//    that finishes last writes the row from the accumulator;
//  * any other row is counted and written by one CTA (a heavy row beyond the
//    accumulators in chunks of S entries: the first chunk writes d = cnt - C,
//    later ones subtract their counts from the written row).
// The write pass clears the counters it reads, ready for the next item.
constexpr int kRowsThreads = 256;

__global__ void __launch_bounds__(kRowsThreads, 5)
    grouped_rows_kernel(const int32_t* __restrict__ ranks, int32_t m, int32_t k, const int32_t* __restrict__ cnt,
                        const uint32_t* __restrict__ off, const uint32_t* __restrict__ entries,
                        const int32_t* __restrict__ ord, const int2* __restrict__ utab,
                        const int32_t* __restrict__ gmeta, uint32_t S, int32_t* __restrict__ hacc,
                        uint32_t* __restrict__ hdone, uint32_t* __restrict__ queue, int32_t* __restrict__ d,
                        int vec4, const int32_t* __restrict__ meta) {
  pdl_enter_early();
  if (meta[1]) return;  // compact form
  extern __shared__ __align__(16) uint32_t rows_smem[];
  uint32_t* C = rows_smem;
  __shared__ int32_t s_last;
  const int32_t wpr = (m + 1) >> 1;
  const int32_t hld = (m + 3) & ~3;  // accumulator row stride
  const int32_t hs = gmeta[0], units = gmeta[1];
  const uint32_t items = uint32_t(units) + uint32_t(m - hs);
  for (int32_t w = threadIdx.x; w < wpr; w += blockDim.x) C[w] = 0u;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  auto count = [&](int32_t j) {
    if (uint32_t(j) < uint32_t(m)) atomicAdd(&C[j >> 1], 1u << ((j & 1) * 16));
  };
  // C += the prefixes of entries [c0, c1). A warp takes 32 entries (one per
  // lane; entry e is position q = e mod k of its ballot, whose q prefix
  // positions are counted) and numbers their (entry, prefix position) pairs
  // consecutively with an inclusive scan of q over the lanes; each lane then
  // takes every 32nd pair, finding its entry by a binary search over the
  // scan. Every lane does useful work whatever the mix of q (the lanes of a
  // short prefix would otherwise idle), and a long prefix is still read by
  // consecutive lanes. kU pairs per lane are in flight at a time.
  auto count_range = [&](uint32_t c0, uint32_t c1) {
    constexpr int kU = 4;
    for (uint32_t base = c0 + 32u * wib; base < c1; base += 32u * nwarp) {
      const uint32_t t = base + lane;
      const uint32_t e = t < c1 ? entries[t] : 0u;
      const int32_t q = t < c1 ? int32_t(e % uint32_t(k)) : 0;
      const uint32_t first = e - uint32_t(q);  // the ballot's first position
      int32_t incl = q;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
      }
      const int32_t excl = incl - q, total = __shfl_sync(0xFFFFFFFFu, incl, 31);
      for (int32_t f0 = 0; f0 < total; f0 += 32 * kU) {
        int32_t jv[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int32_t f = f0 + 32 * u + lane;
          // s = the number of lanes whose pairs all lie below f (at most 31
          // when f < total): pair f belongs to lane s's entry
          int s = 0;
#pragma unroll
          for (int step = 16; step; step >>= 1) {
            const int32_t v = __shfl_sync(0xFFFFFFFFu, incl, s + step - 1);
            if (v <= f) s += step;
          }
          const int32_t ex = __shfl_sync(0xFFFFFFFFu, excl, s);
          const uint32_t st = __shfl_sync(0xFFFFFFFFu, first, s);
          jv[u] = f < total ? ranks[st + uint32_t(f - ex)] : -1;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) count(jv[u]);
      }
    }
  };
  // d[r][.] = base - C (first) or d[r][.] -= C; acc adds an int32 row of
  // counts (the accumulator of a split row); counters cleared
  auto write_row = [&](int32_t r, int32_t base, bool first, const int32_t* acc) {
    int32_t* drow = d + int64_t(r) * m;
    if (vec4) {
      for (int32_t g = threadIdx.x; g < (m >> 2); g += blockDim.x) {
        const int32_t j = 4 * g;
        uint2* cw = reinterpret_cast<uint2*>(C + (j >> 1));
        const uint2 w = *cw;
        *cw = make_uint2(0u, 0u);
        int4* dst = reinterpret_cast<int4*>(drow + j);
        int4 v = first ? make_int4(base, base, base, base) : __ldcs(dst);
        v.x -= int32_t(w.x & 0xFFFFu), v.y -= int32_t(w.x >> 16);
        v.z -= int32_t(w.y & 0xFFFFu), v.w -= int32_t(w.y >> 16);
        if (acc) {
          const int4 a = __ldcg(reinterpret_cast<const int4*>(acc + j));
          v.x -= a.x, v.y -= a.y, v.z -= a.z, v.w -= a.w;
        }
        if (first && r >= j && r < j + 4) {
          const int32_t t = r - j;
          v.x = t == 0 ? 0 : v.x, v.y = t == 1 ? 0 : v.y, v.z = t == 2 ? 0 : v.z, v.w = t == 3 ? 0 : v.w;
        }
        __stcs(dst, v);
      }
    } else {
      for (int32_t w = threadIdx.x; w < wpr; w += blockDim.x) {
        const uint32_t cw = C[w];
        C[w] = 0u;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int32_t j = 2 * w + h;
          if (j >= m) break;
          const int32_t c = int32_t((cw >> (16 * h)) & 0xFFFFu) + (acc ? __ldcg(acc + j) : 0);
          if (first)
            drow[j] = j == r ? 0 : base - c;
          else if (c)
            drow[j] -= c;
        }
      }
    }
  };
  // Thread 0 fetches the next work item while the CTA works on the current
  // one (queue slot at the start of the item, its row after the counting,
  // the row's offsets and count after the write), so that the dependent
  // global round trips of the queue do not stall the CTA between items. The
  // item is handed over through a double buffer: the buffer written during
  // item i is read at the start of item i + 1 and rewritten only during
  // item i + 2, after every thread has passed the barrier that starts i + 1.
  __shared__ int32_t s_next[2][6];  // row, part, index in ord, e0, e1, cnt (row -1: no more work)
  auto resolve = [&](uint32_t u, int32_t& r, int32_t& part, int32_t& t) {
    r = -1, part = -1, t = -1;
    if (u < uint32_t(units)) {
      const int2 ut = utab[u];
      t = ut.x, part = ut.y, r = ord[t];
    } else if (u < items) {
      t = hs + int32_t(u - uint32_t(units)), r = ord[t];
    }
  };
  auto publish = [&](int buf, int32_t r, int32_t part, int32_t t) {
    s_next[buf][0] = r, s_next[buf][1] = part, s_next[buf][2] = t;
    if (r >= 0) {
      s_next[buf][3] = int32_t(off[r]), s_next[buf][4] = int32_t(off[r + 1]), s_next[buf][5] = cnt[r];
    }
  };
  if (threadIdx.x == 0) {
    int32_t r, part, t;
    resolve(atomicAdd(queue, 1u), r, part, t);
    publish(0, r, part, t);
  }
  for (int it = 0;; ++it) {
    __syncthreads();  // the item is published; counters cleared (first pass) / by the last write
    const int cur = it & 1;
    const int32_t r = s_next[cur][0], part = s_next[cur][1], t = s_next[cur][2];
    if (r < 0) return;
    const uint32_t e0 = uint32_t(s_next[cur][3]), e1 = uint32_t(s_next[cur][4]);
    const int32_t cb = s_next[cur][5];
    uint32_t u_next = 0;
    int32_t r_n = -1, part_n = -1, t_n = -1;
    if (threadIdx.x == 0) u_next = atomicAdd(queue, 1u);
    auto after_count = [&]() {
      if (threadIdx.x == 0) resolve(u_next, r_n, part_n, t_n);
    };
    auto after_write = [&]() {
      if (threadIdx.x == 0) publish(cur ^ 1, r_n, part_n, t_n);
    };
    if (part >= 0) {
      // a unit of a split row
      const uint32_t c0 = e0 + uint32_t(part) * S, c1 = min(e1, c0 + S);
      count_range(c0, c1);
      __syncthreads();
      after_count();
      int32_t* acc = hacc + int64_t(t) * hld;
      for (int32_t w = threadIdx.x; w < wpr; w += blockDim.x) {
        const uint32_t cw = C[w];
        if (!cw) continue;
        C[w] = 0u;
        if (cw & 0xFFFFu) atomicAdd(acc + 2 * w, int32_t(cw & 0xFFFFu));
        if (cw >> 16) atomicAdd(acc + 2 * w + 1, int32_t(cw >> 16));
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t nu = (uint32_t(cb) + S - 1) / S;
        s_last = atomicAdd(hdone + t, 1u) == nu - 1 ? 1 : 0;
      }
      __syncthreads();
      if (s_last) {  // every unit's counts are in the accumulator
        __threadfence();
        write_row(r, cb, true, acc);
      }
      after_write();
    } else {
      // a whole row (chunks of S entries for a heavy row beyond the accumulators)
      uint32_t c0 = e0;
      bool fetched = false;
      do {
        const uint32_t c1 = min(e1, c0 + S);
        count_range(c0, c1);
        __syncthreads();
        if (!fetched) after_count(), fetched = true;
        write_row(r, cb, c0 == e0, nullptr);
        c0 = c1;
        if (c0 < e1) __syncthreads();  // the next chunk counts into cleared counters
      } while (c0 < e1);
      after_write();
    }
  }
}

// Compact form, first kernel (one CTA per slice of the ballots), its warps
// split between two jobs that run side by side:
// (a) kFillWarps warps fill the CTA's rows of d as if C were zero: d[i][j] =
//     cnt[i] for listed i and j != i, else 0 (stores, bound by HBM);
// (b) the others count C over A x A for the slice in shared memory (cell
//     [slot i][slot j], 16-bit lanes packed two per word when a slice has at
//     most 65535 ballots, slot j < hw in the low half of word j and slot
//     j >= hw in the high half of word j - hw, hw = ceil(|A| / 2) words per
//     row; else 32-bit; bound by shared-memory atomics) and store it as this
//     CTA's partial.
// Counting: a warp per ballot, its slots staged in shared memory; for every
// position q the lanes add 1 to C[slot at q][slot at p] for p < q, so the
// lanes of one atomic always hit distinct counters (ballots drawn around a
// common order would make lanes on different ballots collide). Ids outside
// [0, m) are skipped (the count pass reports them).
constexpr int kFillWarps = 4;

// *addr += v at a shared-memory byte address. Always issued: a predicated
// shared-memory reduction costs about two extra branch-unit instructions,
// so lanes with nothing to count add to a word of their own instead.
__device__ __forceinline__ void red_shared(uint32_t addr, uint32_t v) {
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// Counter of slot sp in a row: 16-bit packed, slot sp < hw in the low half
// of word sp, slot sp >= hw in the high half of word sp - hw (hw = words per
// row), so that nearby slots take distinct words; else word sp.
template <bool kPacked>
__device__ __forceinline__ uint32_t slot_word(uint32_t sp, uint32_t hw) {
  return kPacked ? (sp < hw ? sp : sp - hw) : sp;
}
template <bool kPacked>
__device__ __forceinline__ uint32_t slot_inc(uint32_t sp, uint32_t hw) {
  return kPacked ? (sp < hw ? 1u : 0x10000u) : 1u;
}
template <bool kPacked>
__device__ __forceinline__ void count_pair(uint32_t* crow, uint32_t sp, uint32_t hw) {
  atomicAdd(crow + slot_word<kPacked>(sp, hw), slot_inc<kPacked>(sp, hw));
}

template <bool kPacked>
__global__ void __launch_bounds__(kCompactThreads, 1)
    compact_pairs_kernel(const int32_t* __restrict__ ranks, int64_t n, int32_t m, int32_t k,
                         const int32_t* __restrict__ cnt, const int32_t* __restrict__ slot,
                         const int32_t* __restrict__ meta, uint32_t* __restrict__ partial, int32_t stage_len,
                         int32_t* __restrict__ d, int vec4) {
  pdl_enter();
  if (!meta[1]) return;  // the grouped form runs instead
  extern __shared__ __align__(16) uint32_t smem_pairs[];
  const int32_t na = meta[0];
  const int32_t wpr = kPacked ? (na + 1) >> 1 : na;
  const uint32_t hw = uint32_t(wpr);
  const int32_t words = na * wpr;
  uint32_t* C = smem_pairs;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  uint16_t* stage = reinterpret_cast<uint16_t*>(smem_pairs + ((words + 3) & ~3));
  for (int32_t t = threadIdx.x; t < words; t += blockDim.x) C[t] = 0u;
  __syncthreads();

  if (wib < kFillWarps) {
    // (a) this CTA's rows of d, 16 bytes per store where rows allow it
    const int ft = threadIdx.x, nft = kFillWarps * 32;
    const int32_t rper = (m + gridDim.x - 1) / gridDim.x;
    const int32_t i0 = min(m, int32_t(blockIdx.x) * rper), i1 = min(m, i0 + rper);
    for (int32_t i = i0; i < i1; ++i) {
      const int32_t b = slot[i] < 0 ? 0 : cnt[i];
      int32_t* drow = d + int64_t(i) * m;
      if (vec4) {  // rows of d start on 16-byte boundaries
        for (int32_t j = 4 * ft; j < m; j += 4 * nft) {
          const int32_t t = i - j;  // diagonal lane inside the 4 entries, if any
          *reinterpret_cast<int4*>(drow + j) =
              make_int4(t == 0 ? 0 : b, t == 1 ? 0 : b, t == 2 ? 0 : b, t == 3 ? 0 : b);
        }
      } else {
        for (int32_t j = ft; j < m; j += nft) drow[j] = j == i ? 0 : b;
      }
    }
  } else {
    // (b) pair counts of this CTA's ballots
    const int64_t vper = (n + gridDim.x - 1) / gridDim.x;
    const int64_t v0 = min(n, int64_t(blockIdx.x) * vper), v1 = min(n, v0 + vper);
    const int cw = wib - kFillWarps;  // counting warp
    if (k <= 64) {
      // Ballots of at most 64 positions: the slots stay in registers (p =
      // lane, lane + 32) and the next ballot's ids are loaded while this one
      // is counted.
      const int ncw = nwarp - kFillWarps;
      constexpr uint32_t kAll = 0xFFFFFFFFu;
      auto slot_of = [&](int32_t c) -> uint32_t {
        const int32_t sc = (c >= 0 && c < m) ? slot[c] : -1;
        return sc < 0 ? uint32_t(kNoSlot) : uint32_t(sc);
      };
      const int32_t qlo = min(k, 32), qhi = k;
      // two ballots ahead: ids of ballot v + 2 ncw in flight, slots of
      // ballot v + ncw being gathered, while ballot v is counted
      auto ids = [&](int64_t u, int32_t& a, int32_t& b) {
        a = (u < v1 && lane < k) ? ranks[u * k + lane] : -1;
        b = (u < v1 && lane + 32 < k) ? ranks[u * k + lane + 32] : -1;
      };
      int64_t v = v0 + cw;
      int32_t c0, c1, n0, n1;
      ids(v, c0, c1);
      ids(v + ncw, n0, n1);
      uint32_t s0 = lane < k ? slot_of(c0) : uint32_t(kNoSlot);
      uint32_t s1 = lane + 32 < k ? slot_of(c1) : uint32_t(kNoSlot);
      for (; v < v1; v += ncw) {
        const uint32_t r0 = s0, r1 = s1;
        s0 = lane < k ? slot_of(n0) : uint32_t(kNoSlot);
        s1 = lane + 32 < k ? slot_of(n1) : uint32_t(kNoSlot);
        ids(v + 2 * ncw, n0, n1);
        const bool clean = (lane >= k || r0 != kNoSlot) && (lane + 32 >= k || r1 != kNoSlot);
        if (__all_sync(kAll, clean)) {  // every id valid (the usual case): no per-entry checks
          // shared-memory byte addresses of this lane's counters in row 0 and
          // the row stride; a lane not above position q adds to its own word
          // of the (here unused) staging area instead (distinct banks, no
          // branch)
          const uint32_t w0 = slot_word<kPacked>(r0, hw), w1 = slot_word<kPacked>(r1, hw);
          const uint32_t i0 = slot_inc<kPacked>(r0, hw), i1 = slot_inc<kPacked>(r1, hw);
          const uint32_t cbase = uint32_t(__cvta_generic_to_shared(C)), rstride = uint32_t(wpr) * 4u;
          const uint32_t a0 = cbase + w0 * 4u, a1 = cbase + w1 * 4u;
          const uint32_t sink = uint32_t(__cvta_generic_to_shared(stage)) + uint32_t(lane) * 4u;
#pragma unroll 4
          for (int32_t q = 1; q < qlo; ++q) {
            const uint32_t sq = __shfl_sync(kAll, r0, q);
            red_shared(lane < q ? a0 + sq * rstride : sink, i0);
          }
#pragma unroll 4
          for (int32_t q = 32; q < qhi; ++q) {
            const uint32_t row = __shfl_sync(kAll, r1, q - 32) * rstride;
            red_shared(a0 + row, i0);
            red_shared(lane + 32 < q ? a1 + row : sink, i1);
          }
          continue;
        }
        for (int32_t q = 1; q < qlo; ++q) {  // rows 1..31: lanes p < q
          const uint32_t sq = __shfl_sync(kAll, r0, q);
          if (sq == kNoSlot) continue;  // uniform over the warp
          if (lane < q && r0 != kNoSlot) count_pair<kPacked>(C + int32_t(sq) * wpr, r0, hw);
        }
        for (int32_t q = 32; q < qhi; ++q) {  // rows 32..63: all low lanes, high lanes p < q
          const uint32_t sq = __shfl_sync(kAll, r1, q - 32);
          if (sq == kNoSlot) continue;
          uint32_t* crow = C + int32_t(sq) * wpr;
          if (r0 != kNoSlot) count_pair<kPacked>(crow, r0, hw);
          if (lane + 32 < q && r1 != kNoSlot) count_pair<kPacked>(crow, r1, hw);
        }
      }
    } else {
      uint16_t* st = stage + cw * stage_len;
      const int ncw = nwarp - kFillWarps;
      for (int64_t v = v0 + cw; v < v1; v += ncw) {
        const int32_t* row = ranks + v * k;
        for (int32_t q = lane; q < k; q += 32) {
          const int32_t c = row[q];
          const int32_t sc = (c >= 0 && c < m) ? slot[c] : -1;
          st[q] = sc < 0 ? kNoSlot : uint16_t(sc);
        }
        __syncwarp();
        // this lane's two low positions (p = lane, lane + 32) in registers
        const uint32_t r0 = lane < k ? st[lane] : kNoSlot;
        const uint32_t r1 = lane + 32 < k ? st[lane + 32] : kNoSlot;
        const int32_t qlo = min(k, 32), qhi = min(k, 64);
        bool clean = (lane >= k || r0 != kNoSlot) && (lane + 32 >= k || r1 != kNoSlot);
        for (int32_t q = 64 + lane; q < k; q += 32) clean &= st[q] != kNoSlot;
        if (__all_sync(0xFFFFFFFFu, clean)) {  // every id valid (the usual case): no per-entry checks
          const uint32_t w0 = slot_word<kPacked>(r0, hw), w1 = slot_word<kPacked>(r1, hw);
          const uint32_t i0 = slot_inc<kPacked>(r0, hw), i1 = slot_inc<kPacked>(r1, hw);
#pragma unroll 4
          for (int32_t q = 1; q < qlo; ++q) {
            const uint32_t sq = __shfl_sync(0xFFFFFFFFu, r0, q);
            if (lane < q) atomicAdd(C + int32_t(sq) * wpr + w0, i0);
          }
#pragma unroll 4
          for (int32_t q = 32; q < qhi; ++q) {
            uint32_t* crow = C + int32_t(__shfl_sync(0xFFFFFFFFu, r1, q - 32)) * wpr;
            atomicAdd(crow + w0, i0);
            if (lane + 32 < q) atomicAdd(crow + w1, i1);
          }
          for (int32_t q = 64; q < k; ++q) {
            uint32_t* crow = C + int32_t(st[q]) * wpr;
            atomicAdd(crow + w0, i0);
            atomicAdd(crow + w1, i1);
            for (int32_t p = 64 + lane; p < q; p += 32) count_pair<kPacked>(crow, st[p], hw);
          }
          __syncwarp();
          continue;
        }
        for (int32_t q = 1; q < qlo; ++q) {  // rows 1..31: lanes p < q
          const uint32_t sq = __shfl_sync(0xFFFFFFFFu, r0, q);
          if (sq == kNoSlot) continue;  // uniform over the warp
          if (lane < q && r0 != kNoSlot) count_pair<kPacked>(C + int32_t(sq) * wpr, r0, hw);
        }
        for (int32_t q = 32; q < qhi; ++q) {  // rows 32..63: all low lanes, high lanes p < q
          const uint32_t sq = __shfl_sync(0xFFFFFFFFu, r1, q - 32);
          if (sq == kNoSlot) continue;
          uint32_t* crow = C + int32_t(sq) * wpr;
          if (r0 != kNoSlot) count_pair<kPacked>(crow, r0, hw);
          if (lane + 32 < q && r1 != kNoSlot) count_pair<kPacked>(crow, r1, hw);
        }
        for (int32_t q = 64; q < k; ++q) {  // long ballots
          const uint32_t sq = st[q];
          if (sq == kNoSlot) continue;
          uint32_t* crow = C + int32_t(sq) * wpr;
          if (r0 != kNoSlot) count_pair<kPacked>(crow, r0, hw);
          if (r1 != kNoSlot) count_pair<kPacked>(crow, r1, hw);
          for (int32_t p = 64 + lane; p < q; p += 32) {
            const uint32_t sp = st[p];
            if (sp != kNoSlot) count_pair<kPacked>(crow, sp, hw);
          }
        }
        __syncwarp();
      }
    }
  }
  __syncthreads();
  uint32_t* out = partial + int64_t(blockIdx.x) * words;
  for (int32_t t = threadIdx.x; t < words; t += blockDim.x) out[t] = C[t];
}

// Compact form, second kernel (one CTA per listed candidate a): sums row a of
// the partial counts over the G slices and sets d[act a][act b] = cnt - C for
// every listed b != a.
template <bool kPacked>
__global__ void __launch_bounds__(512)
    compact_fix_kernel(const uint32_t* __restrict__ partial, int32_t G, int32_t m, const int32_t* __restrict__ cnt,
                       const int32_t* __restrict__ act, const int32_t* __restrict__ meta, int32_t* __restrict__ d) {
  pdl_enter();
  if (!meta[1]) return;
  __shared__ uint32_t red[512][2];
  const int32_t na = meta[0];
  const int32_t wpr = kPacked ? (na + 1) >> 1 : na;
  const int64_t words = int64_t(na) * wpr;
  const int32_t groups = max(1, int32_t(blockDim.x) / max(wpr, 1));
  for (int32_t a = blockIdx.x; a < na; a += gridDim.x) {
    const int32_t gg = threadIdx.x / wpr, w = threadIdx.x - gg * wpr;
    uint32_t lo = 0, hi = 0;
    if (gg < groups) {
      const uint32_t* src = partial + int64_t(a) * wpr + w;
      int32_t g = gg;
      for (; g + 7 * groups < G; g += 8 * groups) {  // eight loads in flight
        uint32_t x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = src[int64_t(g + u * groups) * words];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          if (kPacked) {
            lo += x[u] & 0xFFFFu;
            hi += x[u] >> 16;
          } else {
            lo += x[u];
          }
        }
      }
      for (; g < G; g += groups) {
        const uint32_t x = src[int64_t(g) * words];
        if (kPacked) {
          lo += x & 0xFFFFu;
          hi += x >> 16;
        } else {
          lo += x;
        }
      }
    }
    red[threadIdx.x][0] = lo, red[threadIdx.x][1] = hi;
    __syncthreads();
    if (threadIdx.x < wpr) {
      for (int32_t g = 1; g < groups; ++g) lo += red[g * wpr + threadIdx.x][0], hi += red[g * wpr + threadIdx.x][1];
      const int32_t i = act[a];
      const int32_t base = cnt[i];
      int32_t* drow = d + int64_t(i) * m;
      const int32_t b0 = int32_t(threadIdx.x), b1 = b0 + wpr;  // word w: slots w and w + wpr (packed)
      if (b0 != a) drow[act[b0]] = base - int32_t(lo);
      if (kPacked && b1 < na && b1 != a) drow[act[b1]] = base - int32_t(hi);
    }
    __syncthreads();
  }
}

// Compact form limits for a launch over G CTAs: cmax = the largest |A| it
// takes (0: never), stage = per-warp staging entries (>= k), smem bytes.
struct CompactPlan {
  int G;
  bool packed;
  int32_t cmax, stage;
  size_t smem, partial_words;
};

CompactPlan compact_plan(int64_t n, int32_t m, int32_t k, int sms, uint32_t flags) {
  CompactPlan c;
  c.G = std::max(1, std::min(sms, kCompactMaxCtas));
  const int64_t per = (n + c.G - 1) / c.G;
  c.packed = per <= 65535;
  c.cmax = std::min<int32_t>(m, c.packed ? kCompactMaxPacked : kCompactMaxWide);
  if ((flags & SCHULZE_F_TALLY_GROUPED) || k > c.cmax) c.cmax = 0;
  c.stage = (std::max(c.cmax, 64) + 7) & ~7;
  const size_t wpr = c.packed ? size_t(c.cmax + 1) / 2 : size_t(c.cmax);
  const size_t words = size_t(c.cmax) * wpr;
  c.smem = align_up(words, 4) * 4 + size_t(kCompactThreads / 32) * size_t(c.stage) * 2;
  c.partial_words = size_t(c.G) * std::max<size_t>(words, 1);
  return c;
}

bool choose_dense(int64_t n, int32_t m, int32_t k, uint32_t flags) {
  if (flags & SCHULZE_F_TALLY_DENSE) return true;
  if (flags & SCHULZE_F_TALLY_SPARSE) return false;
  // dense costs ~ m^2 / 2 packed ops per ballot, sparse ~ 4 k^2 / 2
  return double(k) * double(k) * 4.0 > double(m) * double(m);
}

constexpr int kDenseTile = 128;

int32_t dense_tile(int32_t m) { return m <= 64 ? 64 : kDenseTile; }

int64_t dense_voter_chunk(int64_t n, int32_t m) {
  (void)m;
  return std::min<int64_t>(std::max<int64_t>(n, 1), 1 << 16);
}

// Position-compare tally over n ballots whose 16-bit position rows build()
// writes chunk by chunk: build(v0, nv, ldp, pos) fills rows v0 .. v0+nv-1.
// `full`: strict full orders, only the upper tiles are counted and mirrored.
template <class Build>
int dense_tally(schulze_ctx* ctx, int64_t n, int32_t m, bool full, bool guard_ok, int32_t* wide, int32_t* d,
                void* ws, cudaStream_t stream, Build build) {
  const size_t mm = size_t(m) * size_t(m) * sizeof(int32_t);
  const int sms = ctx->sm_count > 0 ? ctx->sm_count : 148;
  Carver cv(ws);
  const int32_t tile = dense_tile(m);
  const int32_t ldp = int32_t(align_up(size_t(m), size_t(tile)));
  const int32_t nbt = ldp / tile;
  const int32_t ntiles = full ? nbt * (nbt + 1) / 2 : nbt * nbt;
  const int64_t chunk = dense_voter_chunk(n, m);
  uint16_t* pos = cv.take<uint16_t>(size_t(chunk) * size_t(ldp));
  // voter split inside a chunk so that the grid covers the GPU about eight
  // times over: the CTAs stage positions between barriers, and several per
  // SM hide each other's staging (m = 1024, n = 20000: two per SM 2.57 ms for
  // weak orders, eight 1.71 ms; the partial counts go into d with atomics)
  int32_t vsplit = int32_t(std::max<int64_t>(1, (8LL * sms + ntiles - 1) / ntiles));
  vsplit = int32_t(std::min<int64_t>(vsplit, std::max<int64_t>(1, std::min<int64_t>(n, chunk) / 64)));
  const bool accumulate = vsplit > 1 || n > chunk;
  if (accumulate && cudaMemsetAsync(d, 0, mm, stream) != cudaSuccess) return SCHULZE_ECUDA;
  for (int64_t v0 = 0; v0 < n; v0 += chunk) {
    const int64_t nv = std::min<int64_t>(chunk, n - v0);
    int32_t vchunk = int32_t((nv + vsplit - 1) / vsplit);
    vchunk = std::min<int32_t>(vchunk, kMaxVoterChunk);
    const int32_t gy = int32_t((nv + vchunk - 1) / vchunk);
    build(v0, nv, ldp, pos);
    dim3 grid(ntiles, gy);
    // gy > 1 or several chunks: the kernel adds atomically into zeroed d
    Launch L(ctx, stream, "tally_dense", double(nv) * double(m) * double(m - 1) / (full ? 2.0 : 1.0));
    if (tile == 64)
      dense_tally_kernel<64, 8, 8><<<grid, 64, 0, stream>>>(pos, ldp, nv, m, nbt, vchunk, full ? 1 : 0,
                                                             accumulate ? 1 : 0, guard_ok ? 1 : 0, wide, d);
    else
      dense_tally_kernel<128, 8, 8><<<grid, 256, 0, stream>>>(pos, ldp, nv, m, nbt, vchunk, full ? 1 : 0,
                                                               accumulate ? 1 : 0, guard_ok ? 1 : 0, wide, d);
    if (int rc = check_launch()) return rc;
  }
  if (full && nbt > 1) {
    Launch L(ctx, stream, "tally_mirror", double(m) * double(m) * 4.0);
    dim3 g((m + 31) / 32, (m + 31) / 32), b(32, 8);
    mirror_kernel<<<g, b, 0, stream>>>(d, m, tile, n);
  }
  return check_launch();
}

}  // namespace

// Grouped form geometry: S entries per unit of a heavy row (about eight
// units per SM over all entries, 512 .. 65535 so that a unit's 16-bit
// counters cannot overflow), hcap rows with accumulators (every row with
// more than S entries, within 256 MB), the unit table's capacity.
constexpr int kSmsForSizing = 160;  // at least the SM count of the GPUs this runs on (GB300: 152)

struct GroupedPlan {
  uint32_t S;
  int32_t hcap, hld;
  int64_t utab_cap;
};

GroupedPlan grouped_plan(int64_t n, int32_t m, int32_t k, int sms) {
  GroupedPlan g;
  const uint64_t total = uint64_t(n) * uint64_t(k);
  g.S = uint32_t(std::min<uint64_t>(65535, std::max<uint64_t>(512, total / (uint64_t(std::max(sms, 1)) * 8))));
  g.hld = (m + 3) & ~3;
  const int64_t fit = std::max<int64_t>(1, (int64_t(1) << 26) / g.hld);
  g.hcap = int32_t(std::min<int64_t>(std::min<int64_t>(m, int64_t(total / g.S) + 1), fit));
  g.utab_cap = int64_t(total / g.S) + g.hcap + 1;
  return g;
}

size_t grouped_bytes(const GroupedPlan& g) {
  return align_up(size_t(g.utab_cap) * 8, 256) + 256 + align_up(size_t((g.hld + kPlanTile - 1) / kPlanTile) * kAggWords * 4, 256) +
         align_up(size_t(g.hcap) * size_t(g.hld) * 4, 256) + align_up(size_t(g.hcap) * 4, 256);
}

size_t tally_workspace_bytes(int64_t n, int32_t m, int32_t k, uint32_t flags) {
  if (choose_dense(n, m, k, flags)) {
    int32_t tile = dense_tile(m);
    size_t ldp = align_up(size_t(m), size_t(tile));
    return align_up(size_t(dense_voter_chunk(n, m)) * ldp * 2, 256) + 4096;
  }
  size_t total = size_t(n) * size_t(k);
  // partial counts for up to kCompactMaxCtas slices, either counter width
  const size_t cp = size_t(std::min(m, kCompactMaxPacked)), cw = size_t(std::min(m, kCompactMaxWide));
  const size_t partial_words = size_t(kCompactMaxCtas) * std::max(cp * ((cp + 1) / 2), cw * cw);
  return align_up(size_t(m) * 4, 256) + 2 * align_up((size_t(m) + 1) * 4, 256) + align_up(size_t(m) * 4, 256) +
         256 + align_up(total * 4, 256) + 2 * align_up(size_t(m) * 4, 256) + 256 + align_up(partial_words * 4, 256) +
         grouped_bytes(grouped_plan(n, m, k, kSmsForSizing)) + 4096;
}

int tally_launch(schulze_ctx* ctx, const int32_t* ranks, int64_t n, int32_t m, int32_t k, int32_t* d,
                 uint32_t flags, void* ws, cudaStream_t stream, int32_t* hint, int32_t* hint_valid) {
  const size_t mm = size_t(m) * size_t(m) * sizeof(int32_t);
  const bool sparse_path = n > 0 && k > 0 && !choose_dense(n, m, k, flags);
  // (the sparse path clears hint_valid with its counters)
  if (hint && !sparse_path && cudaMemsetAsync(hint_valid, 0, sizeof(int32_t), stream) != cudaSuccess)
    return SCHULZE_ECUDA;
  if (n == 0 || k == 0) {
    return cudaMemsetAsync(d, 0, mm, stream) == cudaSuccess ? SCHULZE_OK : SCHULZE_ECUDA;
  }
  const int sms = ctx->sm_count > 0 ? ctx->sm_count : 148;
  Carver cv(ws);
  if (choose_dense(n, m, k, flags)) {
    // strict full orders: d[j][i] = n - d[i][j]
    return dense_tally(ctx, n, m, k >= m - 1, k <= 32767, nullptr, d, ws, stream,
                       [&](int64_t v0, int64_t nv, int32_t ldp, uint16_t* pos) {
                         const int pb = int(std::min<int64_t>((nv + 7) / 8, int64_t(sms) * 16));
                         Launch L(ctx, stream, "tally_positions", double(nv) * (double(k) * 4.0 + double(ldp) * 2.0));
                         pos_build_kernel<<<pb, 256, 0, stream>>>(ranks, v0, nv, m, k, ldp, pos, ctx->status);
                       });
  }
  // sparse
  const uint32_t total = uint32_t(uint64_t(n) * uint64_t(k));
  int32_t* cnt = cv.take<int32_t>(size_t(m));
  uint32_t* off = cv.take<uint32_t>(size_t(m) + 1);
  uint32_t* cursor = cv.take<uint32_t>(size_t(m) + 1);
  int32_t* ord = cv.take<int32_t>(size_t(m));
  uint32_t* queue = cv.take<uint32_t>(1);
  uint32_t* entries = cv.take<uint32_t>(total);
  int32_t* slot = cv.take<int32_t>(size_t(m));
  int32_t* act = cv.take<int32_t>(size_t(m));
  int32_t* meta = cv.take<int32_t>(2);
  const CompactPlan cp = compact_plan(n, m, k, sms, flags);
  uint32_t* partial = cv.take<uint32_t>(cp.partial_words);
  const GroupedPlan gp = grouped_plan(n, m, k, std::min(sms, kSmsForSizing));  // within the sized workspace
  int2* utab = reinterpret_cast<int2*>(cv.take<char>(size_t(gp.utab_cap) * 8));
  int32_t* gmeta = cv.take<int32_t>(2);
  uint32_t* agg = cv.take<uint32_t>(size_t((m + kPlanTile - 1) / kPlanTile) * kAggWords);
  int32_t* hacc = cv.take<int32_t>(size_t(gp.hcap) * size_t(gp.hld));
  uint32_t* hdone = cv.take<uint32_t>(size_t(gp.hcap));
  {
    ZeroSpans z;
    z.p[0] = reinterpret_cast<uint32_t*>(cnt), z.words[0] = m;
    z.p[1] = reinterpret_cast<uint32_t*>(hint_valid), z.words[1] = hint ? 1 : 0;
    z.p[2] = queue, z.words[2] = 1;
    if (int rc = zero_async(ctx, z, stream)) return rc;
  }
  const bool local_hist = m <= kLocalHistMax;
  {
    const int threads = 512;
    const size_t smem = (local_hist ? size_t(m) * 4 : 0) + size_t(threads / 32) * size_t((m + 31) / 32) * 4;
    auto kern = local_hist ? sparse_count_kernel<true> : sparse_count_kernel<false>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess || per_sm < 1)
      per_sm = 1;
    // about one ballot per warp: the pass is bound by load latency
    const int blocks = int(std::max<int64_t>(1, std::min<int64_t>((n + 15) / 16, int64_t(sms) * per_sm)));
    Launch L(ctx, stream, "tally_count", double(total) * 4.0);
    launch_pdl(kern, dim3(blocks), dim3(threads), smem, stream, false, ranks, n, m, k, cnt, ctx->status);
  }
  {
    const int32_t tiles = (m + kPlanTile - 1) / kPlanTile;
    {
      Launch L(ctx, stream, "tally_plan", double(m) * 4.0);
      launch_pdl(plan_tiles_kernel, dim3(tiles), dim3(kPlanTile), 0, stream, false, static_cast<const int32_t*>(cnt),
                 m, gp.S, agg);
    }
    Launch L(ctx, stream, "tally_place", double(m) * 20.0);
    launch_pdl(plan_place_kernel, dim3(tiles), dim3(kPlanTile), 0, stream, false, static_cast<const int32_t*>(cnt), m,
               static_cast<const uint32_t*>(agg), tiles, gp.S, gp.hcap, off, cursor, ord, utab, gmeta, cp.cmax, slot,
               act, meta, hint, hint_valid);
  }
  if (cp.cmax > 0) {
    Launch L(ctx, stream, "tally_compact_pairs", double(m) * double(m) * 4.0 + double(total) * 4.0);
    auto kern = cp.packed ? compact_pairs_kernel<true> : compact_pairs_kernel<false>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(cp.smem));
    launch_pdl(kern, dim3(cp.G), dim3(kCompactThreads), cp.smem, stream, false, ranks, n, m, k,
               static_cast<const int32_t*>(cnt), static_cast<const int32_t*>(slot), static_cast<const int32_t*>(meta),
               partial, int32_t(cp.stage), d, rows_vec16(d, m));
  }
  if (cp.cmax > 0) {
    Launch L(ctx, stream, "tally_compact_fix", 0.0);
    auto kern = cp.packed ? compact_fix_kernel<true> : compact_fix_kernel<false>;
    launch_pdl(kern, dim3(std::min(cp.cmax, 2 * sms)), dim3(512), 0, stream, false,
               static_cast<const uint32_t*>(partial), int32_t(cp.G), m, static_cast<const int32_t*>(cnt),
               static_cast<const int32_t*>(act), static_cast<const int32_t*>(meta), d);
  }
  {
    Launch L(ctx, stream, "tally_group", double(total) * 8.0);
    if (local_hist) {
      const size_t smem = size_t(m) * 8;
      const int blocks = int(std::min<uint64_t>((uint64_t(total) + 4095) / 4096, uint64_t(sms)));
      cudaFuncSetAttribute(sparse_scatter_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      launch_pdl(sparse_scatter_kernel<true>, dim3(blocks), dim3(kScatterThreads), smem, stream, false, ranks, total, m, cursor,
                 entries, static_cast<const int32_t*>(meta), static_cast<const int32_t*>(gmeta), hacc, hdone);
    } else {
      const int blocks = int(std::min<uint64_t>((uint64_t(total) + 255) / 256, uint64_t(sms) * 16));
      launch_pdl(sparse_scatter_kernel<false>, dim3(blocks), dim3(256), 0, stream, false, ranks, total, m, cursor,
                 entries, static_cast<const int32_t*>(meta), static_cast<const int32_t*>(gmeta), hacc, hdone);
    }
  }
  if (int rc = check_launch()) return rc;
  {
    // persistent rows kernel: every CTA resident, rows from the plan's queue
    const size_t smem = align_up(size_t((m + 1) / 2) * 4, 16);
    cudaFuncSetAttribute(grouped_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    cudaFuncSetAttribute(grouped_rows_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                         int(cudaSharedmemCarveoutMaxShared));
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, grouped_rows_kernel, kRowsThreads, smem) !=
            cudaSuccess || per_sm < 1) {
      cudaGetLastError();
      per_sm = 1;
    }
    const int grid = int(std::min<int64_t>(int64_t(per_sm) * sms, m));
    Launch L(ctx, stream, "tally_rows", double(m) * double(m) * 4.0 + double(total) * 4.0);
    launch_pdl(grouped_rows_kernel, dim3(grid), dim3(kRowsThreads), smem, stream, false, ranks, m, k,
               static_cast<const int32_t*>(cnt), static_cast<const uint32_t*>(off),
               static_cast<const uint32_t*>(entries), static_cast<const int32_t*>(ord),
               static_cast<const int2*>(utab), static_cast<const int32_t*>(gmeta), gp.S, hacc, hdone, queue, d,
               rows_vec16(d, m), static_cast<const int32_t*>(meta));
  }
  return check_launch();
}

size_t tally_positions_workspace_bytes(int64_t n, int32_t m) {
  const int32_t tile = dense_tile(m);
  const size_t ldp = align_up(size_t(m), size_t(tile));
  return align_up(size_t(dense_voter_chunk(n, m)) * ldp * 2, 256) + 4096;
}

int tally_positions_launch(schulze_ctx* ctx, const int32_t* pos_in, int64_t n, int32_t m, int32_t* d, void* ws,
                           cudaStream_t stream) {
  if (n == 0) return cudaMemsetAsync(d, 0, size_t(m) * size_t(m) * 4, stream) == cudaSuccess ? SCHULZE_OK : SCHULZE_ECUDA;
  const int sms = ctx->sm_count > 0 ? ctx->sm_count : 148;
  // the flag word sits after the position rows in the workspace
  int32_t* wide = reinterpret_cast<int32_t*>(static_cast<char*>(ws) + tally_positions_workspace_bytes(n, m) - 256);
  if (cudaMemsetAsync(wide, 0, sizeof(int32_t), stream) != cudaSuccess) return SCHULZE_ECUDA;
  return dense_tally(ctx, n, m, false, true, wide, d, ws, stream,
                     [&](int64_t v0, int64_t nv, int32_t ldp, uint16_t* pos) {
                       const int g = int(std::max<int64_t>(1, std::min<int64_t>((nv * ldp + 255) / 256, int64_t(sms) * 8)));
                       Launch L(ctx, stream, "tally_positions_copy", double(nv) * double(m) * 4.0);
                       pos_copy_kernel<<<g, 256, 0, stream>>>(pos_in, v0, nv, m, ldp, pos, ctx->status, wide);
                     });
}

}  // namespace schulze
