// Widest paths, all pairs (Sect. 2.1 definition; Sect. 4 "straightforward
// algorithm" computing p(a, b) for every pair), as a blocked Floyd-Warshall
// in the (max, min) semiring.
//
// Edge weights are winning votes, w[i][j] = d[i][j] if d[i][j] > d[j][i]
// else 0. They are packed into a zero-padded square workspace W (int16 when
// every count fits in 15 bits, else int32) whose rows and columns follow a
// relabeling of the candidates: candidates with at least one outgoing edge
// first, then those without (ids kept in order inside each group). The
// closure commutes with relabeling, and rows without edges stay zero, so
// their tiles are never touched.
//
// Only the candidates with edges (the "warm" ones, nw of them) need work:
// rows of cold candidates are zero in W and in p. W holds the warm rows only
// (padded to whole tiles), over all relabeled columns; warm columns come
// first. The closure has two parts:
//   * the warm square (nw x nw): paths between warm candidates never pass a
//     cold one (no outgoing edges), so it is the closure of W restricted to
//     them: repeated squaring on one thread-block cluster for up to
//     kClusterMaxWarm warm candidates, else the persistent blocked
//     Floyd-Warshall kernel below;
//   * the cold columns: p[i][c] = max(w[i][c], max_x min(p[i][x], w[x][c]))
//     over warm x, one (max, min) product with the closed warm square.
//
// When the caller's tally says the warm candidates are exactly the listed
// ones of a top-k profile (hint), every cold column is the same vector: for
// an unlisted c and a listed x, d[x][c] = cnt[x] (every ballot listing x puts
// it above c) and d[c][x] = 0, so w[x][c] = cnt[x] for all such c. The cold
// product then reduces to one column u[i] = max(w[i][c], max_x min(p[i][x],
// w[x][c])), which p, W's cold columns and beaten_by take from there.
//
// The persistent warm-square closure runs in rounds of B = 64 candidates; round r
//   1. closes the diagonal tile (r, r) by plain Floyd-Warshall,
//   2. updates the row and column panels: X = max(X, D (x) X) / max(X, X (x) D)
//      with D the closed diagonal tile,
//   3. updates every other tile: X(i, j) = max(X, W(i, r) (x) W(r, j)),
// where (x) is the (max, min) product. Widths only grow and every value
// written is the width of a real path, so the order of the updates inside a
// phase does not matter and the result is the exact closure. An update whose
// operand tile is all zero cannot change anything and is skipped.
//
// All rounds run in ONE persistent cooperative launch: the CTAs take work
// items from a global queue in a fixed order in which the next round's
// diagonal and panel items come right after the current round's tiles in
// that row and column ("lookahead"), so they overlap the rest of the round.
// Each tile carries a progress word (rounds applied, plus a nonzero bit); an
// item waits (bounded, clock-limited spin) until the tiles it reads have
// reached its round. Every wait is on an item earlier in the queue, which a
// resident CTA already holds, so the schedule cannot deadlock.
#include <cooperative_groups.h>

#include <algorithm>
#include <mutex>
#include <type_traits>

#include "internal.cuh"
#include "tiles.cuh"
#include "scan.cuh"

namespace schulze {
namespace {

using tiles::kB;        // block / tile size
using tiles::kThreads;  // threads per CTA
using tiles::BlockBarrier;
using tiles::Ops;
using tiles::diag_closure;
using tiles::diag_closure_local;

constexpr uint32_t kNZ = 1u << 30;         // progress word: tile has a nonzero entry
constexpr uint32_t kRoundMask = kNZ - 1u;  // progress word: rounds applied
constexpr long long kSpinLimitCycles = 4000000000LL;  // ~2 s at 2 GHz, unless the context sets another

// ------------------------------------------------------------ relabel

// rowflag[i] = 1 iff candidate i has an outgoing edge (some j with
// d[i][j] > d[j][i]); also reports SCHULZE_EDATA for an entry outside
// [0, bound]. Each CTA takes 64 x 64 block pairs (A, B), A <= B: thread
// (r, c) holds d[A+r][B+c..c+3] and d[B+r][A+c..c+3] in registers (16-byte
// loads when rows are 16-byte aligned), both tiles go to shared memory, and
// each held entry is compared with its transposed partner from there.
constexpr int kFlagT = 64;
__global__ void __launch_bounds__(256) rowflag_kernel(const int32_t* __restrict__ d, int32_t m, int64_t bound,
                                                      int32_t* __restrict__ rowflag, int32_t* status,
                                                      const int32_t* __restrict__ hint_valid, int vec4) {
  pdl_enter_early();
  if (hint_valid && *hint_valid) return;  // the caller's tally already knows the flags
  __shared__ int32_t t1[kFlagT][kFlagT + 1], t2[kFlagT][kFlagT + 1];  // t1 = d[A.., B..], t2 = d[B.., A..]
  const int32_t nbt = (m + kFlagT - 1) / kFlagT;
  const int64_t npairs = int64_t(nbt) * (nbt + 1) / 2;
  const int lane = threadIdx.x & 31;
  const int rq = threadIdx.x >> 4, c4 = (threadIdx.x & 15) * 4;  // rows rq + 16 q, columns c4 .. c4 + 3
  const bool vec = vec4 != 0;  // rows of d start on 16-byte boundaries
  int32_t a = 0;           // pairs (a, b), a <= b, numbered row by row
  int64_t rowstart = 0;    // number of the pair (a, a)
  bool bad = false;
  for (int64_t t = blockIdx.x; t < npairs; t += gridDim.x) {
    while (t >= rowstart + (nbt - a)) rowstart += nbt - a, ++a;
    const int32_t A = a * kFlagT, B = (a + int32_t(t - rowstart)) * kFlagT;
    int32_t x1[4][4], x2[4][4];
    auto load = [&](int32_t R, int32_t Cc, int32_t (&x)[4][4]) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int32_t i = R + rq + 16 * q, j = Cc + c4;
        if (vec) {
          int4 v = make_int4(0, 0, 0, 0);
          if (i < m && j < m) v = __ldcs(reinterpret_cast<const int4*>(d + int64_t(i) * m + j));
          x[q][0] = v.x, x[q][1] = v.y, x[q][2] = v.z, x[q][3] = v.w;
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e) x[q][e] = (i < m && j + e < m) ? d[int64_t(i) * m + j + e] : 0;
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) bad |= x[q][e] < 0 || int64_t(x[q][e]) > bound;
      }
    };
    load(A, B, x1);
    if (A != B) load(B, A, x2);
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        t1[rq + 16 * q][c4 + e] = x1[q][e];
        if (A != B) t2[rq + 16 * q][c4 + e] = x2[q][e];
      }
    __syncthreads();
    // side 0: row A + r, columns B + c: edge when t1[r][c] > (t2 or t1)[c][r]
    // side 1: row B + r, columns A + c: edge when t2[r][c] > t1[c][r]
    const int32_t(*T)[kFlagT + 1] = A == B ? t1 : t2;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = rq + 16 * q;
      bool e0 = false, e1 = false;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int c = c4 + e;
        e0 |= (A + r != B + c) && x1[q][e] > T[c][r];
        if (A != B) e1 |= x2[q][e] > t1[c][r];
      }
      // padding entries are 0 on both sides, so they never count
      const uint32_t b0 = __ballot_sync(0xFFFFFFFFu, e0), b1 = __ballot_sync(0xFFFFFFFFu, e1);
      if ((lane & 15) == 0) {
        const uint32_t sh = lane & 16;
        if ((b0 >> sh) & 0xFFFFu) atomicOr(&rowflag[A + r], 1);
        if ((b1 >> sh) & 0xFFFFu) atomicOr(&rowflag[B + r], 1);
      }
    }
    __syncthreads();
  }
  if (bad) set_status(status, SCHULZE_EDATA);
}

// Stable partition: perm[new] = old, candidates with edges first; inv[old] = new.
// The flags come from rowflag_kernel; when the tally set *hint_valid it has
// written the relabeling of its own flags already, and this launch returns.
__global__ void __launch_bounds__(1024) relabel_kernel(const int32_t* __restrict__ rowflag, int32_t m,
                                                       int32_t* __restrict__ perm, int32_t* __restrict__ inv,
                                                       int32_t* __restrict__ warm_out,
                                                       const int32_t* __restrict__ hint_valid) {
  pdl_enter_early();
  __shared__ uint32_t part[33];
  extern __shared__ uint32_t relabel_smem[];  // m words when m <= kScanSmem
  if (hint_valid && *hint_valid) return;
  // rank[c] = 1 for warm c, scanned into the warm rank (in shared memory, or
  // in place in inv for long candidate lists)
  uint32_t* rank = m <= kScanSmem ? relabel_smem : reinterpret_cast<uint32_t*>(inv);
  for (int32_t c = threadIdx.x; c < m; c += blockDim.x) rank[c] = rowflag[c] ? 1u : 0u;
  __syncthreads();
  const int32_t warm = int32_t(block_exclusive_scan(rank, m, part));
  if (threadIdx.x == 0) *warm_out = warm;
  for (int32_t c = threadIdx.x; c < m; c += blockDim.x) {
    const int32_t before = int32_t(rank[c]);                 // warm candidates before c
    const int32_t nw = rowflag[c] ? before : warm + (c - before);  // cold ones keep their order
    perm[nw] = c;
    inv[c] = nw;
  }
}

// W[a][b] = w[perm[a]][perm[b]] for the warm rows a < 64 * nbr (0 outside
// m x m, on the diagonal and where d does not beat its transpose; w is d, or
// the margin d - d^T with `margin`). One CTA
// pass per row a: with x = perm[a], the threads walk b, reading d[x][perm b]
// (along row x) and d[perm b][x] (down column x); a warp that writes a
// nonzero sets the nonzero bit of its 64 x 64 tile's progress word.
//
// With the tally's flags (hint valid), a candidate y without edges is one no
// ballot lists, so d[y][x] = 0 and that read is skipped.
// With uniform cold columns only the square (b < 64 nbr) is written, and
// ucol[a] receives the cold columns' common value for row a.
template <typename E>
__global__ void __launch_bounds__(512) pack_kernel(const int32_t* __restrict__ d, int32_t m, int32_t mp,
                                                   const int32_t* __restrict__ perm, const int32_t* __restrict__ warm,
                                                   E* __restrict__ W, uint32_t* __restrict__ prog, int32_t nb,
                                                   const int32_t* __restrict__ hint,
                                                   const int32_t* __restrict__ hint_valid, int32_t* __restrict__ ucol,
                                                   int margin) {
  pdl_enter();
  const bool hv = hint_valid && *hint_valid;
  const int32_t rows = (*warm + kB - 1) / kB * kB;  // W rows to write
  const bool uc = hv && rows < m;                    // uniform cold columns beyond the square
  const int32_t bend = uc ? rows : mp;
  const int lane = threadIdx.x & 31;
  constexpr int kU = 8;  // columns per thread and pass, their loads issued together
  for (int32_t a = blockIdx.x; a < rows; a += gridDim.x) {
    E* wrow = W + int64_t(a) * mp;
    const int32_t x = a < m ? perm[a] : -1;
    const int32_t* drow = x >= 0 ? d + int64_t(x) * m : nullptr;
    if (uc && threadIdx.x == 0) ucol[a] = (x >= 0 && a < *warm) ? max(drow[perm[rows]], 0) : 0;
    for (int32_t b0 = 0; b0 < bend; b0 += kU * blockDim.x) {
      int32_t y[kU], v[kU], u[kU];
#pragma unroll
      for (int q = 0; q < kU; ++q) {
        const int32_t b = b0 + q * blockDim.x + threadIdx.x;
        y[q] = (x >= 0 && b < m && b < bend && b != a) ? perm[b] : -1;
      }
#pragma unroll
      for (int q = 0; q < kU; ++q) {
        v[q] = y[q] >= 0 ? drow[y[q]] : 0;
        u[q] = (y[q] >= 0 && !(hv && !hint[y[q]])) ? d[int64_t(y[q]) * m + x] : 0;
      }
#pragma unroll
      for (int q = 0; q < kU; ++q) {
        const int32_t b = b0 + q * blockDim.x + threadIdx.x;
        const int32_t out = v[q] > u[q] ? (margin ? v[q] - u[q] : v[q]) : 0;
        if (b < bend) wrow[b] = E(out);
        if (__any_sync(0xFFFFFFFFu, out != 0) && lane == 0) atomicOr(&prog[(a / kB) * nb + (b / kB)], kNZ);
      }
    }
  }
}

// p[x][y] = W[inv[x]][inv[y]] for warm x and y != x; every other entry 0
// (cold rows are written as zeros without reading W). One row per CTA pass.
template <typename E>
__global__ void __launch_bounds__(256) widen_kernel(const E* __restrict__ W, int32_t mp, int32_t m,
                                                    const int32_t* __restrict__ inv,
                                                    const int32_t* __restrict__ perm,
                                                    const int32_t* __restrict__ warm, int32_t* __restrict__ p,
                                                    const int32_t* __restrict__ hint_valid,
                                                    const int32_t* __restrict__ ucold, int vec4) {
  pdl_enter();
  const int32_t nw = *warm;
  const int32_t rows = (nw + kB - 1) / kB * kB;
  const bool uc = hint_valid && *hint_valid && rows < m;  // cold columns beyond the square: ucold[ix]
  // kR rows per pass: their relabeled indices are loaded together (lane r of
  // each warp holds row r's) instead of one dependent load per row
  constexpr int kR = 8;
  const int lane = threadIdx.x & 31;
  for (int32_t xb = blockIdx.x; xb < m; xb += kR * gridDim.x) {
    const int32_t xl = xb + lane * int32_t(gridDim.x);
    const int32_t ixl = (lane < kR && xl < m) ? inv[xl] : 0;
    for (int r = 0; r < kR; ++r) {
      const int32_t x = xb + r * int32_t(gridDim.x);
      if (x >= m) break;
      const int32_t ix = __shfl_sync(0xFFFFFFFFu, ixl, r);
      int32_t* prow = p + int64_t(x) * m;
      // a cold row is zero; with uniform cold columns a warm row is
      // ucold[ix] outside the square, whose columns (relabeled b < rows,
      // candidate perm[b]) come from W after the fill
      if (ix >= nw || uc) {
        const int32_t fill = ix >= nw ? 0 : ucold[ix];
        if (vec4) {
          for (int32_t y = 4 * threadIdx.x; y < m; y += 4 * blockDim.x)
            *reinterpret_cast<int4*>(prow + y) = make_int4(fill, fill, fill, fill);
        } else {
          for (int32_t y = threadIdx.x; y < m; y += blockDim.x) prow[y] = fill;
        }
        if (ix >= nw) continue;
        __syncthreads();  // the square's columns after the fill (the branch is the same in the whole CTA)
        const E* wrow = W + int64_t(ix) * mp;
        for (int32_t b = threadIdx.x; b < rows; b += blockDim.x) prow[perm[b]] = b == ix ? 0 : int32_t(wrow[b]);
        continue;
      }
      const E* wrow = W + int64_t(ix) * mp;
      if (vec4) {
        constexpr int kU = 4;  // int4 groups per thread and pass, loads issued together
        for (int32_t y0 = 0; y0 < m; y0 += 4 * kU * blockDim.x) {
          int4 iv[kU];
  #pragma unroll
          for (int q = 0; q < kU; ++q) {
            const int32_t y = y0 + 4 * (q * blockDim.x + threadIdx.x);
            iv[q] = y < m ? *reinterpret_cast<const int4*>(inv + y) : make_int4(0, 0, 0, 0);
          }
          int4 v[kU];
          const int32_t uv = uc ? ucold[ix] : 0;
          auto at = [&](int32_t iy) { return (uc && iy >= rows) ? uv : int32_t(wrow[iy]); };
  #pragma unroll
          for (int q = 0; q < kU; ++q) v[q] = make_int4(at(iv[q].x), at(iv[q].y), at(iv[q].z), at(iv[q].w));
  #pragma unroll
          for (int q = 0; q < kU; ++q) {
            const int32_t y = y0 + 4 * (q * blockDim.x + threadIdx.x);
            if (y >= m) continue;
            if (x >= y && x < y + 4) {
              const int32_t t = x - y;
              v[q].x = t == 0 ? 0 : v[q].x, v[q].y = t == 1 ? 0 : v[q].y;
              v[q].z = t == 2 ? 0 : v[q].z, v[q].w = t == 3 ? 0 : v[q].w;
            }
            *reinterpret_cast<int4*>(prow + y) = v[q];
          }
        }
      } else {
        for (int32_t y = threadIdx.x; y < m; y += blockDim.x) {
          const int32_t iy = inv[y];
          prow[y] = (y == x) ? 0 : (uc && iy >= rows) ? ucold[ix] : int32_t(wrow[iy]);
        }
      }
    }
  }
}

// ----------------------------------------------------- work queue

enum ItemKind : int32_t { kDiag = 0, kPanel = 1, kTile = 2 };
struct Item {
  int32_t kind, r, i, j;
};

// The candidates with outgoing edges occupy the first nbr tile rows after
// relabeling; the other rows of W are zero and stay zero, and a round over a
// block of them cannot change anything (min(x, 0) = 0). So rounds run over
// r < nbr and only tile rows i < nbr are updated. The queue is written for
// nc >= nbr tile columns (nbr * nbr * nc items); the closure runs it on the
// warm square (nc = nbr) and leaves the cold columns to cold_product_kernel.
//
// Queue order, stage by stage:
//   stage 0:             D(0) P(0) L(0)
//   stage s (1..nbr-1):  D(s) P(s) R(s-1) L(s)     (no L in the last one)
//   stage nbr:           R(nbr-1)
// D(r): diagonal tile; P(r): row panel (r, j != r) then column panel
// (i < nbr, i != r); L(r): round-r tiles that are the next round's panels
// (tile row r+1, then tile column r+1); R(r): the other round-r tiles.
struct Shape {
  int32_t nbr, nb;
  int64_t P, L, Rmid, Rlast;
};

__device__ __forceinline__ Shape make_shape(int32_t nbr, int32_t nb) {
  Shape sh;
  sh.nbr = nbr, sh.nb = nb;
  sh.P = int64_t(nb - 1) + (nbr - 1);
  sh.L = int64_t(nb - 1) + (nbr - 2);
  sh.Rmid = int64_t(nbr - 2) * (nb - 2);
  sh.Rlast = int64_t(nbr - 1) * (nb - 1);
  return sh;
}

__device__ __forceinline__ int64_t stage_size(int32_t s, const Shape& sh) {
  int64_t z = 0;
  if (s < sh.nbr) z += 1 + sh.P;
  if (s >= 1) z += (s - 1 < sh.nbr - 1) ? sh.Rmid : sh.Rlast;
  if (s < sh.nbr - 1) z += sh.L;
  return z;
}

__device__ Item decode_item(int64_t t, const Shape& sh) {
  const int32_t nbr = sh.nbr, nb = sh.nb;
  int32_t s;
  const int64_t s0 = stage_size(0, sh);
  if (t < s0) {
    s = 0;
  } else {
    t -= s0;
    const int64_t mid = int64_t(nbr) * nb;  // stages 1 .. nbr-2 all hold nbr * nb items
    const int64_t nmid = nbr >= 2 ? nbr - 2 : 0;
    if (t < nmid * mid) {
      s = 1 + int32_t(t / mid);
      t -= int64_t(s - 1) * mid;
    } else {
      t -= nmid * mid;
      s = 1 + int32_t(nmid);
      const int64_t z = stage_size(s, sh);
      if (t >= z) {
        t -= z;
        s += 1;
      }
    }
  }
  Item it{kDiag, 0, 0, 0};
  if (s < nbr) {
    if (t == 0) {
      it.kind = kDiag, it.r = s, it.i = s, it.j = s;
      return it;
    }
    t -= 1;
    if (t < sh.P) {
      it.kind = kPanel, it.r = s;
      if (t < nb - 1) {
        it.i = s, it.j = int32_t(t) + (t >= s);
      } else {
        const int32_t q = int32_t(t - (nb - 1));
        it.i = q + (q >= s), it.j = s;
      }
      return it;
    }
    t -= sh.P;
  }
  if (s >= 1) {
    const int32_t r = s - 1;
    it.kind = kTile, it.r = r;
    if (r == nbr - 1) {
      const int32_t wc = nb - 1;
      if (t < sh.Rlast) {
        const int32_t a = int32_t(t / wc), b = int32_t(t % wc);
        it.i = a + (a >= r), it.j = b + (b >= r);
        return it;
      }
      t -= sh.Rlast;
    } else {
      const int32_t wc = nb - 2;
      if (t < sh.Rmid) {
        const int32_t a = int32_t(t / wc), b = int32_t(t % wc);
        it.i = a < r ? a : a + 2;
        it.j = b < r ? b : b + 2;
        return it;
      }
      t -= sh.Rmid;
    }
  }
  const int32_t r = s;  // L(s)
  it.kind = kTile, it.r = r;
  if (t < nb - 1) {
    it.i = r + 1, it.j = int32_t(t) + (t >= r);
  } else {
    const int32_t q = int32_t(t - (nb - 1));
    it.i = q < r ? q : q + 2, it.j = r + 1;
  }
  return it;
}

struct Sync {
  uint32_t* prog;                // [nb * nb] progress words
  uint32_t* head;                // queue head
  uint32_t* abort_flag;          // set when a wait times out
  int32_t* status;
  const int32_t* warm;           // candidates with outgoing edges
  unsigned long long* counters;  // [0] tile updates done, [1] diagonal closures done, [2] items
  long long spin_limit;          // clock cycles a wait may take before it gives up
};

// Thread 0 waits until prog[idx] has applied at least `need` rounds; returns
// the word, or 0xFFFFFFFF after a timeout (which also raises the abort flag).
__device__ uint32_t wait_round(const Sync& sy, int32_t idx, uint32_t need) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(sy.prog + idx) : "memory");
    if ((v & kRoundMask) >= need) return v;
    if (*reinterpret_cast<volatile uint32_t*>(sy.abort_flag)) return 0xFFFFFFFFu;
    if (clock64() - t0 > sy.spin_limit) {
      set_status(sy.status, SCHULZE_ETIMEOUT);
      atomicExch(sy.abort_flag, 1u);
      return 0xFFFFFFFFu;
    }
    __nanosleep(64);
  }
}

__device__ __forceinline__ void publish(const Sync& sy, int32_t idx, uint32_t word) {
  __threadfence();
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(sy.prog + idx), "r"(word) : "memory");
}

// Warm squares up to this size are closed by closure_cluster_kernel (the
// square must fit one CTA's shared memory), larger ones by the persistent
// kernel.
template <typename E>
constexpr int32_t kClusterMaxWarm = sizeof(E) == 2 ? 256 : 192;

// CTAs per SM: five for int32 lanes (at most 96 registers a thread; the
// tile update needs 92), which measured fastest against four and six; seven
// for packed int16 lanes (72 registers, as the unbounded build took)
#define SCHULZE_PERSIST_BOUNDS __launch_bounds__(kThreads, sizeof(E) == 2 ? 7 : 5)
// The next work item of a persistent CTA, as thread 0 prepares it while the
// CTA computes the current one: the item, the progress words it waits for
// (own tile: `need` rounds applied; panel: the closed diagonal; tile: both
// panels) and their values as first loaded.
struct Pending {
  Item it;
  int32_t dep[3];
  uint32_t need[3];
  uint32_t val[3];
};

__device__ __forceinline__ uint32_t load_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <typename E, int kMix>
__global__ void SCHULZE_PERSIST_BOUNDS closure_persistent_kernel(E* __restrict__ W, int32_t ld, int32_t nb, Sync sy) {
  pdl_enter_early();
  __shared__ __align__(16) typename Ops<E, kMix>::Smem sm;
  __shared__ __align__(16) int32_t rowbuf[2][kB];
  __shared__ int32_t s_item[2][4];  // kind, round, tile row, tile column (double-buffered)
  __shared__ uint32_t s_flags[2];   // bit 0: skip the update; bit 1: tile already nonzero
  __shared__ int32_t s_slow[2];     // the next item still has to wait (double-buffered)
  constexpr uint32_t kFail = 0xFFFFFFFFu;
  const int32_t nbr = (*sy.warm + kB - 1) / kB;
  if (*sy.warm <= kClusterMaxWarm<E>) return;  // closure_cluster_kernel's case
  const Shape sh = make_shape(nbr, nbr);  // the warm square; nb is the progress-word row stride
  const int64_t total_items = int64_t(nbr) * nbr * nbr;
  // Thread 0 runs the schedule. While the CTA computes item i it claims the
  // next queue slot, decodes it and loads the progress words it depends on.
  // After its own part of item i it looks at them again without waiting:
  // when all are there, it writes the next item into the other half of the
  // double buffer, which the barrier ending item i makes visible, so one
  // barrier per item is left besides the operand barrier inside the update.
  // When one is not there yet, nothing waits before item i is published (the
  // missing tile may itself wait, through other CTAs, for item i): thread 0
  // publishes, then waits (bounded) and hands the item over behind one more
  // barrier. The schedule stays deadlock-free: a CTA holds at most one
  // claimed, unstarted item, later in the queue than its current one, and
  // only waits once its current item is published, so the earliest
  // unfinished item is always being computed (its dependencies are earlier,
  // hence finished) and completes.
  __shared__ Pending nx;  // thread 0's alone (kept out of every thread's registers)
  auto issue = [&](uint32_t t) {  // thread 0: claim decoded, dependencies' words loaded
    nx.it = Item{-1, 0, 0, 0};
    nx.dep[0] = nx.dep[1] = nx.dep[2] = -1;
    if (int64_t(t) >= total_items || *reinterpret_cast<volatile uint32_t*>(sy.abort_flag)) return;
    nx.it = decode_item(int64_t(t), sh);
    const Item& it = nx.it;
    const uint32_t r = uint32_t(it.r);
    nx.dep[0] = it.i * nb + it.j, nx.need[0] = r;  // rounds 0 .. r-1 applied
    if (it.kind == kPanel) {
      nx.dep[1] = it.r * nb + it.r, nx.need[1] = r + 1;
    } else if (it.kind == kTile) {
      nx.dep[1] = it.i * nb + it.r, nx.need[1] = r + 1;
      nx.dep[2] = it.r * nb + it.j, nx.need[2] = r + 1;
    }
#pragma unroll
    for (int q = 0; q < 3; ++q)
      if (nx.dep[q] >= 0) nx.val[q] = load_acquire(sy.prog + nx.dep[q]);
  };
  // thread 0, no waiting: every dependency of the next item there (those not
  // seen yet are loaded once more)
  auto ready = [&]() -> bool {
    if (nx.it.kind < 0) return true;
    bool all = true;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      if (nx.dep[q] < 0 || (nx.val[q] & kRoundMask) >= nx.need[q]) continue;
      nx.val[q] = load_acquire(sy.prog + nx.dep[q]);
      all = all && (nx.val[q] & kRoundMask) >= nx.need[q];
    }
    return all;
  };
  // thread 0: wait for what is still missing (bounded), decide the flags,
  // write the next item into s_item[buf]
  auto decide = [&](int buf) {
    if (nx.it.kind >= 0) {
      bool ok = true;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        if (nx.dep[q] < 0 || !ok || (nx.val[q] & kRoundMask) >= nx.need[q]) continue;
        nx.val[q] = wait_round(sy, nx.dep[q], nx.need[q]);
        ok = nx.val[q] != kFail;
      }
      if (!ok) nx.it.kind = -1;
    }
    uint32_t flags = 0;
    if (nx.it.kind >= 0) {
      __threadfence();
      const uint32_t own = nx.val[0];
      if (nx.it.kind == kDiag) {
        if (!(own & kNZ)) flags |= 1u;
      } else if (nx.it.kind == kPanel) {
        if (!(nx.val[1] & kNZ) || !(own & kNZ)) flags |= 1u;
      } else if (!(nx.val[1] & kNZ) || !(nx.val[2] & kNZ)) {
        flags |= 1u;
      }
      if (own & kNZ) flags |= 2u;
    }
    s_item[buf][0] = nx.it.kind, s_item[buf][1] = nx.it.r, s_item[buf][2] = nx.it.i, s_item[buf][3] = nx.it.j;
    s_flags[buf] = flags;
  };
  if (threadIdx.x == 0) {
    issue(atomicAdd(sy.head, 1u));
    decide(0);  // nothing computed yet: waiting here delays no one
  }
  __syncthreads();
  for (int buf = 0;; buf ^= 1) {
    const int32_t kind = s_item[buf][0], r = s_item[buf][1], i = s_item[buf][2], j = s_item[buf][3];
    const uint32_t flags = s_flags[buf];
    if (kind < 0) return;
    if (threadIdx.x == 0) issue(atomicAdd(sy.head, 1u));  // loads in flight during this item
    bool nz = (flags & 2u) != 0;
    if (!(flags & 1u)) {
      if (kind == kDiag)
        nz = diag_closure_local<E>(W, ld, r, rowbuf, threadIdx.x, BlockBarrier{});
      else
        nz = Ops<E, kMix>::update_local(W, ld, i, j, r, sm, threadIdx.x, BlockBarrier{});
    }
    if (threadIdx.x == 0) {
      const bool fast = ready();
      if (fast) decide(buf ^ 1);
      s_slow[buf] = fast ? 0 : 1;
    }
    nz = __syncthreads_or(nz) != 0;  // every store of the tile done; next item or s_slow[buf] visible
    if (threadIdx.x == 0) {
      publish(sy, i * nb + j, uint32_t(r + 1) | (nz ? kNZ : 0u));
      if (!(flags & 1u)) atomicAdd(&sy.counters[kind == kDiag ? 1 : 0], 1ull);
      atomicAdd(&sy.counters[2], 1ull);
    }
    if (s_slow[buf]) {  // the next item's tiles were not all there: wait now that this one is published
      if (threadIdx.x == 0) decide(buf ^ 1);
      __syncthreads();
    }
  }
}

// Warm squares of at most kClusterMaxWarm candidates: the closure by
// repeated (max, min) squaring, in place, on a cluster of kClusterCtas CTAs
// (one per SM). Every CTA holds a copy of the square S (n = nw rounded up to
// 64, row-major) in shared memory; CTA q owns the warm rows q, q + 8, ... A
// sweep sets, for every owned row i and column j,
//   S[i][j] = max(S[i][j], max_{k < nw} min(S[i][k], S[k][j])),
// reading whatever the copy holds: widths only grow and every value is the
// width of a real path, so a mix of older and newer entries is still a lower
// bound of the closure. Each changed 16-byte piece is copied into the other
// CTAs (distributed shared memory). Sweep t covers at least the paths of up
// to 2^t edges, so at most ceil(log2 nw) + 1 sweeps run: the cluster stops
// after the first sweep in which no CTA changed anything, when S (x) S <= S
// held for the whole square, i.e. S is closed. Rows of cold candidates are
// zero and stay zero; columns run over all of S. Each CTA then writes its
// rows back into W and sets the nonzero bits of the 64 x 64 tiles of W for
// cold_product_kernel.
constexpr int kClusterCtas = 8;
constexpr int kClusterThreads = 512;
constexpr int kMaxSweeps = 40;  // > ceil(log2 256) + 1: never reached

// acc (16 bytes of a row) = max(acc, min(a(k), b0), min(a(k + 1), b1)) with
// b0, b1 the same 16 bytes of rows k and k + 1 and a the row's entries k,
// k + 1 (one 32-bit word of 16-bit lanes, or an int2)
__device__ __forceinline__ void sweep_step(uint4& acc, uint32_t a, const uint4& b0, const uint4& b1) {
  const uint32_t l = __byte_perm(a, 0, 0x1010), h = __byte_perm(a, 0, 0x3232);
  acc.x = __vimax3_s16x2(acc.x, __vmins2(l, b0.x), __vmins2(h, b1.x));
  acc.y = __vimax3_s16x2(acc.y, __vmins2(l, b0.y), __vmins2(h, b1.y));
  acc.z = __vimax3_s16x2(acc.z, __vmins2(l, b0.z), __vmins2(h, b1.z));
  acc.w = __vimax3_s16x2(acc.w, __vmins2(l, b0.w), __vmins2(h, b1.w));
}
__device__ __forceinline__ void sweep_step(uint4& acc, int2 a, const uint4& b0, const uint4& b1) {
  auto f = [&](uint32_t x, uint32_t u, uint32_t v) {
    return uint32_t(__vimax3_s32(int32_t(x), min(a.x, int32_t(u)), min(a.y, int32_t(v))));
  };
  acc.x = f(acc.x, b0.x, b1.x);
  acc.y = f(acc.y, b0.y, b1.y);
  acc.z = f(acc.z, b0.z, b1.z);
  acc.w = f(acc.w, b0.w, b1.w);
}

__device__ __forceinline__ bool differs(const uint4& a, const uint4& b) {
  return ((a.x ^ b.x) | (a.y ^ b.y) | (a.z ^ b.z) | (a.w ^ b.w)) != 0u;
}

template <typename E>
__global__ void __cluster_dims__(kClusterCtas, 1, 1) __launch_bounds__(kClusterThreads, 1)
    closure_cluster_kernel(E* __restrict__ W, int32_t ld, int32_t nb, const int32_t* __restrict__ warm,
                           uint32_t* __restrict__ prog, unsigned long long* counters) {
  pdl_enter();
  using AW = typename std::conditional<sizeof(E) == 2, uint32_t, int2>::type;  // a row's entries k, k + 1
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int32_t nw = *warm;
  if (nw == 0 || nw > kClusterMaxWarm<E>) return;  // the same branch in every CTA
  extern __shared__ __align__(16) unsigned char cluster_smem[];
  uint4* S4 = reinterpret_cast<uint4*>(cluster_smem);
  const AW* A = reinterpret_cast<const AW*>(cluster_smem);  // row i, entries k, k + 1: A[i * n / 2 + k / 2]
  __shared__ uint32_t tnz[4][4];                  // 64 x 64 tiles of W holding a nonzero
  __shared__ uint32_t flags[2][kClusterCtas];     // CTA o changed something in the sweep (two buffers)
  const int32_t n = (nw + kB - 1) / kB * kB;      // square side: whole 64-wide tiles
  constexpr int kPer16 = 16 / sizeof(E);          // entries per 16-byte piece
  const int32_t Q = n / kPer16;                   // pieces per row
  const int32_t nwe = (nw + 1) & ~1;              // pivots, in pairs (row nw, if read, is zero)
  const int t = threadIdx.x;
  const unsigned q = cl.block_rank();
  {
    // rows 0 .. nwe - 1 of W, eight 16-byte loads in flight per thread
    const int32_t total = nwe * Q;
    constexpr int kU = 8;
    for (int32_t e0 = t; e0 < total; e0 += kU * kClusterThreads) {
      uint4 v[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int32_t e = e0 + u * kClusterThreads;
        if (e < total) v[u] = __ldcg(reinterpret_cast<const uint4*>(W + int64_t(e / Q) * ld) + e % Q);
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int32_t e = e0 + u * kClusterThreads;
        if (e < total) S4[e] = v[u];
      }
    }
  }
  if (t < 16) tnz[t >> 2][t & 3] = 0u;
  if (t < 2 * kClusterCtas) flags[t / kClusterCtas][t % kClusterCtas] = 0u;
  cl.sync();  // every copy loaded, every flag clear, before any remote write
  const int32_t own = int32_t(q) < nw ? (nw - int32_t(q) + kClusterCtas - 1) / kClusterCtas : 0;
  const int32_t items = (own + 1) / 2 * Q;  // (pair of owned rows, piece)
  int sweeps = 0;
  while (sweeps < kMaxSweeps) {
    bool changed = false;
    for (int32_t it = t; it < items; it += kClusterThreads) {
      const int32_t rp = it / Q, c = it % Q;
      const int32_t i0 = int32_t(q) + kClusterCtas * (2 * rp), i1 = i0 + kClusterCtas;
      const bool has1 = i1 < nw;
      const uint4 x0 = S4[i0 * Q + c], x1 = has1 ? S4[i1 * Q + c] : x0;
      uint4 acc0 = x0, acc1 = x1;
      const AW* a0p = A + i0 * (n / 2);
      const AW* a1p = A + (has1 ? i1 : i0) * (n / 2);
#pragma unroll 4
      for (int32_t k = 0; k < nwe; k += 2) {
        const uint4 b0 = S4[k * Q + c], b1 = S4[(k + 1) * Q + c];
        sweep_step(acc0, a0p[k >> 1], b0, b1);
        sweep_step(acc1, a1p[k >> 1], b0, b1);
      }
      if (differs(acc0, x0)) {
        changed = true;
        S4[i0 * Q + c] = acc0;
#pragma unroll
        for (int o = 1; o < kClusterCtas; ++o)
          *cl.map_shared_rank(S4 + i0 * Q + c, (q + o) % kClusterCtas) = acc0;
      }
      if (has1 && differs(acc1, x1)) {
        changed = true;
        S4[i1 * Q + c] = acc1;
#pragma unroll
        for (int o = 1; o < kClusterCtas; ++o)
          *cl.map_shared_rank(S4 + i1 * Q + c, (q + o) % kClusterCtas) = acc1;
      }
    }
    ++sweeps;
    const int any = __syncthreads_or(changed);
    if (any && t < kClusterCtas) *cl.map_shared_rank(&flags[sweeps & 1][q], unsigned(t)) = 1u;
    cl.sync();  // this sweep's copies and flags visible everywhere
    const int more = __syncthreads_or(t < kClusterCtas && flags[sweeps & 1][t] != 0u);
    if (t < kClusterCtas) flags[sweeps & 1][t] = 0u;  // rewritten two sweeps on, after the next barrier
    if (!more) break;  // the same decision in every CTA
  }
  // each CTA writes its rows back with a zero diagonal; nonzero bits per
  // 64 x 64 tile of W. No CTA writes into another any more.
  for (int32_t it = t; it < own * Q; it += kClusterThreads) {
    const int32_t r = it / Q, c = it % Q;
    const int32_t i = int32_t(q) + kClusterCtas * r, j0 = c * kPer16;
    uint4 v = S4[i * Q + c];
    if (i >= j0 && i < j0 + kPer16) {
      const int e = i - j0;
      const int w = sizeof(E) == 2 ? e >> 1 : e;
      const uint32_t keep = sizeof(E) == 2 ? ((e & 1) ? 0x0000FFFFu : 0xFFFF0000u) : 0u;
      v.x = w == 0 ? v.x & keep : v.x;
      v.y = w == 1 ? v.y & keep : v.y;
      v.z = w == 2 ? v.z & keep : v.z;
      v.w = w == 3 ? v.w & keep : v.w;
    }
    *reinterpret_cast<uint4*>(W + int64_t(i) * ld + j0) = v;
    if (v.x | v.y | v.z | v.w) tnz[i / kB][j0 / kB] = 1u;
  }
  __syncthreads();
  if (t < 16 && tnz[t >> 2][t & 3]) atomicOr(&prog[(t >> 2) * nb + (t & 3)], kNZ);
  if (t == 0 && q == 0)  // entry updates, in 64 x 64 x 64 tile units
    atomicAdd(&counters[0], (unsigned long long)sweeps * uint64_t(nw) * uint64_t(nw) * uint64_t(n) / 262144ull);
}

// Uniform cold columns: u[i] = max(ucol[i], max_x min(W[i][x], ucol[x]))
// over the warm x (a warp per warm row i, lanes over x), and ucount = the
// number of warm rows with u > 0.
template <typename E>
__global__ void __launch_bounds__(256) uniform_cold_kernel(const E* __restrict__ W, int32_t mp, int32_t m,
                                                           const int32_t* __restrict__ warm,
                                                           const int32_t* __restrict__ hint_valid,
                                                           const int32_t* __restrict__ ucol, int32_t* __restrict__ u,
                                                           int32_t* __restrict__ ucount) {
  pdl_enter();
  const int32_t nw = *warm;
  const int32_t rows = (nw + kB - 1) / kB * kB;
  if (!(hint_valid && *hint_valid && rows < m)) return;
  const int lane = threadIdx.x & 31;
  const int64_t wid = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t i = wid; i < nw; i += nwarps) {
    const E* wrow = W + i * mp;
    int32_t best = 0;
    for (int32_t x = lane; x < nw; x += 32) best = max(best, min(int32_t(wrow[x]), ucol[x]));
#pragma unroll
    for (int o = 16; o; o >>= 1) best = max(best, __shfl_xor_sync(0xFFFFFFFFu, best, o));
    if (lane == 0) {
      const int32_t ui = max(best, ucol[i]);
      u[i] = ui;
      if (ui > 0) atomicAdd(ucount, 1);
    }
  }
}

// Cold columns for warm squares that fit shared memory (the cluster
// closure's sizes): every CTA keeps the closed square P (nwp x nwp, rows
// padded by one word against bank conflicts) and walks strips of
// kStripWords words (16-bit pairs, or int32 entries) of cold columns:
// X[i][j] = max(X[i][j], max_k min(P[i][k], X[k][j])) for the warm rows i,
// with X[k][j] staged before any row of the strip is written. Thread t keeps
// words w and w + 8 (w = t % 8) of rows t / 8 + 64 r, r < 4, so that each
// load of P or of the strip feeds several updates.
constexpr int kStripWords = 16;

template <typename E>
__global__ void __launch_bounds__(512, 1) cold_strip_kernel(E* __restrict__ W, int32_t ld, int32_t m,
                                                            const int32_t* __restrict__ warm,
                                                            unsigned long long* counters,
                                                            const int32_t* __restrict__ hint_valid) {
  pdl_enter_early();
  using Wd = typename std::conditional<sizeof(E) == 2, uint32_t, int32_t>::type;  // one word
  constexpr int kPer = sizeof(Wd) / sizeof(E);                                  // entries per word
  const int32_t nw = *warm;
  if (nw == 0 || nw > kClusterMaxWarm<E>) return;  // the tile kernel's case
  const int32_t nwp = (nw + kB - 1) / kB * kB;
  if (hint_valid && *hint_valid && nwp < m) return;  // uniform cold columns
  const int32_t rowwords = ld / kPer;
  const int32_t nstrips = (rowwords - nwp / kPer + kStripWords - 1) / kStripWords;
  if (int32_t(blockIdx.x) >= nstrips) return;
  extern __shared__ __align__(16) unsigned char strip_smem[];
  const int32_t pw = nwp / kPer, pst = pw + 1;  // words per row of P, padded (odd)
  Wd* P = reinterpret_cast<Wd*>(strip_smem);
  Wd* B = P + nwp * pst;  // [nwp][kStripWords]
  const int t = threadIdx.x;
  for (int32_t e = t; e < nwp * (pw / 4); e += blockDim.x) {  // 16-byte reads of W
    const int32_t i = e / (pw / 4), c4 = e % (pw / 4);
    const uint4 v = __ldcg(reinterpret_cast<const uint4*>(W + int64_t(i) * ld) + c4);
    Wd* dst = P + i * pst + 4 * c4;
    dst[0] = Wd(v.x), dst[1] = Wd(v.y), dst[2] = Wd(v.z), dst[3] = Wd(v.w);
  }
  const int w = t & 7, rg = t >> 3;  // words w, w + 8; rows rg + 64 r
  const int32_t K = (nw + 1) & ~1;   // rows >= nw are zero
  unsigned long long done = 0;
  for (int32_t s = blockIdx.x; s < nstrips; s += gridDim.x) {
    const int32_t c0 = pw + s * kStripWords;  // first word of the strip
    __syncthreads();  // P loaded / the previous strip's B consumed
    for (int32_t e = t; e < nwp * kStripWords; e += blockDim.x) {
      const int32_t k = e / kStripWords, c = c0 + e % kStripWords;
      B[e] = c < rowwords ? reinterpret_cast<const Wd*>(W + int64_t(k) * ld)[c] : Wd(0);
    }
    __syncthreads();
    Wd acc[4][2];
    bool row_ok[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int32_t i = rg + 64 * r;
      row_ok[r] = i < nw;
      acc[r][0] = row_ok[r] ? B[i * kStripWords + w] : Wd(0);
      acc[r][1] = row_ok[r] ? B[i * kStripWords + w + 8] : Wd(0);
    }
#pragma unroll 2
    for (int32_t k = 0; k < K; k += 2) {
      const Wd b00 = B[k * kStripWords + w], b01 = B[k * kStripWords + w + 8];
      const Wd b10 = B[(k + 1) * kStripWords + w], b11 = B[(k + 1) * kStripWords + w + 8];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        if (!row_ok[r]) continue;
        const Wd* prow = P + (rg + 64 * r) * pst;
        if constexpr (sizeof(E) == 2) {
          const uint32_t a = prow[k >> 1];
          const uint32_t alo = (a & 0xFFFFu) | (a << 16), ahi = (a >> 16) | (a & 0xFFFF0000u);
          acc[r][0] = __vimax3_s16x2(acc[r][0], __vmins2(alo, b00), __vmins2(ahi, b10));
          acc[r][1] = __vimax3_s16x2(acc[r][1], __vmins2(alo, b01), __vmins2(ahi, b11));
        } else {
          const int32_t a0 = prow[k], a1 = prow[k + 1];
          acc[r][0] = __vimax3_s32(acc[r][0], min(a0, b00), min(a1, b10));
          acc[r][1] = __vimax3_s32(acc[r][1], min(a0, b01), min(a1, b11));
        }
      }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      if (!row_ok[r]) continue;
      Wd* dst = reinterpret_cast<Wd*>(W + int64_t(rg + 64 * r) * ld) + c0;
      if (c0 + w < rowwords) dst[w] = acc[r][0];
      if (c0 + w + 8 < rowwords) dst[w + 8] = acc[r][1];
    }
    ++done;
  }
  if (t == 0 && done) atomicAdd(&counters[0], done);
}

// Cold columns: X(i, j) = max(X, W(i, k) (x) W(k, j)) for every warm tile row
// i, cold tile column j and warm k, with the warm square already closed. Each
// (i, j) is one work item (a 128-thread CTA applies its k in order). An item
// may read a W(k, j) that another item is raising at the same time; every
// value either one sees is the width of a real path and the closed square
// composes with itself without growing (p(i,x) and p(x,y) give a walk no
// wider than p(i,y)), so the result is the exact closure either way.
template <typename E, int kMix>
__global__ void __launch_bounds__(kThreads) cold_product_kernel(E* __restrict__ W, int32_t ld, int32_t nb,
                                                                 int32_t m, const int32_t* __restrict__ warm,
                                                                 const uint32_t* __restrict__ prog,
                                                                 unsigned long long* counters,
                                                                 const int32_t* __restrict__ hint_valid) {
  pdl_enter_early();
  __shared__ __align__(16) typename Ops<E, kMix>::Smem sm;
  if (*warm <= kClusterMaxWarm<E>) return;  // cold_strip_kernel's case
  if (hint_valid && *hint_valid && (*warm + kB - 1) / kB * kB < m) return;  // uniform cold columns
  const int32_t nbr = (*warm + kB - 1) / kB;
  const int32_t nc = nb - nbr;
  const int64_t items = int64_t(nbr) * nc;
  unsigned long long done = 0;
  for (int64_t t = blockIdx.x; t < items; t += gridDim.x) {
    const int32_t i = int32_t(t / nc), j = nbr + int32_t(t % nc);
    for (int32_t k = 0; k < nbr; ++k) {
      const uint32_t a = prog[i * nb + k], b = prog[k * nb + j];
      if ((a & kNZ) && (b & kNZ)) {
        Ops<E, kMix>::update(W, ld, i, j, k, sm, threadIdx.x, BlockBarrier{});
        ++done;
      }
    }
  }
  if (threadIdx.x == 0 && done) atomicAdd(&counters[0], done);
}

// beaten_by straight from the closed warm rows of W, for callers that need
// the ranking but not a second pass over p: a cold candidate x (no outgoing
// edge, p[x][*] = 0) is beaten by every warm j with p[j][x] > 0; a warm x by
// every warm j with p[j][x] > p[x][j]; cold candidates beat nobody. CTA =
// 32 relabeled columns x 8 row groups.
template <typename E>
__global__ void __launch_bounds__(512) wextract_kernel(const E* __restrict__ W, int32_t mp, int32_t m,
                                                       const int32_t* __restrict__ perm,
                                                       const int32_t* __restrict__ warm, int32_t* __restrict__ bb,
                                                       const int32_t* __restrict__ hint_valid,
                                                       const int32_t* __restrict__ ucount) {
  pdl_enter();
  constexpr int kG = 16;  // row groups
  __shared__ int32_t part[kG][33];
  const int32_t nw = *warm;
  const int32_t rows = (nw + kB - 1) / kB * kB;
  const bool uc = hint_valid && *hint_valid && rows < m;
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  for (int32_t b0 = blockIdx.x * 32; b0 < m; b0 += gridDim.x * 32) {
    if (uc && b0 >= rows) {  // uniform cold columns: beaten by the warm rows with u > 0
      if (g == 0 && b0 + lane < m) bb[perm[b0 + lane]] = *ucount;
      continue;
    }
    const int32_t b = b0 + lane;
    int32_t c = 0;
    if (b < m) {
      if (b < nw) {
#pragma unroll 4
        for (int32_t j = g; j < nw; j += kG)
          c += (j != b && int32_t(W[int64_t(j) * mp + b]) > int32_t(W[int64_t(b) * mp + j]));
      } else {
#pragma unroll 8
        for (int32_t j = g; j < nw; j += kG) c += W[int64_t(j) * mp + b] != E(0);
      }
    }
    part[g][lane] = c;
    __syncthreads();
    if (g == 0 && b < m) {
      int32_t tot = 0;
#pragma unroll
      for (int h = 0; h < kG; ++h) tot += part[h][lane];
      bb[perm[b]] = tot;
    }
    __syncthreads();
  }
}

// Scratch of one closure: W (warm rows x all columns, padded square), the
// progress words, queue head, abort flag, and the relabeling.
struct ClosureBufs {
  void* W;
  uint32_t* prog;
  int32_t *rowflag, *perm, *inv, *warm;
  unsigned long long* counters;
  // optional: warm flags known from the tally, used when *hint_valid != 0
  const int32_t* hint = nullptr;
  const int32_t* hint_valid = nullptr;
  // uniform cold columns (used only with a valid hint): ucol, u [m], ucount
  int32_t *ucol = nullptr, *ucold = nullptr, *ucount = nullptr;
  bool margin = false;  // margin weights instead of winning votes
};

// Rowflags, relabel, pack, closure of the warm square, cold product, widen.
// ctx may be null (no counting, no profiling). kMix: the min/max units of
// the int32 tile updates (tiles::update2_s32).
template <typename E, int kMix>
int closure_pipeline_mix(schulze_ctx* ctx, int sms, const int32_t* d, int32_t m, int64_t bound, int32_t* p,
                         const ClosureBufs& bf, int32_t* status, cudaStream_t stream, int32_t* bb_out, bool side) {
  const int32_t mp = int32_t(align_up(size_t(m), kB));
  const int32_t nb = mp / kB;
  E* W = static_cast<E*>(bf.W);
  uint32_t* head = bf.prog + size_t(nb) * size_t(nb);
  uint32_t* abort_flag = head + 1;
  {
    // progress words, queue head and abort flag; row flags; the uniform count
    ZeroSpans z;
    z.p[0] = bf.prog, z.words[0] = int64_t(nb) * nb + 2;
    z.p[1] = reinterpret_cast<uint32_t*>(bf.rowflag), z.words[1] = m;
    z.p[2] = reinterpret_cast<uint32_t*>(bf.ucount), z.words[2] = 1;
    if (int rc = zero_async(ctx, z, stream)) return rc;
  }
  const double mm = double(m) * double(m);
  auto grid_for = [&](const void* fn, int threads, size_t smem, int64_t cap) {
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess || per_sm < 1) {
      cudaGetLastError();
      per_sm = 1;
    }
    return int(std::max<int64_t>(1, std::min<int64_t>(int64_t(per_sm) * sms, cap)));
  };
  {
    const int64_t nbt = (m + kFlagT - 1) / kFlagT;
    const int g = grid_for(reinterpret_cast<const void*>(rowflag_kernel), 256, 0, nbt * (nbt + 1) / 2);
    Launch L(ctx, stream, "closure_rowflags", mm * 4.0);
    launch_pdl(rowflag_kernel, dim3(g), dim3(256), 0, stream, false, d, m, bound, bf.rowflag, status, bf.hint_valid,
               rows_vec16(d, m));
  }
  {
    Launch L(ctx, stream, "closure_relabel", double(m) * 12.0);
    const size_t smem = m <= kScanSmem ? size_t(m) * 4 : 0;
    cudaFuncSetAttribute(relabel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    launch_pdl(relabel_kernel, dim3(1), dim3(1024), smem, stream, false,
               static_cast<const int32_t*>(bf.rowflag), m, bf.perm, bf.inv, bf.warm, bf.hint_valid);
  }
  {
    const int g = grid_for(reinterpret_cast<const void*>(pack_kernel<E>), 512, 0, mp);
    Launch L(ctx, stream, "closure_pack", 0.0);
    launch_pdl(pack_kernel<E>, dim3(g), dim3(512), 0, stream, false, d, m, mp,
               static_cast<const int32_t*>(bf.perm), static_cast<const int32_t*>(bf.warm), W, bf.prog, nb, bf.hint,
               bf.hint_valid, bf.ucol, bf.margin ? 1 : 0);
  }
  if (int rc = check_launch()) return rc;
  {
    const size_t smem = size_t(kClusterMaxWarm<E>) * kClusterMaxWarm<E> * sizeof(E);
    cudaFuncSetAttribute(closure_cluster_kernel<E>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    Launch L(ctx, stream, "closure_cluster", 0.0);
    launch_pdl(closure_cluster_kernel<E>, dim3(kClusterCtas), dim3(kClusterThreads), smem, stream, false, W, mp, nb,
               static_cast<const int32_t*>(bf.warm), bf.prog, bf.counters);
  }
  if (int rc = check_launch()) return rc;
  {
    // persistent grid: every CTA resident (cooperative launch)
    const int grid = grid_for(reinterpret_cast<const void*>(closure_persistent_kernel<E, kMix>), kThreads, 0,
                              int64_t(nb) * nb * nb);
    Sync sy{bf.prog, head, abort_flag, status, bf.warm, bf.counters,
            ctx ? ctx->wait_limit_cycles : kSpinLimitCycles};
    E* Wp = W;
    int32_t ldp = mp, nbp = nb;
    Launch L(ctx, stream, "closure_persistent", double(m) * mm);
    if (launch_pdl(closure_persistent_kernel<E, kMix>, dim3(grid), dim3(kThreads), 0, stream, true, Wp, ldp, nbp, sy) !=
        cudaSuccess) {
      cudaGetLastError();
      return SCHULZE_ECUDA;
    }
  }
  {
    const size_t cw = size_t(kClusterMaxWarm<E>);
    const size_t smem = (cw * (cw * sizeof(E) / 4 + 1) + cw * kStripWords) * 4;
    cudaFuncSetAttribute(cold_strip_kernel<E>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    Launch L(ctx, stream, "closure_cold_strips", 0.0);
    launch_pdl(cold_strip_kernel<E>, dim3(sms), dim3(512), smem, stream, false, W, mp, m,
               static_cast<const int32_t*>(bf.warm), bf.counters, bf.hint_valid);
  }
  {
    const int g = grid_for(reinterpret_cast<const void*>(cold_product_kernel<E, kMix>), kThreads, 0, int64_t(nb) * nb);
    Launch L(ctx, stream, "closure_cold", 0.0);
    launch_pdl(cold_product_kernel<E, kMix>, dim3(g), dim3(kThreads), 0, stream, false, W, mp, nb, m,
               static_cast<const int32_t*>(bf.warm), static_cast<const uint32_t*>(bf.prog), bf.counters,
               bf.hint_valid);
  }
  if (bf.hint_valid) {
    Launch L(ctx, stream, "closure_cold_uniform", 0.0);
    launch_pdl(uniform_cold_kernel<E>, dim3(std::max(1, std::min(sms, (m + 7) / 8))), dim3(256), 0, stream, false,
               static_cast<const E*>(W), mp, m, static_cast<const int32_t*>(bf.warm), bf.hint_valid,
               static_cast<const int32_t*>(bf.ucol), bf.ucold, bf.ucount);
  }
  {
    // p is written from W (and the uniform cold values); with a side stream
    // it is written there while beaten_by and the ranking come out of W on
    // stream, with at most four CTAs per SM so that those kernels find room
    const bool fork = side && bb_out && ctx && ctx->side_stream;
    cudaStream_t wst = stream;
    int g = grid_for(reinterpret_cast<const void*>(widen_kernel<E>), 256, 0, m);
    if (fork) {
      if (cudaEventRecord(ctx->side_fork, stream) != cudaSuccess ||
          cudaStreamWaitEvent(ctx->side_stream, ctx->side_fork, 0) != cudaSuccess)
        return SCHULZE_ECUDA;
      ctx->side_pending = true;  // joined by the caller, whatever happens next
      wst = ctx->side_stream;
      g = std::min(g, 4 * sms);
    }
    Launch L(ctx, wst, "closure_widen", mm * 4.0);
    launch_pdl(widen_kernel<E>, dim3(g), dim3(256), 0, wst, false, static_cast<const E*>(W), mp, m,
               static_cast<const int32_t*>(bf.inv), static_cast<const int32_t*>(bf.perm),
               static_cast<const int32_t*>(bf.warm), p, bf.hint_valid, static_cast<const int32_t*>(bf.ucold),
               rows_vec16(p, m));
    if (fork && cudaEventRecord(ctx->side_join, wst) != cudaSuccess) return SCHULZE_ECUDA;
  }
  if (bb_out) {
    Launch L(ctx, stream, "closure_beaten_by", 0.0);
    launch_pdl(wextract_kernel<E>, dim3((m + 31) / 32), dim3(512), 0, stream, false, static_cast<const E*>(W), mp, m,
               static_cast<const int32_t*>(bf.perm), static_cast<const int32_t*>(bf.warm), bb_out, bf.hint_valid,
               static_cast<const int32_t*>(bf.ucount));
  }
  return check_launch();
}

// The int32 tile updates share their work between the integer and the fp32
// min/max units (the counts' bit patterns order alike on both) unless a
// count could reach the fp32 infinity pattern 0x7F800000.
template <typename E>
int closure_pipeline(schulze_ctx* ctx, int sms, const int32_t* d, int32_t m, int64_t bound, int32_t* p,
                     const ClosureBufs& bf, int32_t* status, cudaStream_t stream, int32_t* bb_out = nullptr,
                     bool side = false) {
  if constexpr (sizeof(E) == 4 && tiles::kS32Mix != 0) {
    if (bound < 0x7F800000LL)
      return closure_pipeline_mix<E, tiles::kS32Mix>(ctx, sms, d, m, bound, p, bf, status, stream, bb_out, side);
  }
  return closure_pipeline_mix<E, 0>(ctx, sms, d, m, bound, p, bf, status, stream, bb_out, side);
}

template <typename E>
int run_closure(schulze_ctx* ctx, const int32_t* d, int32_t m, int64_t bound, int32_t* p, void* ws,
                cudaStream_t stream, int32_t* bb_out, int32_t* hint, const int32_t* hint_valid,
                bool margin, bool side) {
  const int32_t mp = int32_t(align_up(size_t(m), kB));
  const int32_t nb = mp / kB;
  Carver cv(ws);
  ClosureBufs bf;
  bf.W = cv.take<E>(size_t(mp) * size_t(mp));
  bf.prog = cv.take<uint32_t>(size_t(nb) * size_t(nb) + 2);
  bf.rowflag = cv.take<int32_t>(size_t(m));
  bf.perm = cv.take<int32_t>(size_t(m));
  bf.inv = cv.take<int32_t>(size_t(m));
  bf.warm = cv.take<int32_t>(1);
  if (hint) {  // the relabeling lives with the tally's flags (written there when they are valid)
    bf.perm = hint + m;
    bf.inv = hint + 2 * size_t(m);
    bf.warm = hint + 3 * size_t(m);
  }
  bf.ucol = cv.take<int32_t>(size_t(m));
  bf.ucold = cv.take<int32_t>(size_t(m));
  bf.ucount = cv.take<int32_t>(1);
  bf.counters = ctx->counters;
  bf.hint = hint;
  bf.hint_valid = hint_valid;
  bf.margin = margin;
  const int sms = ctx->sm_count > 0 ? ctx->sm_count : 1;
  return closure_pipeline<E>(ctx, sms, d, m, bound, p, bf, ctx->status, stream, bb_out, side);
}

}  // namespace

size_t closure_workspace_bytes(int32_t m, int64_t bound, uint32_t flags) {
  size_t mp = align_up(size_t(m), kB);
  size_t nb = mp / kB;
  return align_up(mp * mp * (use_s16(bound, flags) ? 2 : 4), 256) + align_up((nb * nb + 2) * 4, 256) +
         6 * align_up(size_t(m) * 4, 256) + 4096;
}

int closure_launch(schulze_ctx* ctx, const int32_t* d, int32_t m, int64_t bound, int32_t* p, uint32_t flags,
                   void* ws, cudaStream_t stream, int32_t* beaten_by, int32_t* hint,
                   const int32_t* hint_valid, bool side) {
  const bool margin = (flags & SCHULZE_F_MARGIN) != 0;
  if (use_s16(bound, flags))
    return run_closure<int16_t>(ctx, d, m, bound, p, ws, stream, beaten_by, hint, hint_valid, margin, side);
  return run_closure<int32_t>(ctx, d, m, bound, p, ws, stream, beaten_by, hint, hint_valid, margin, side);
}

// ------------------------------------------------- allocation-free variant
//
// schulze_strongest_paths_static runs the same kernels as closure_launch on
// scratch that lives in a file-scope device array instead of a context's
// cudaMalloc'ed workspace, for callers that cannot allocate device memory.
// The array is sized for m <= kStaticMaxM; every GPU that loads the library
// holds it until the process exits.

namespace {

constexpr int32_t kStaticMaxM = 1024;
constexpr size_t kStaticMp = 1024;  // kStaticMaxM rounded up to the tile size
constexpr size_t kStaticNb = kStaticMp / kB;
// byte offsets inside the array (each 256-aligned)
constexpr size_t kStW = 0;                                            // W: up to kStaticMp^2 int32
constexpr size_t kStProg = kStW + kStaticMp * kStaticMp * 4;          // progress words + head + abort
constexpr size_t kStRowflag = kStProg + align_up((kStaticNb * kStaticNb + 2) * 4, 256);
constexpr size_t kStPerm = kStRowflag + kStaticMaxM * 4;
constexpr size_t kStInv = kStPerm + kStaticMaxM * 4;
constexpr size_t kStWarm = kStInv + kStaticMaxM * 4;
constexpr size_t kStCounters = kStWarm + 256;                         // 3 x u64, never read back
constexpr size_t kStaticBytes = kStCounters + 256;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_static_mutex;
unsigned char* g_static_ptr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device. In host code the
// symbol's name is only a host-side stand-in, so the address is looked up
// once per device, with that device current, and cached.
int static_scratch(int device, unsigned char** out) {
  if (device < 0 || device >= kMaxDevices) return SCHULZE_EINVAL;
  std::lock_guard<std::mutex> lock(g_static_mutex);
  if (!g_static_ptr[device]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_static_scratch) != cudaSuccess || !ptr) {
      cudaGetLastError();
      return SCHULZE_ECUDA;
    }
    g_static_ptr[device] = static_cast<unsigned char*>(ptr);
  }
  *out = g_static_ptr[device];
  return SCHULZE_OK;
}

template <typename E>
int run_closure_static(unsigned char* base, int device, const int32_t* d, int32_t m, int64_t bound, int32_t* p,
                       int32_t* status, cudaStream_t stream, bool margin) {
  ClosureBufs bf;
  bf.margin = margin;
  bf.W = base + kStW;
  bf.prog = reinterpret_cast<uint32_t*>(base + kStProg);
  bf.rowflag = reinterpret_cast<int32_t*>(base + kStRowflag);
  bf.perm = reinterpret_cast<int32_t*>(base + kStPerm);
  bf.inv = reinterpret_cast<int32_t*>(base + kStInv);
  bf.warm = reinterpret_cast<int32_t*>(base + kStWarm);
  bf.counters = reinterpret_cast<unsigned long long*>(base + kStCounters);
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms < 1)
    return SCHULZE_ECUDA;
  // the array keeps the previous call's contents: the pipeline resets what
  // must start at zero (progress words, queue head, abort flag, row flags)
  return closure_pipeline<E>(nullptr, sms, d, m, bound, p, bf, status, stream);
}

}  // namespace

}  // namespace schulze

extern "C" int schulze_strongest_paths_static(const int32_t* d, int32_t m, int64_t bound, int32_t* p,
                                              uint32_t flags, int32_t* status, schulze_stream_t stream) {
  using namespace schulze;
  if (!d || !p || d == p || m < 1 || bound < 0) return SCHULZE_EINVAL;
  if ((flags & SCHULZE_F_FORCE_S16) && ((flags & SCHULZE_F_FORCE_S32) || bound > 32767)) return SCHULZE_EINVAL;
  if (m > kStaticMaxM) return SCHULZE_ETOOBIG;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return SCHULZE_ECUDA;
  unsigned char* base = nullptr;
  if (int rc = static_scratch(device, &base)) return rc;
  const bool margin = (flags & SCHULZE_F_MARGIN) != 0;
  if (use_s16(bound, flags))
    return run_closure_static<int16_t>(base, device, d, m, bound, p, status, stream, margin);
  return run_closure_static<int32_t>(base, device, d, m, bound, p, status, stream, margin);
}
