// Batched elections: thousands of independent elections of uneven size
// (m <= 1024) run in ONE persistent launch. Each CTA takes whole elections
// from a queue ordered by decreasing cost (longest first), and runs the path
// of Sect. 2.1 for each: ballot checks, pairwise tally, winning-votes
// weights, widest-path closure (blocked Floyd-Warshall in the (max, min)
// semiring with four 128-thread tile groups), winners and ranking.
//
// The plan (schulze_batch_create) computes the layout and the job order on
// the host, uploads the job table and reserves per-CTA scratch, so a run
// allocates nothing and can be captured in a CUDA graph.
#include <string.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <numeric>
#include <string>
#include <vector>

#include "count.cuh"
#include "internal.cuh"
#include "tiles.cuh"

namespace schulze {
namespace {

constexpr int kBT = 512;                        // threads per batch CTA
constexpr int kGroups = kBT / tiles::kThreads;  // tile groups of 128 threads
constexpr int32_t kBatchMaxM = 1024;
constexpr int64_t kFlushVoters = 32768;  // 16-bit lane counters are flushed before they can overflow

struct Job {
  int32_t n, m, k, e;
  int64_t ranks_off, mat_off, vec_off;
  int32_t chunk;  // ballots staged per tally step (the schedule of the election's m-bucket)
  int32_t gpt;    // tile groups that share one tally tile, splitting its ballots (1, 2 or 4)
  int32_t seg;    // schulze_batch_run_host: the segment whose arrival mark the job waits for
  int32_t pad;
};

// Elections are grouped by m into buckets, each with its own tally schedule
// (ballots staged per step, tile groups per tally tile), which
// schulze_batch_autotune times and caches.
constexpr int kBuckets = 5;
constexpr int32_t kBucketMax[kBuckets] = {64, 128, 256, 512, 1024};
inline int bucket_of(int32_t m) {
  int b = 0;
  while (b + 1 < kBuckets && m > kBucketMax[b]) ++b;
  return b;
}
constexpr int kChunkChoices[4] = {8, 16, 32, 64};
constexpr int kGptChoices[3] = {1, 2, 4};
// ballot ids a thread holds for the next step (16: the kernel then fits 128
// registers without spilling, which outweighs the longer steps that 32 allows)
constexpr int kPrefetch = 16;

struct BatchArgs {
  const Job* jobs;
  int32_t njobs;
  uint32_t* head;
  const int32_t* ranks;
  int32_t* d;
  int32_t* p;
  int32_t* winners;
  int32_t* order;
  int32_t* beaten_by;
  unsigned char* scratch;
  size_t slot_bytes;  // per CTA: W slot, then a d slot when the caller passes no d
  size_t w_bytes;
  int32_t* status;
  // schulze_batch_run_host: arrival marks of the ballot segments (set by the
  // copy stream after each segment's copy; null otherwise) and the bound on
  // a wait for one, in SM clock cycles
  const int32_t* seg_flag;
  long long wait_limit;
};

// Dynamic shared memory of one batch CTA, reused stage by stage. The tally
// stages `chunk` ballots as position rows of mpad (m rounded up to 64)
// entries: dup[chunk][mpad] (position in both 16-bit halves, guard bits set)
// then pos[chunk][mpad] (16-bit), carved from `raw`.
constexpr size_t kStageBytes = sizeof(tiles::SmemS32) * kGroups + 2 * tiles::kB * 4;
union BatchSmem {
  unsigned char raw[kStageBytes];
  struct {
    tiles::SmemS32 t[kGroups];
    int32_t rowbuf[2][tiles::kB];
  } c32;
  struct {
    tiles::SmemS16 t[kGroups];
    int32_t rowbuf[2][tiles::kB];
  } c16;
  int32_t bb[kBatchMaxM];
};

// ------------------------------------------------------------- tally

constexpr int kTT = 64;  // tally tile: 64 x 64 counters per group, 8 x 4 per thread
constexpr int kDiagBlocks = 72;  // 8 x 4 blocks of a diagonal tile on or above the diagonal

// The election's d, tile by tile: the four 128-thread groups take tiles of
// 64 x 64 entries, jb.gpt groups per tile (4 / gpt tiles per round), and
// count them in 16-bit lanes (two columns per word, the row operand
// duplicated into both halves); the groups of one tile take alternate
// staged ballots and add their counts into d (zeroed first) with atomics,
// so an election of one or two tiles still keeps every group busy (and so
// does a last round with one or two tiles left, whatever jb.gpt is).
// Ballots are staged `chunk` at a time as full position rows (unlisted
// candidates at position k), so one staging serves the four tiles of a
// round. Counters are added into d every kFlushVoters ballots. Full
// rankings count only the tiles above the diagonal and the thread blocks of
// the diagonal tiles on or above it (whole diagonal tiles when groups share
// tiles), and mirror the rest: d[j][i] = n - d[i][j]. The first round also checks the ballots: an
// id out of range, or one whose position slot is already taken within the
// same ballot, is reported as SCHULZE_EDATA.
__device__ void tally(const Job& jb, const int32_t* __restrict__ ranks, int32_t* __restrict__ dm, BatchSmem& sm,
                      int32_t* status) {
  const int32_t n = jb.n, m = jb.m, k = jb.k;
  const bool full = k >= m - 1;
  const int32_t nbt = (m + kTT - 1) / kTT;
  const int tid = threadIdx.x, g = tid / tiles::kThreads, lt = tid % tiles::kThreads;
  const int tx = lt % (kTT / 4), ty = lt / (kTT / 4);
  // Full rankings with one group per tile: the tiles above the diagonal are
  // tasks of their own, and the 8 x 4 thread blocks of the diagonal tiles on
  // or above the diagonal (tx >= 2 ty: 72 of 128 per tile) are packed into
  // tasks of 128 blocks; the blocks below are mirrored with the lower tiles.
  const bool packdiag = full && jb.gpt == 1;
  const int32_t noff = nbt * (nbt - 1) / 2;
  const int32_t ntiles = !full ? nbt * nbt : packdiag ? noff + (nbt * kDiagBlocks + 127) / 128 : nbt * (nbt + 1) / 2;
  // positions are below 2^15 (m <= 1024): the row operand carries the guard
  // bits of count_lt2
  const uint32_t unl = uint32_t(k) & 0xFFFFu, unl2 = unl | (unl << 16) | kGuard2;
  const int32_t mpad = int32_t(align_up(size_t(m), kTT));
  const int chunk = jb.chunk;  // chunk * mpad * 6 <= sizeof(BatchSmem), chunk * k <= kBT * kPrefetch (plan)
  const int gpt = jb.gpt, tpr = kGroups / gpt;  // tiles per round
  // a last round with fewer tiles than groups shares them out: one tile to
  // all four groups, two tiles to two groups each
  const int32_t rem_last = ntiles % tpr;
  const int gpt_last = rem_last == 0 ? gpt : kGroups / (rem_last == 1 ? 1 : rem_last == 2 ? 2 : 4);
  uint32_t* dup = reinterpret_cast<uint32_t*>(sm.raw);                         // [chunk][mpad]
  uint16_t* pos = reinterpret_cast<uint16_t*>(sm.raw + size_t(chunk) * mpad * 4);  // [chunk][mpad]
  // ballot ids of a step: thread tid holds positions q0 + u * lanes of ballot
  // vv of the step; the next step's ids are loaded before this step's counts
  const int lanes = kBT / chunk;
  const int vv = tid / lanes, q0 = tid % lanes;
  int32_t cv[kPrefetch];
  auto load_ids = [&](int64_t v0n) {
    const bool have = v0n + vv < n;
    const int32_t* row = ranks + (v0n + vv) * k;
#pragma unroll
    for (int u = 0; u < kPrefetch; ++u) {
      const int32_t q = q0 + u * lanes;
      cv[u] = (have && q < k) ? __ldcg(row + q) : -1;  // L2 only: see schulze_batch_run_host
    }
  };
  if (gpt > 1 || gpt_last > 1)  // the groups of a tile add into d (visible after the first barrier below)
    for (int64_t t = tid; t < int64_t(m) * m; t += kBT) dm[t] = 0;
  for (int32_t t0 = 0; t0 < ntiles; t0 += tpr) {
    // this group's task and its share of the staged ballots; the thread's
    // 8 x 4 block of d starts at row R0, column C0 (act: it has one)
    const int gr = ntiles - t0 < tpr ? gpt_last : gpt, phase = g % gr;
    const int32_t tt = t0 + g / gr;
    int32_t R0 = 0, C0 = 0;
    bool act = tt < ntiles;
    if (act) {
      if (packdiag && tt >= noff) {  // packed blocks of the diagonal tiles
        const int32_t idx = (tt - noff) * 128 + lt;
        act = idx < nbt * kDiagBlocks;
        const int32_t dt = idx / kDiagBlocks;
        int blk = idx % kDiagBlocks, by = 0;
        while (blk >= kTT / 4 - 2 * by) blk -= kTT / 4 - 2 * by, ++by;  // row group by holds 16 - 2 by blocks
        R0 = dt * kTT + by * 8, C0 = dt * kTT + (2 * by + blk) * 4;
      } else {
        int32_t bi = 0, bj = 0;
        if (full) {  // tiles bi <= bj in order (bi < bj when the diagonal is packed)
          const int32_t dlt = packdiag ? 1 : 0;
          int32_t rem = tt;
          while (rem >= nbt - bi - dlt) rem -= nbt - bi - dlt, ++bi;
          bj = bi + dlt + rem;
        } else {
          bi = tt / nbt, bj = tt % nbt;
        }
        R0 = bi * kTT + ty * 8, C0 = bj * kTT + tx * 4;
      }
    }
    const bool check = t0 == 0;
    uint32_t acc[8][2];
#pragma unroll
    for (int r = 0; r < 8; ++r) acc[r][0] = acc[r][1] = 0u;
    bool first_flush = true;
    load_ids(0);
    for (int64_t v0 = 0; v0 < n; v0 += chunk) {
      const int nv = int(n - v0 < chunk ? n - v0 : int64_t(chunk));
      __syncthreads();
      if (k < m || check) {  // unlisted candidates sit at position k
        for (int t = tid; t < chunk * mpad; t += kBT) {
          dup[t] = unl2;
          pos[t] = uint16_t(unl);
        }
        __syncthreads();
      } else if (mpad > m) {  // full ballots fill 0..m-1; the padding stays unlisted
        for (int t = tid; t < chunk * (mpad - m); t += kBT) {
          const int w = t / (mpad - m), c = m + t % (mpad - m);
          dup[w * mpad + c] = unl2;
          pos[w * mpad + c] = uint16_t(unl);
        }
      }
      if (vv < nv) {  // this step's ids, loaded during the previous step
#pragma unroll
        for (int u = 0; u < kPrefetch; ++u) {
          const int32_t q = q0 + u * lanes;
          if (q >= k) break;
          const int32_t c = cv[u];
          if (c < 0 || c >= m) {
            if (check) set_status(status, SCHULZE_EDATA);
            continue;
          }
          const uint32_t q2 = uint32_t(q) | (uint32_t(q) << 16) | kGuard2;
          if (check) {
            if (atomicExch(&dup[vv * mpad + c], q2) != unl2) set_status(status, SCHULZE_EDATA);
          } else {
            dup[vv * mpad + c] = q2;
          }
          pos[vv * mpad + c] = uint16_t(q);
        }
      }
      if (v0 + chunk < n) load_ids(v0 + chunk);  // in flight while this step counts
      __syncthreads();
      if (act) {
        for (int u = phase; u < nv; u += gr) {
          uint32_t a[8], b[2];
          const uint4 a0 = *reinterpret_cast<const uint4*>(&dup[u * mpad + R0]);
          const uint4 a1 = *reinterpret_cast<const uint4*>(&dup[u * mpad + R0 + 4]);
          a[0] = a0.x, a[1] = a0.y, a[2] = a0.z, a[3] = a0.w, a[4] = a1.x, a[5] = a1.y, a[6] = a1.z, a[7] = a1.w;
          const uint2 bv = *reinterpret_cast<const uint2*>(&pos[u * mpad + C0]);
          b[0] = bv.x, b[1] = bv.y;
#pragma unroll
          for (int r = 0; r < 8; ++r) {
            acc[r][0] = count_lt2(acc[r][0], a[r], b[0]);
            acc[r][1] = count_lt2(acc[r][1], a[r], b[1]);
          }
        }
        const bool last = v0 + chunk >= n;
        if (last || ((v0 + chunk) % kFlushVoters) == 0) {
#pragma unroll
          for (int r = 0; r < 8; ++r) {
            const int32_t i = R0 + r;
#pragma unroll
            for (int w = 0; w < 2; ++w) {
              const int32_t j = C0 + 2 * w;
              if (i < m) {
                int32_t* dst = dm + int64_t(i) * m + j;
                const int32_t lo = int32_t(acc[r][w] & 0xFFFFu), hi = int32_t(acc[r][w] >> 16);
                if (gr > 1) {
                  if (j < m && lo) atomicAdd(dst, lo);
                  if (j + 1 < m && hi) atomicAdd(dst + 1, hi);
                } else {
                  if (j < m) dst[0] = (first_flush ? 0 : dst[0]) + lo;
                  if (j + 1 < m) dst[1] = (first_flush ? 0 : dst[1]) + hi;
                }
              }
            }
            acc[r][0] = acc[r][1] = 0u;
          }
          first_flush = false;
        }
      }
    }
  }
  __syncthreads();
  if (full && (nbt > 1 || packdiag)) {
    // the tiles below the diagonal and, when packed, the blocks of the
    // diagonal tiles below it (column block (j % 64) / 4 < 2 (i % 64) / 8)
    for (int64_t t = threadIdx.x; t < int64_t(m) * m; t += kBT) {
      const int32_t i = int32_t(t / m), j = int32_t(t % m);
      if (i / kTT > j / kTT || (packdiag && i / kTT == j / kTT && (j % kTT) / 4 < 2 * ((i % kTT) / 8)))
        dm[t] = n - dm[int64_t(j) * m + i];
    }
  }
  __syncthreads();
}

// ----------------------------------------------------------- stages

template <typename E>
__device__ void pack(const int32_t* __restrict__ dm, int32_t m, int32_t mp, E* __restrict__ W) {
  for (int64_t t = threadIdx.x; t < int64_t(mp) * mp; t += kBT) {
    const int32_t i = int32_t(t / mp), j = int32_t(t % mp);
    int32_t out = 0;
    if (i < m && j < m && i != j) {
      const int32_t a = dm[int64_t(i) * m + j], b = dm[int64_t(j) * m + i];
      if (a > b) out = a;
    }
    W[t] = E(out);
  }
  __syncthreads();
}

template <typename E>
__device__ void closure(E* __restrict__ W, int32_t mp, BatchSmem& sm) {
  using Ops = tiles::Ops<E>;
  const int32_t nb = mp / tiles::kB;
  const int g = threadIdx.x / tiles::kThreads, lt = threadIdx.x % tiles::kThreads;
  const tiles::GroupBarrier bar{1 + g};
  auto& ts = sizeof(E) == 2 ? reinterpret_cast<typename Ops::Smem*>(sm.c16.t)[g]
                            : reinterpret_cast<typename Ops::Smem*>(sm.c32.t)[g];
  int32_t(*rowbuf)[tiles::kB] = sizeof(E) == 2 ? sm.c16.rowbuf : sm.c32.rowbuf;
  for (int32_t r = 0; r < nb; ++r) {
    if (g == 0) tiles::diag_closure<E>(W, mp, r, rowbuf, lt, bar);
    __syncthreads();
    for (int32_t t = g; t < 2 * (nb - 1); t += kGroups) {  // row, then column panel tiles
      if (t < nb - 1)
        Ops::update(W, mp, r, t + (t >= r), r, ts, lt, bar);
      else
        Ops::update(W, mp, (t - (nb - 1)) + ((t - (nb - 1)) >= r), r, r, ts, lt, bar);
    }
    __syncthreads();
    for (int32_t t = g; t < (nb - 1) * (nb - 1); t += kGroups) {
      int32_t i = t / (nb - 1), j = t % (nb - 1);
      Ops::update(W, mp, i + (i >= r), j + (j >= r), r, ts, lt, bar);
    }
    __syncthreads();
  }
}

template <typename E>
__device__ void extract(const Job& jb, const E* __restrict__ W, int32_t mp, const BatchArgs& a, BatchSmem& sm) {
  const int32_t m = jb.m;
  int32_t* bb = sm.bb;
  for (int32_t i = threadIdx.x; i < m; i += kBT) bb[i] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int32_t i = w; i < m; i += kBT / 32) {
    int32_t beaten_i = 0;
    for (int32_t j0 = i + 1 + lane; j0 < m; j0 += 32 * 4) {
      int32_t wij[4], wji[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {  // loads first: the transposed ones are strided
        const int32_t j = j0 + 32 * u;
        wij[u] = j < m ? int32_t(W[int64_t(i) * mp + j]) : 0;
        wji[u] = j < m ? int32_t(W[int64_t(j) * mp + i]) : 0;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (wji[u] > wij[u]) ++beaten_i;
        else if (wij[u] > wji[u]) atomicAdd(&bb[j0 + 32 * u], 1);
      }
    }
    for (int o = 16; o; o >>= 1) beaten_i += __shfl_xor_sync(0xFFFFFFFFu, beaten_i, o);
    if (lane == 0 && beaten_i) atomicAdd(&bb[i], beaten_i);
  }
  __syncthreads();
  for (int32_t i = threadIdx.x; i < m; i += kBT) {
    const int32_t mine = bb[i];
    if (a.winners) a.winners[jb.vec_off + i] = mine == 0;
    if (a.beaten_by) a.beaten_by[jb.vec_off + i] = mine;
    if (a.order) {
      int32_t pos = 0;
      for (int32_t j = 0; j < m; ++j) {
        const int32_t o = bb[j];
        pos += (o < mine) || (o == mine && j < i);
      }
      a.order[jb.vec_off + pos] = i;
    }
  }
  if (a.p) {
    int32_t* pm = a.p + jb.mat_off;
    for (int64_t t = threadIdx.x; t < int64_t(m) * m; t += kBT) {
      const int32_t i = int32_t(t / m), j = int32_t(t % m);
      pm[t] = (i == j) ? 0 : int32_t(W[int64_t(i) * mp + j]);
    }
  }
  __syncthreads();
}

template <typename E>
__global__ void __launch_bounds__(kBT, 1) batch_kernel(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BatchSmem& sm = *reinterpret_cast<BatchSmem*>(smem_raw);
  __shared__ int32_t s_job;
  unsigned char* slot = a.scratch + size_t(blockIdx.x) * a.slot_bytes;
  E* W = reinterpret_cast<E*>(slot);
  int32_t* dslot = reinterpret_cast<int32_t*>(slot + a.w_bytes);
  for (;;) {
    if (threadIdx.x == 0) s_job = int32_t(atomicAdd(a.head, 1u));
    __syncthreads();
    const int32_t ji = s_job;
    __syncthreads();
    if (ji >= a.njobs) return;
    const Job jb = a.jobs[ji];
    if (a.seg_flag) {
      // the job's ballots may still be on their way: thread 0 waits (bounded)
      // for its segment's arrival mark, which the copy stream writes after
      // the segment's copy; the ballots are then read from L2, where the copy
      // landed (the tally reads them with L2-only loads, so no line cached in
      // L1 before the mark can be stale)
      __shared__ int32_t s_arrived;
      if (threadIdx.x == 0) {
        const long long t0 = clock64();
        int32_t seen = 0;
        for (;;) {
          asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(seen) : "l"(a.seg_flag + jb.seg) : "memory");
          if (seen || clock64() - t0 > a.wait_limit) break;
          __nanosleep(200);
        }
        if (!seen) set_status(a.status, SCHULZE_ETIMEOUT);
        s_arrived = seen;
      }
      __syncthreads();
      if (!s_arrived) return;  // this CTA stops; the status word reports the timeout
    }
    const int32_t* ranks = a.ranks + jb.ranks_off;
    int32_t* dm = a.d ? a.d + jb.mat_off : dslot;
    const int32_t m = jb.m;
    if (jb.n == 0 || jb.k == 0) {
      for (int64_t t = threadIdx.x; t < int64_t(m) * m; t += kBT) dm[t] = 0;
      __syncthreads();
    } else {
      tally(jb, ranks, dm, sm, a.status);
    }
    const int32_t mp = int32_t(align_up(size_t(m), tiles::kB));
    pack<E>(dm, m, mp, W);
    closure<E>(W, mp, sm);
    extract<E>(jb, W, mp, a, sm);
  }
}

}  // namespace
}  // namespace schulze

struct schulze_batch {
  schulze_ctx* ctx = nullptr;
  int32_t E = 0;
  bool s16 = true;
  int32_t m_max = 0;
  std::vector<schulze::Job> jobs_host;  // in queue order
  std::vector<int64_t> ranks_off, mat_off, vec_off;  // in the caller's order
  int64_t ranks_elems = 0, mat_elems = 0, vec_elems = 0;
  schulze::Job* jobs_dev = nullptr;
  uint32_t* head = nullptr;
  unsigned char* scratch = nullptr;
  size_t slot_bytes = 0, w_bytes = 0;
  int grid = 0;
  int32_t tally_policy = 0;  // 0: each m-bucket's ballots per step; 1: eight everywhere
  int32_t order_policy = 0;  // 0 longest first, 1 the caller's order
  int32_t bucket_chunk[schulze::kBuckets] = {32, 32, 32, 16, 16};
  int32_t bucket_gpt[schulze::kBuckets] = {1, 1, 1, 1, 1};
  size_t smem = 0;
  // schulze_batch_run_host (allocated at its first call): device ballots and
  // outputs, the caller's elections cut into segments of about equal ballot
  // bytes with each segment's job table (longest first), the copy stream and
  // one event per segment
  int32_t* host_ranks = nullptr;
  int32_t* host_out = nullptr;  // winners [vec_elems], then order [vec_elems]
  int32_t* seg_flag = nullptr;  // arrival mark per segment
  int32_t* host_one = nullptr;  // page-locked 1, copied into a mark
  schulze::Job* seg_jobs_dev = nullptr;
  std::vector<int32_t> seg_elec0;  // per segment: its first election
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t flags_clear = nullptr;
};

namespace schulze {
namespace {

double job_cost(const Job& j) {
  const double m = j.m, n = j.n, k = j.k;
  const double tally = (k >= m - 1 ? 0.5 : 1.0) * n * m * m;
  const double mp = std::ceil(m / 64.0) * 64.0;
  return tally + 1.5 * mp * mp * mp;
}

// Whether `chunk` ballots of an election with m candidates can be staged:
// the position rows fit the shared memory, and a thread holds at most
// kPrefetch ids of a step (chunk * m <= kBT * kPrefetch, as k <= m).
bool chunk_fits(int32_t m, int32_t chunk) {
  const size_t mpad = align_up(size_t(m), 64);
  return chunk >= 1 && chunk <= kBT && size_t(chunk) * mpad * 6 <= kStageBytes &&
         int64_t(chunk) * m <= int64_t(kBT) * kPrefetch;
}

int32_t job_chunk(const schulze_batch* b, int32_t m) {
  if (b->tally_policy == 1) return 8;
  int32_t c = b->bucket_chunk[bucket_of(m)];
  while (c > 8 && !chunk_fits(m, c)) c /= 2;
  return c;
}

int32_t job_gpt(const schulze_batch* b, int32_t m) { return b->tally_policy == 1 ? 1 : b->bucket_gpt[bucket_of(m)]; }

bool gpt_valid(int32_t g) { return g == 1 || g == 2 || g == 4; }

void order_jobs(schulze_batch* b) {
  std::vector<Job> js(size_t(b->E));
  for (int32_t e = 0; e < b->E; ++e) js[e] = b->jobs_host[e];
  std::sort(js.begin(), js.end(), [](const Job& x, const Job& y) { return x.e < y.e; });
  if (b->order_policy == 0)
    std::stable_sort(js.begin(), js.end(), [](const Job& x, const Job& y) { return job_cost(x) > job_cost(y); });
  for (Job& j : js) j.chunk = job_chunk(b, j.m), j.gpt = job_gpt(b, j.m);
  b->jobs_host = js;
}

int upload_jobs(schulze_batch* b) {
  if (b->E == 0) return SCHULZE_OK;
  if (cudaMemcpy(b->jobs_dev, b->jobs_host.data(), sizeof(Job) * size_t(b->E), cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return SCHULZE_ECUDA;
  return SCHULZE_OK;
}

// One launch over `njobs` jobs of the uploaded table (the whole plan, or a
// subset uploaded by the autotuner), outputs to the per-CTA scratch or the
// caller's buffers.
int launch_jobs(schulze_batch* b, int32_t njobs, const int32_t* ranks, int32_t* d, int32_t* p, int32_t* winners,
                int32_t* order, int32_t* beaten_by, cudaStream_t stream, const Job* jobs = nullptr,
                const int32_t* seg_flag = nullptr) {
  if (cudaMemsetAsync(b->head, 0, 4, stream) != cudaSuccess) return SCHULZE_ECUDA;
  BatchArgs a;
  a.jobs = jobs ? jobs : b->jobs_dev;
  a.seg_flag = seg_flag;
  a.wait_limit = b->ctx->wait_limit_cycles;
  a.njobs = njobs;
  a.head = b->head;
  a.ranks = ranks;
  a.d = d, a.p = p, a.winners = winners, a.order = order, a.beaten_by = beaten_by;
  a.scratch = b->scratch;
  a.slot_bytes = b->slot_bytes;
  a.w_bytes = b->w_bytes;
  a.status = b->ctx->status;
  Launch L(b->ctx, stream, "batch_elections", double(njobs));
  if (b->s16)
    batch_kernel<int16_t><<<b->grid, kBT, b->smem, stream>>>(a);
  else
    batch_kernel<int32_t><<<b->grid, kBT, b->smem, stream>>>(a);
  return check_launch();
}

size_t batch_smem(bool s16) {
  (void)s16;
  return sizeof(BatchSmem);
}

}  // namespace
}  // namespace schulze

using namespace schulze;

extern "C" {

int schulze_batch_create(schulze_ctx* ctx, int32_t E, const int32_t* n, const int32_t* m, const int32_t* k,
                         schulze_batch** out) {
  AbiRange abi_range("schulze_batch_create");
  if (!ctx || !out || E < 0 || (E > 0 && (!n || !m || !k))) return SCHULZE_EINVAL;
  *out = nullptr;
  for (int32_t e = 0; e < E; ++e)
    if (m[e] < 1 || m[e] > kBatchMaxM || n[e] < 0 || k[e] < 0 || k[e] > m[e]) return SCHULZE_EINVAL;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return SCHULZE_ECUDA;
  schulze_batch* b = new (std::nothrow) schulze_batch();
  if (!b) return SCHULZE_ENOMEM;
  b->ctx = ctx;
  b->E = E;
  b->ranks_off.resize(size_t(E));
  b->mat_off.resize(size_t(E));
  b->vec_off.resize(size_t(E));
  b->jobs_host.resize(size_t(E));
  int64_t ro = 0, mo = 0, vo = 0;
  for (int32_t e = 0; e < E; ++e) {
    b->ranks_off[e] = ro, b->mat_off[e] = mo, b->vec_off[e] = vo;
    b->jobs_host[e] = Job{n[e], m[e], k[e], e, ro, mo, vo};
    ro += int64_t(n[e]) * k[e];
    mo += int64_t(m[e]) * m[e];
    vo += m[e];
    b->m_max = std::max(b->m_max, m[e]);
    if (n[e] > 32767) b->s16 = false;
  }
  b->ranks_elems = ro, b->mat_elems = mo, b->vec_elems = vo;
  order_jobs(b);
  b->smem = batch_smem(b->s16);
  int per_sm = 0;
  const void* fn = b->s16 ? reinterpret_cast<const void*>(batch_kernel<int16_t>)
                          : reinterpret_cast<const void*>(batch_kernel<int32_t>);
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(b->smem));
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBT, b->smem) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    delete b;
    return SCHULZE_ECUDA;
  }
  b->grid = int(std::max<int64_t>(1, std::min<int64_t>(int64_t(per_sm) * ctx->sm_count, std::max(E, 1))));
  const size_t mp = align_up(size_t(std::max(b->m_max, 1)), tiles::kB);
  b->w_bytes = align_up(mp * mp * (b->s16 ? 2 : 4), 256);
  b->slot_bytes = b->w_bytes + align_up(size_t(b->m_max) * size_t(b->m_max) * 4, 256);
  if (cudaMalloc(&b->jobs_dev, sizeof(Job) * size_t(std::max(E, 1))) != cudaSuccess ||
      cudaMalloc(&b->head, 256) != cudaSuccess ||
      cudaMalloc(&b->scratch, b->slot_bytes * size_t(b->grid)) != cudaSuccess) {
    cudaGetLastError();
    if (b->jobs_dev) cudaFree(b->jobs_dev);
    if (b->head) cudaFree(b->head);
    if (b->scratch) cudaFree(b->scratch);
    delete b;
    return SCHULZE_ENOMEM;
  }
  if (int rc = upload_jobs(b)) {
    schulze_batch_destroy(b);
    return rc;
  }
  *out = b;
  return SCHULZE_OK;
}

int schulze_batch_destroy(schulze_batch* b) {
  if (!b) return SCHULZE_EINVAL;
  cudaSetDevice(b->ctx->device);
  cudaDeviceSynchronize();
  cudaFree(b->jobs_dev);
  cudaFree(b->head);
  cudaFree(b->scratch);
  if (b->host_ranks) cudaFree(b->host_ranks);
  if (b->host_out) cudaFree(b->host_out);
  if (b->seg_jobs_dev) cudaFree(b->seg_jobs_dev);
  if (b->seg_flag) cudaFree(b->seg_flag);
  if (b->host_one) cudaFreeHost(b->host_one);
  if (b->copy_stream) cudaStreamDestroy(b->copy_stream);
  if (b->flags_clear) cudaEventDestroy(b->flags_clear);
  delete b;
  return SCHULZE_OK;
}

namespace {

// schulze_batch_run_host's state: at the first call the buffers and the
// segments of the caller's elections (contiguous ballots, about equal ballot
// bytes); at every call the job table: segment after segment, each one's
// elections longest first, with the plan's schedule of that moment.
int host_path_setup(schulze_batch* b) {
  if (!b->host_out) {
    constexpr int kSegments = 8;
    const int nseg = std::max(1, std::min<int>(kSegments, b->E));
    b->seg_elec0.assign(1, 0);
    const double per = double(std::max<int64_t>(b->ranks_elems, 1)) / nseg;
    for (int32_t e = 1; e < b->E && int(b->seg_elec0.size()) < nseg; ++e)
      if (double(b->ranks_off[e]) >= per * double(b->seg_elec0.size())) b->seg_elec0.push_back(e);
    b->seg_elec0.push_back(b->E);
    const size_t ns = b->seg_elec0.size() - 1;
    if (cudaMalloc(&b->host_ranks, sizeof(int32_t) * size_t(std::max<int64_t>(b->ranks_elems, 1))) != cudaSuccess ||
        cudaMalloc(&b->host_out, sizeof(int32_t) * 2 * size_t(std::max<int64_t>(b->vec_elems, 1))) != cudaSuccess ||
        cudaMalloc(&b->seg_jobs_dev, sizeof(Job) * size_t(b->E)) != cudaSuccess ||
        cudaMalloc(&b->seg_flag, sizeof(int32_t) * ns) != cudaSuccess ||
        cudaMallocHost(&b->host_one, sizeof(int32_t)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->flags_clear, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return SCHULZE_ENOMEM;  // what was allocated is freed by schulze_batch_destroy
    }
    *b->host_one = 1;
  }
  std::vector<Job> by_e(size_t(b->E));
  for (const Job& j : b->jobs_host) by_e[size_t(j.e)] = j;
  std::vector<Job> table;
  table.reserve(size_t(b->E));
  for (size_t s = 0; s + 1 < b->seg_elec0.size(); ++s) {
    const size_t t0 = table.size();
    for (int32_t e = b->seg_elec0[s]; e < b->seg_elec0[s + 1]; ++e) {
      table.push_back(by_e[size_t(e)]);
      table.back().seg = int32_t(s);
    }
    std::stable_sort(table.begin() + int64_t(t0), table.end(),
                     [](const Job& x, const Job& y) { return job_cost(x) > job_cost(y); });
  }
  return cudaMemcpy(b->seg_jobs_dev, table.data(), sizeof(Job) * table.size(), cudaMemcpyHostToDevice) == cudaSuccess
             ? SCHULZE_OK
             : SCHULZE_ECUDA;
}

}  // namespace

int schulze_batch_run_host(schulze_batch* b, const int32_t* ranks_host, int32_t* winners_host, int32_t* order_host,
                           schulze_stream_t stream) {
  AbiRange abi_range("schulze_batch_run_host");
  if (!b || (b->ranks_elems > 0 && !ranks_host)) return SCHULZE_EINVAL;
  if (cudaSetDevice(b->ctx->device) != cudaSuccess) return SCHULZE_ECUDA;
  if (b->E == 0) return SCHULZE_OK;
  if (int rc = host_path_setup(b)) return rc;
  const size_t ns = b->seg_elec0.size() - 1;
  int32_t* win = b->host_out;
  int32_t* ord = b->host_out + b->vec_elems;
  // the arrival marks cleared on stream, and the copy stream after that:
  // each segment's ballots, then its mark; meanwhile one launch over every
  // election on stream, each CTA waiting for the mark of its job's segment
  if (cudaMemsetAsync(b->seg_flag, 0, sizeof(int32_t) * ns, stream) != cudaSuccess ||
      cudaEventRecord(b->flags_clear, stream) != cudaSuccess ||
      cudaStreamWaitEvent(b->copy_stream, b->flags_clear, 0) != cudaSuccess)
    return SCHULZE_ECUDA;
  for (size_t s = 0; s < ns; ++s) {
    const int64_t r0 = b->ranks_off[b->seg_elec0[s]];
    const int64_t r1 = b->seg_elec0[s + 1] < b->E ? b->ranks_off[b->seg_elec0[s + 1]] : b->ranks_elems;
    if (r1 > r0 && cudaMemcpyAsync(b->host_ranks + r0, ranks_host + r0, sizeof(int32_t) * size_t(r1 - r0),
                                   cudaMemcpyHostToDevice, b->copy_stream) != cudaSuccess)
      return SCHULZE_ECUDA;
    if (cudaMemcpyAsync(b->seg_flag + s, b->host_one, sizeof(int32_t), cudaMemcpyHostToDevice, b->copy_stream) !=
        cudaSuccess)
      return SCHULZE_ECUDA;
  }
  if (int rc = launch_jobs(b, b->E, b->host_ranks, nullptr, nullptr, winners_host ? win : nullptr,
                           order_host ? ord : nullptr, nullptr, stream, b->seg_jobs_dev, b->seg_flag))
    return rc;
  const size_t vb = sizeof(int32_t) * size_t(b->vec_elems);
  if ((winners_host && cudaMemcpyAsync(winners_host, win, vb, cudaMemcpyDeviceToHost, stream) != cudaSuccess) ||
      (order_host && cudaMemcpyAsync(order_host, ord, vb, cudaMemcpyDeviceToHost, stream) != cudaSuccess))
    return SCHULZE_ECUDA;
  if (cudaStreamSynchronize(stream) != cudaSuccess || cudaStreamSynchronize(b->copy_stream) != cudaSuccess)
    return SCHULZE_ECUDA;
  return SCHULZE_OK;
}

int schulze_batch_layout(const schulze_batch* b, int64_t* ranks_elems, int64_t* mat_elems, int64_t* vec_elems,
                         int64_t* ranks_off, int64_t* mat_off, int64_t* vec_off) {
  if (!b) return SCHULZE_EINVAL;
  if (ranks_elems) *ranks_elems = b->ranks_elems;
  if (mat_elems) *mat_elems = b->mat_elems;
  if (vec_elems) *vec_elems = b->vec_elems;
  for (int32_t e = 0; e < b->E; ++e) {
    if (ranks_off) ranks_off[e] = b->ranks_off[e];
    if (mat_off) mat_off[e] = b->mat_off[e];
    if (vec_off) vec_off[e] = b->vec_off[e];
  }
  return SCHULZE_OK;
}

int schulze_batch_run(schulze_batch* b, const int32_t* ranks, int32_t* d, int32_t* p, int32_t* winners,
                      int32_t* order, int32_t* beaten_by, schulze_stream_t stream) {
  AbiRange abi_range("schulze_batch_run");
  if (!b || (b->ranks_elems > 0 && !ranks)) return SCHULZE_EINVAL;
  if (cudaSetDevice(b->ctx->device) != cudaSuccess) return SCHULZE_ECUDA;
  if (b->E == 0) return SCHULZE_OK;
  return launch_jobs(b, b->E, ranks, d, p, winners, order, beaten_by, stream);
}

int schulze_batch_set_schedule(schulze_batch* b, int32_t tally_policy, int32_t order_policy) {
  if (!b || tally_policy < 0 || tally_policy > 1 || order_policy < 0 || order_policy > 1) return SCHULZE_EINVAL;
  if (cudaSetDevice(b->ctx->device) != cudaSuccess) return SCHULZE_ECUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return SCHULZE_ECUDA;
  b->tally_policy = tally_policy;
  b->order_policy = order_policy;
  order_jobs(b);
  return upload_jobs(b);
}

int schulze_batch_set_bucket_chunk(schulze_batch* b, int32_t bucket, int32_t chunk) {
  if (!b || bucket < 0 || bucket >= kBuckets || !chunk_fits(kBucketMax[bucket], chunk) || (chunk & (chunk - 1)))
    return SCHULZE_EINVAL;
  if (cudaSetDevice(b->ctx->device) != cudaSuccess) return SCHULZE_ECUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return SCHULZE_ECUDA;
  b->bucket_chunk[bucket] = chunk;
  order_jobs(b);
  return upload_jobs(b);
}

int schulze_batch_set_bucket_tiles(schulze_batch* b, int32_t bucket, int32_t groups_per_tile) {
  if (!b || bucket < 0 || bucket >= kBuckets || !gpt_valid(groups_per_tile)) return SCHULZE_EINVAL;
  if (cudaSetDevice(b->ctx->device) != cudaSuccess) return SCHULZE_ECUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return SCHULZE_ECUDA;
  b->bucket_gpt[bucket] = groups_per_tile;
  order_jobs(b);
  return upload_jobs(b);
}

int schulze_batch_bucket_tiles(const schulze_batch* b, int32_t* groups_per_tile) {
  if (!b || !groups_per_tile) return SCHULZE_EINVAL;
  for (int q = 0; q < kBuckets; ++q) groups_per_tile[q] = b->bucket_gpt[q];
  return SCHULZE_OK;
}

int schulze_batch_bucket_schedule(const schulze_batch* b, int32_t* bucket_max_m, int32_t* chunks,
                                  int32_t* elections) {
  if (!b) return SCHULZE_EINVAL;
  for (int q = 0; q < kBuckets; ++q) {
    if (bucket_max_m) bucket_max_m[q] = kBucketMax[q];
    if (chunks) chunks[q] = b->bucket_chunk[q];
    if (elections) elections[q] = 0;
  }
  if (elections)
    for (const Job& j : b->jobs_host) ++elections[bucket_of(j.m)];
  return SCHULZE_OK;
}

int schulze_batch_autotune(schulze_batch* b, const int32_t* ranks, const char* cache_path, int32_t* best_tile,
                           int32_t* best_order, schulze_stream_t stream) {
  AbiRange abi_range("schulze_batch_autotune");
  if (!b || (b->ranks_elems > 0 && !ranks)) return SCHULZE_EINVAL;
  if (cudaSetDevice(b->ctx->device) != cudaSuccess) return SCHULZE_ECUDA;
  // cache keys: GPU, counter width, then per m-bucket its election count and
  // mean ballot count (the tally schedule), per batch its totals (the order)
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, b->ctx->device);
  auto clean = [](char* key) {
    for (char* c = key; *c; ++c)
      if (*c == ' ' || *c == '\t' || *c == '\n') *c = '_';  // the cache line format splits on blanks
  };
  std::vector<std::pair<std::string, int>> cached;
  if (cache_path) {  // line format: <key> <value>
    if (FILE* f = fopen(cache_path, "r")) {
      char line[512];
      while (fgets(line, sizeof(line), f)) {
        char k2[400];
        int v2;
        if (sscanf(line, "%399s %d", k2, &v2) == 2) cached.emplace_back(k2, v2);
      }
      fclose(f);
    }
  }
  auto lookup = [&](const char* key) {
    int v = -1;
    for (const auto& kv : cached)
      if (kv.first == key) v = kv.second;
    return v;
  };
  std::vector<std::pair<std::string, int>> fresh;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // best of two timed runs after a warm-up
  auto time_jobs = [&](int32_t njobs, float* ms_out) -> int {
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(e0, stream);
      if (int rc = launch_jobs(b, njobs, ranks, nullptr, nullptr, nullptr, nullptr, nullptr, stream)) return rc;
      cudaEventRecord(e1, stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) return SCHULZE_ECUDA;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) best = std::min(best, ms);
    }
    *ms_out = best;
    return SCHULZE_OK;
  };
  int rc = SCHULZE_OK;
  b->tally_policy = 0;
  for (int q = 0; q < kBuckets && rc == SCHULZE_OK; ++q) {
    std::vector<Job> sub;
    double nsum = 0.0;
    for (const Job& j : b->jobs_host)
      if (bucket_of(j.m) == q) sub.push_back(j), nsum += j.n;
    if (sub.empty()) continue;
    // the cached value is chunk * 8 + groups per tile
    char key[400];
    snprintf(key, sizeof(key), "%.100s|s16=%d|bucket<=%d|chunk_gpt|elections=%zu|mean_n=%lld", prop.name,
             b->s16 ? 1 : 0, kBucketMax[q], sub.size(), (long long)(nsum / double(sub.size())));
    clean(key);
    int best_v = lookup(key);
    if (best_v < 0 || !chunk_fits(kBucketMax[q], best_v / 8) || !gpt_valid(best_v % 8)) {
      // time this bucket's elections alone for every staging size that fits
      // and every number of groups per tally tile
      float best = 1e30f;
      best_v = b->bucket_chunk[q] * 8 + b->bucket_gpt[q];
      for (int c : kChunkChoices) {
        if (!chunk_fits(kBucketMax[q], c)) continue;
        for (int g : kGptChoices) {
          for (Job& j : sub) j.chunk = c, j.gpt = g;
          if (cudaMemcpy(b->jobs_dev, sub.data(), sizeof(Job) * sub.size(), cudaMemcpyHostToDevice) !=
              cudaSuccess) {
            rc = SCHULZE_ECUDA;
            break;
          }
          float ms = 0.f;
          if ((rc = time_jobs(int32_t(sub.size()), &ms)) != SCHULZE_OK) break;
          if (ms < best) best = ms, best_v = c * 8 + g;
        }
        if (rc != SCHULZE_OK) break;
      }
      fresh.emplace_back(key, best_v);
    }
    b->bucket_chunk[q] = best_v / 8;
    b->bucket_gpt[q] = best_v % 8;
  }
  int32_t bo = -1;
  if (rc == SCHULZE_OK) {
    char key[400];
    snprintf(key, sizeof(key), "%.100s|s16=%d|order|E=%d|R=%lld|M=%lld|mmax=%d", prop.name, b->s16 ? 1 : 0, b->E,
             (long long)b->ranks_elems, (long long)b->mat_elems, b->m_max);
    clean(key);
    bo = lookup(key);
    if (bo < 0 || bo > 1) {
      float best = 1e30f;
      for (int32_t o = 0; o <= 1 && rc == SCHULZE_OK; ++o) {
        b->order_policy = o;
        order_jobs(b);
        if ((rc = upload_jobs(b)) != SCHULZE_OK) break;
        float ms = 0.f;
        if ((rc = time_jobs(b->E, &ms)) != SCHULZE_OK) break;
        if (ms < best) best = ms, bo = o;
      }
      fresh.emplace_back(key, bo);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // the plan's job table back in full with the chosen schedule
  b->order_policy = bo >= 0 ? bo : 0;
  order_jobs(b);
  if (int rc2 = upload_jobs(b)) return rc2;
  if (rc != SCHULZE_OK) return rc;
  if (cache_path && !fresh.empty()) {
    if (FILE* f = fopen(cache_path, "a")) {
      for (const auto& kv : fresh) fprintf(f, "%s %d\n", kv.first.c_str(), kv.second);
      fclose(f);
    }
  }
  if (best_tile) *best_tile = 0;  // each m-bucket's own ballots per step
  if (best_order) *best_order = b->order_policy;
  return SCHULZE_OK;
}

}  // extern "C"
