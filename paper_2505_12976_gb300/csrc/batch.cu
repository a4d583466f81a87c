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
};

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
  int32_t tally_policy;  // ballots staged per tally step: 0 sixteen, 1 eight
};

// Dynamic shared memory of one batch CTA, reused stage by stage.
constexpr int kChunkMax = 16;  // ballots staged per tally step (policy 0; policy 1 stages 8)
union BatchSmem {
  struct {
    uint32_t dup[kChunkMax][kBatchMaxM];  // position of every candidate, in both 16-bit halves
    uint16_t pos[kChunkMax][kBatchMaxM];  // the same positions, one per 16-bit slot
  } stage;
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

// The election's d, tile by tile: each of the four 128-thread groups owns one
// 64 x 64 tile of d per round and counts it over all ballots in 16-bit lanes
// (two columns per word, the row operand duplicated into both halves).
// Ballots are staged `chunk` at a time as full position rows (unlisted
// candidates at position k), so one staging serves the four tiles of a
// round. Counters are added into d every kFlushVoters ballots. Full
// rankings count only the tiles on and above the diagonal and mirror the
// rest: d[j][i] = n - d[i][j]. The first round also checks the ballots: an
// id out of range, or one whose position slot is already taken within the
// same ballot, is reported as SCHULZE_EDATA.
__device__ void tally(const Job& jb, const int32_t* __restrict__ ranks, int32_t* __restrict__ dm, int chunk,
                      BatchSmem& sm, int32_t* status) {
  const int32_t n = jb.n, m = jb.m, k = jb.k;
  const bool full = k >= m - 1;
  const int32_t nbt = (m + kTT - 1) / kTT;
  const int32_t ntiles = full ? nbt * (nbt + 1) / 2 : nbt * nbt;
  const int tid = threadIdx.x, g = tid / tiles::kThreads, lt = tid % tiles::kThreads;
  const int tx = lt % (kTT / 4), ty = lt / (kTT / 4);
  // positions are below 2^15 (m <= 1024): the row operand carries the guard
  // bits of count_lt2
  const uint32_t unl = uint32_t(k) & 0xFFFFu, unl2 = unl | (unl << 16) | kGuard2;
  const int32_t mpad = int32_t(align_up(size_t(m), kTT));
  for (int32_t t0 = 0; t0 < ntiles; t0 += kGroups) {
    // this group's tile (bi, bj)
    const int32_t tt = t0 + g;
    int32_t bi = 0, bj = 0;
    if (tt < ntiles) {
      if (full) {
        int32_t rem = tt;
        while (rem >= nbt - bi) rem -= nbt - bi, ++bi;
        bj = bi + rem;
      } else {
        bi = tt / nbt, bj = tt % nbt;
      }
    }
    const int32_t I0 = bi * kTT, J0 = bj * kTT;
    const bool check = t0 == 0;
    uint32_t acc[8][2];
#pragma unroll
    for (int r = 0; r < 8; ++r) acc[r][0] = acc[r][1] = 0u;
    bool first_flush = true;
    for (int64_t v0 = 0; v0 < n; v0 += chunk) {
      const int nv = int(n - v0 < chunk ? n - v0 : int64_t(chunk));
      __syncthreads();
      if (k < m || check) {  // unlisted candidates sit at position k
        for (int t = tid; t < chunk * mpad; t += kBT) {
          const int vv = t / mpad, c = t % mpad;
          sm.stage.dup[vv][c] = unl2;
          sm.stage.pos[vv][c] = uint16_t(unl);
        }
        __syncthreads();
      } else if (mpad > m) {  // full ballots fill 0..m-1; the padding stays unlisted
        for (int t = tid; t < chunk * (mpad - m); t += kBT) {
          const int vv = t / (mpad - m), c = m + t % (mpad - m);
          sm.stage.dup[vv][c] = unl2;
          sm.stage.pos[vv][c] = uint16_t(unl);
        }
      }
      // 32 lanes per ballot row, sixteen loads in flight per thread
      const int lanes = kBT / chunk;  // threads per staged ballot (32 or 64)
      const int vv = tid / lanes, q0 = tid % lanes;
      if (vv < nv) {
        const int32_t* row = ranks + (v0 + vv) * k;
        for (int32_t qb = q0; qb < k; qb += lanes * 16) {
          int32_t cv[16];
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            const int32_t q = qb + u * lanes;
            cv[u] = q < k ? __ldcs(row + q) : -1;
          }
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            const int32_t q = qb + u * lanes;
            if (q >= k) break;
            const int32_t c = cv[u];
            if (c < 0 || c >= m) {
              if (check) set_status(status, SCHULZE_EDATA);
              continue;
            }
            const uint32_t q2 = uint32_t(q) | (uint32_t(q) << 16) | kGuard2;
            if (check) {
              if (atomicExch(&sm.stage.dup[vv][c], q2) != unl2) set_status(status, SCHULZE_EDATA);
            } else {
              sm.stage.dup[vv][c] = q2;
            }
            sm.stage.pos[vv][c] = uint16_t(q);
          }
        }
      }
      __syncthreads();
      if (tt < ntiles) {
        for (int u = 0; u < nv; ++u) {
          uint32_t a[8], b[2];
          const uint4 a0 = *reinterpret_cast<const uint4*>(&sm.stage.dup[u][I0 + ty * 8]);
          const uint4 a1 = *reinterpret_cast<const uint4*>(&sm.stage.dup[u][I0 + ty * 8 + 4]);
          a[0] = a0.x, a[1] = a0.y, a[2] = a0.z, a[3] = a0.w, a[4] = a1.x, a[5] = a1.y, a[6] = a1.z, a[7] = a1.w;
          const uint2 bv = *reinterpret_cast<const uint2*>(&sm.stage.pos[u][J0 + tx * 4]);
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
            const int32_t i = I0 + ty * 8 + r;
#pragma unroll
            for (int w = 0; w < 2; ++w) {
              const int32_t j = J0 + tx * 4 + 2 * w;
              if (i < m) {
                int32_t* dst = dm + int64_t(i) * m + j;
                if (j < m) dst[0] = (first_flush ? 0 : dst[0]) + int32_t(acc[r][w] & 0xFFFFu);
                if (j + 1 < m) dst[1] = (first_flush ? 0 : dst[1]) + int32_t(acc[r][w] >> 16);
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
  if (full && nbt > 1) {
    for (int64_t t = threadIdx.x; t < int64_t(m) * m; t += kBT) {
      const int32_t i = int32_t(t / m), j = int32_t(t % m);
      if (i / kTT > j / kTT) dm[t] = n - dm[int64_t(j) * m + i];
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
    const int32_t* ranks = a.ranks + jb.ranks_off;
    int32_t* dm = a.d ? a.d + jb.mat_off : dslot;
    const int32_t m = jb.m;
    if (jb.n == 0 || jb.k == 0) {
      for (int64_t t = threadIdx.x; t < int64_t(m) * m; t += kBT) dm[t] = 0;
      __syncthreads();
    } else {
      tally(jb, ranks, dm, a.tally_policy == 1 ? 8 : kChunkMax, sm, a.status);
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
  int32_t tally_policy = 0;
  int32_t order_policy = 0;  // 0 longest first, 1 the caller's order
  size_t smem = 0;
};

namespace schulze {
namespace {

double job_cost(const Job& j) {
  const double m = j.m, n = j.n, k = j.k;
  const double tally = (k >= m - 1 ? 0.5 : 1.0) * n * m * m;
  const double mp = std::ceil(m / 64.0) * 64.0;
  return tally + 1.5 * mp * mp * mp;
}

void order_jobs(schulze_batch* b) {
  std::vector<Job> js(size_t(b->E));
  for (int32_t e = 0; e < b->E; ++e) js[e] = b->jobs_host[e];
  std::sort(js.begin(), js.end(), [](const Job& x, const Job& y) { return x.e < y.e; });
  if (b->order_policy == 0)
    std::stable_sort(js.begin(), js.end(), [](const Job& x, const Job& y) { return job_cost(x) > job_cost(y); });
  b->jobs_host = js;
}

int upload_jobs(schulze_batch* b) {
  if (b->E == 0) return SCHULZE_OK;
  if (cudaMemcpy(b->jobs_dev, b->jobs_host.data(), sizeof(Job) * size_t(b->E), cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return SCHULZE_ECUDA;
  return SCHULZE_OK;
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
  delete b;
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
  if (!b || (b->ranks_elems > 0 && !ranks)) return SCHULZE_EINVAL;
  if (cudaSetDevice(b->ctx->device) != cudaSuccess) return SCHULZE_ECUDA;
  if (b->E == 0) return SCHULZE_OK;
  if (cudaMemsetAsync(b->head, 0, 4, stream) != cudaSuccess) return SCHULZE_ECUDA;
  BatchArgs a;
  a.jobs = b->jobs_dev;
  a.njobs = b->E;
  a.head = b->head;
  a.ranks = ranks;
  a.d = d, a.p = p, a.winners = winners, a.order = order, a.beaten_by = beaten_by;
  a.scratch = b->scratch;
  a.slot_bytes = b->slot_bytes;
  a.w_bytes = b->w_bytes;
  a.status = b->ctx->status;
  a.tally_policy = b->tally_policy;
  Launch L(b->ctx, stream, "batch_elections", double(b->E));
  if (b->s16)
    batch_kernel<int16_t><<<b->grid, kBT, b->smem, stream>>>(a);
  else
    batch_kernel<int32_t><<<b->grid, kBT, b->smem, stream>>>(a);
  return check_launch();
}

int schulze_batch_set_schedule(schulze_batch* b, int32_t tally_policy, int32_t order_policy) {
  if (!b || tally_policy < 0 || tally_policy > 1 || order_policy < 0 || order_policy > 1) return SCHULZE_EINVAL;
  if (cudaSetDevice(b->ctx->device) != cudaSuccess) return SCHULZE_ECUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return SCHULZE_ECUDA;
  b->tally_policy = tally_policy;
  if (order_policy != b->order_policy) {
    b->order_policy = order_policy;
    order_jobs(b);
    if (int rc = upload_jobs(b)) return rc;
  }
  return SCHULZE_OK;
}

int schulze_batch_autotune(schulze_batch* b, const int32_t* ranks, const char* cache_path, int32_t* best_tile,
                           int32_t* best_order, schulze_stream_t stream) {
  if (!b || (b->ranks_elems > 0 && !ranks)) return SCHULZE_EINVAL;
  if (cudaSetDevice(b->ctx->device) != cudaSuccess) return SCHULZE_ECUDA;
  // batch signature for the cache: size, totals, largest election, GPU
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, b->ctx->device);
  char key[256];
  snprintf(key, sizeof(key), "%.100s|E=%d|R=%lld|M=%lld|mmax=%d|s16=%d", prop.name, b->E,
           (long long)b->ranks_elems, (long long)b->mat_elems, b->m_max, b->s16 ? 1 : 0);
  for (char* c = key; *c; ++c)
    if (*c == ' ' || *c == '\t' || *c == '\n') *c = '_';  // the cache line format splits on blanks
  int32_t bt = -1, bo = -1;
  if (cache_path) {  // line format: <key> <tally_policy> <order_policy>
    if (FILE* f = fopen(cache_path, "r")) {
      char line[512];
      while (fgets(line, sizeof(line), f)) {
        char k2[256];
        int t2, o2;
        if (sscanf(line, "%255s %d %d", k2, &t2, &o2) == 3 && strcmp(k2, key) == 0) bt = t2, bo = o2;
      }
      fclose(f);
    }
  }
  if (bt < 0) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int32_t o = 0; o <= 1; ++o)
      for (int32_t t = 0; t <= 1; ++t) {
        if (int rc = schulze_batch_set_schedule(b, t, o)) return rc;
        float total = 0.f;
        for (int rep = 0; rep < 2; ++rep) {
          cudaEventRecord(e0, stream);
          if (int rc = schulze_batch_run(b, ranks, nullptr, nullptr, nullptr, nullptr, nullptr, stream)) return rc;
          cudaEventRecord(e1, stream);
          if (cudaEventSynchronize(e1) != cudaSuccess) return SCHULZE_ECUDA;
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (rep > 0) total += ms;  // first run warms up
        }
        if (total < best) best = total, bt = t, bo = o;
      }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cache_path) {
      if (FILE* f = fopen(cache_path, "a")) {
        fprintf(f, "%s %d %d\n", key, bt, bo);
        fclose(f);
      }
    }
  }
  if (int rc = schulze_batch_set_schedule(b, bt, bo)) return rc;
  if (best_tile) *best_tile = bt;
  if (best_order) *best_order = bo;
  return SCHULZE_OK;
}

}  // extern "C"
