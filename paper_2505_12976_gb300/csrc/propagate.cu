// Winners only, by the paper's vertex-centric algorithm (Sect. 4, Alg. 1-4),
// restated on the dense tally for one GPU: a comparator for the closure
// path. Every candidate c keeps a status (unknown / loser / winner); each
// iteration of the while-loop
//   * preprocessing (Alg. 2): unknown c starts as its own source and target
//     (s = t = c, widths "infinite"), decided ones as relays (s = t = none);
//   * forward-backward propagation (Alg. 3), in synchronous rounds until
//     nothing changes: c keeps the smallest source id reaching it and, for
//     that id, the widest width over its incoming edges (u, c) of
//     min(width at u, w(u, c)); likewise the smallest target id it reaches
//     and the widest width, against the edges;
//   * postprocessing (Alg. 4): loser marks from s < t, s > t, the widths of a
//     found SCC, and incoming edges from another SCC; then the unknown c with
//     s = t = c become winners.
// Readings: a decided status never changes (marks only turn unknown into
// loser); the optional zeroing of edges into dominated SCCs is left out.
//
// Edge weights come from d on the fly: with a = d[c][u] and b = d[u][c],
// the outgoing edge (c, u) weighs a if a > b (a - b with margins) and the
// incoming edge (u, c) weighs b if b > a. A transposed copy of d makes both
// come from row c, so a warp per candidate reads two rows, coalesced.
#include <algorithm>

#include "internal.cuh"

namespace schulze {
namespace {

constexpr int32_t kNone = 0x7fffffff;  // no id / infinite width
constexpr int32_t kUnknown = 0, kLoser = 1, kWinner = 2;
constexpr int kWarps = 8;              // candidates per CTA (a warp each)

__device__ __forceinline__ int32_t edge(int32_t x, int32_t y, bool margin) {
  return x > y ? (margin ? x - y : x) : 0;
}

// dT = d transposed, through 32 x 32 shared-memory tiles.
__global__ void transpose_kernel(const int32_t* __restrict__ d, int32_t m, int32_t* __restrict__ dT) {
  __shared__ int32_t tile[32][33];
  const int32_t bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int32_t i = by + r, j = bx + threadIdx.x;
    tile[r][threadIdx.x] = (i < m && j < m) ? d[int64_t(i) * m + j] : 0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int32_t i = bx + r, j = by + threadIdx.x;
    if (i < m && j < m) dT[int64_t(i) * m + j] = tile[threadIdx.x][r];
  }
}

// Initialisation-of-vertices (Alg. 1): c is a loser when its heaviest
// incoming edge outweighs its heaviest outgoing one. Warp per candidate.
__global__ void __launch_bounds__(32 * kWarps) init_kernel(const int32_t* __restrict__ d,
                                                           const int32_t* __restrict__ dT, int32_t m, int margin,
                                                           int32_t* __restrict__ status) {
  const int lane = threadIdx.x & 31;
  const int32_t c = blockIdx.x * kWarps + (threadIdx.x >> 5);
  if (c >= m) return;
  const int32_t* dr = d + int64_t(c) * m;
  const int32_t* tr = dT + int64_t(c) * m;
  int32_t in = 0, out = 0;
  for (int32_t u = lane; u < m; u += 32) {
    if (u == c) continue;
    const int32_t a = dr[u], b = tr[u];
    out = max(out, edge(a, b, margin));
    in = max(in, edge(b, a, margin));
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    in = max(in, __shfl_xor_sync(0xFFFFFFFFu, in, o));
    out = max(out, __shfl_xor_sync(0xFFFFFFFFu, out, o));
  }
  if (lane == 0) status[c] = in > out ? kLoser : kUnknown;
}

// Preprocessing (Alg. 2): state[c] = {s, ws, t, wt}.
__global__ void preprocess_kernel(const int32_t* __restrict__ status, int32_t m, int4* __restrict__ state) {
  for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x)
    state[c] = status[c] == kUnknown ? make_int4(c, kNone, c, kNone) : make_int4(kNone, 0, kNone, 0);
}

// (id, width) with the smallest id first and, for equal ids, the widest
// width first, as one 64-bit key (smaller is better).
__device__ __forceinline__ uint64_t key(int32_t id, int32_t width) {
  return (uint64_t(uint32_t(id)) << 32) | uint64_t(0xFFFFFFFFu - uint32_t(width));
}

// One propagation round (Alg. 3), synchronous: reads state, writes next;
// *changed is set when some candidate's pair changes.
__global__ void __launch_bounds__(32 * kWarps) propagate_kernel(const int32_t* __restrict__ d,
                                                                const int32_t* __restrict__ dT, int32_t m,
                                                                int margin, const int4* __restrict__ state,
                                                                int4* __restrict__ next, int32_t* changed) {
  const int lane = threadIdx.x & 31;
  const int32_t c = blockIdx.x * kWarps + (threadIdx.x >> 5);
  if (c >= m) return;
  const int32_t* dr = d + int64_t(c) * m;
  const int32_t* tr = dT + int64_t(c) * m;
  const int4 me = state[c];
  uint64_t fwd = key(me.x, me.y), bwd = key(me.z, me.w);
  for (int32_t u = lane; u < m; u += 32) {
    if (u == c) continue;
    const int32_t a = dr[u], b = tr[u];
    const int32_t win = edge(b, a, margin), wout = edge(a, b, margin);
    if (win == 0 && wout == 0) continue;
    const int4 su = state[u];
    if (win > 0 && su.x != kNone) fwd = min(fwd, key(su.x, min(su.y, win)));   // along (u, c)
    if (wout > 0 && su.z != kNone) bwd = min(bwd, key(su.z, min(su.w, wout)));  // against (c, u)
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    fwd = min(fwd, __shfl_xor_sync(0xFFFFFFFFu, fwd, o));
    bwd = min(bwd, __shfl_xor_sync(0xFFFFFFFFu, bwd, o));
  }
  if (lane == 0) {
    const int4 nx = make_int4(int32_t(fwd >> 32), int32_t(0xFFFFFFFFu - uint32_t(fwd)), int32_t(bwd >> 32),
                              int32_t(0xFFFFFFFFu - uint32_t(bwd)));
    next[c] = nx;
    if (nx.x != me.x || nx.y != me.y || nx.z != me.z || nx.w != me.w) *changed = 1;
  }
}

// Postprocessing (Alg. 4), the marks: lose[c] for a loser, scc_lose[x] for
// every member of the SCC labelled x (slot m stands for "no id").
__global__ void __launch_bounds__(32 * kWarps) marks_kernel(const int32_t* __restrict__ d,
                                                            const int32_t* __restrict__ dT, int32_t m, int margin,
                                                            const int4* __restrict__ state,
                                                            int32_t* __restrict__ lose,
                                                            int32_t* __restrict__ scc_lose) {
  const int lane = threadIdx.x & 31;
  const int32_t c = blockIdx.x * kWarps + (threadIdx.x >> 5);
  if (c >= m) return;
  const int4 me = state[c];
  if (lane == 0) {
    if (me.x < me.z) {
      lose[c] = 1;
    } else if (me.x > me.z) {
      lose[me.z] = 1;  // an id: t < s
    } else if (me.x != kNone) {
      if (me.y > me.w) lose[c] = 1;
      else if (me.y < me.w) lose[me.x] = 1;
    }
  }
  // an incoming edge (v, c) from another SCC
  const int32_t* dr = d + int64_t(c) * m;
  const int32_t* tr = dT + int64_t(c) * m;
  bool other = false;
  for (int32_t v = lane; v < m && !other; v += 32) {
    if (v == c || edge(tr[v], dr[v], margin) == 0) continue;
    const int4 sv = state[v];
    other = sv.x != me.x || sv.z != me.z;
  }
  if (__any_sync(0xFFFFFFFFu, other) && lane == 0) {
    if (me.x == me.z)
      scc_lose[me.x == kNone ? m : me.x] = 1;
    else
      lose[c] = 1;
  }
}

// Postprocessing, applied: unknown candidates marked (or in a marked SCC)
// become losers; then unknown c with s = t = c become winners. decided[0]
// counts the changes.
__global__ void apply_kernel(const int4* __restrict__ state, int32_t m, const int32_t* __restrict__ lose,
                             const int32_t* __restrict__ scc_lose, int32_t* __restrict__ status,
                             int32_t* __restrict__ decided) {
  for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) {
    if (status[c] != kUnknown) continue;
    const int4 me = state[c];
    const bool in_lost = me.x == me.z && scc_lose[me.x == kNone ? m : me.x];
    if (lose[c] || in_lost) {
      status[c] = kLoser;
      atomicAdd(decided, 1);
    } else if (me.x == c && me.z == c) {
      status[c] = kWinner;
      atomicAdd(decided, 1);
    }
  }
}

__global__ void winners_out_kernel(const int32_t* __restrict__ status, int32_t m, int32_t* __restrict__ winners,
                                   int32_t* __restrict__ unknown) {
  for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) {
    winners[c] = status[c] == kWinner;
    if (status[c] == kUnknown) atomicAdd(unknown, 1);
  }
}

}  // namespace

size_t propagation_workspace_bytes(int32_t m) {
  const size_t mm = align_up(size_t(m) * size_t(m) * 4, 256), mv = align_up((size_t(m) + 1) * 4, 256);
  return mm + 2 * align_up(size_t(m) * 16, 256) + 4 * mv + 4096;
}

int winners_propagation_launch(schulze_ctx* ctx, const int32_t* d, int32_t m, bool margin, int32_t* winners,
                               int32_t* stats, void* ws, cudaStream_t stream) {
  Carver cv(ws);
  int32_t* dT = cv.take<int32_t>(size_t(m) * size_t(m));
  int4* state = cv.take<int4>(size_t(m));
  int4* next = cv.take<int4>(size_t(m));
  int32_t* status = cv.take<int32_t>(size_t(m) + 1);
  int32_t* lose = cv.take<int32_t>(size_t(m) + 1);
  int32_t* scc_lose = cv.take<int32_t>(size_t(m) + 1);
  int32_t* words = cv.take<int32_t>(size_t(m) + 1);  // [0] changed, [1] decided, [2] unknown
  const int mg = margin ? 1 : 0;
  const int wb = (m + kWarps - 1) / kWarps;
  const int g = std::max(1, std::min((m + 255) / 256, 1024));
  {
    Launch L(ctx, stream, "propagation_transpose", double(m) * double(m) * 8.0);
    transpose_kernel<<<dim3((m + 31) / 32, (m + 31) / 32), dim3(32, 8), 0, stream>>>(d, m, dT);
  }
  {
    Launch L(ctx, stream, "propagation_init", double(m) * double(m) * 8.0);
    init_kernel<<<wb, 32 * kWarps, 0, stream>>>(d, dT, m, mg, status);
  }
  if (int rc = check_launch()) return rc;
  int32_t iterations = 0, rounds = 0;
  for (;;) {
    int32_t host[3] = {0, 0, 0};
    if (cudaMemsetAsync(words, 0, 3 * sizeof(int32_t), stream) != cudaSuccess) return SCHULZE_ECUDA;
    winners_out_kernel<<<g, 256, 0, stream>>>(status, m, winners, words + 2);
    if (cudaMemcpyAsync(host, words, sizeof(host), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
      return SCHULZE_ECUDA;
    if (host[2] == 0) break;  // no unknown candidate left
    if (iterations >= m) return SCHULZE_EDATA;  // every iteration decides one at least
    ++iterations;
    preprocess_kernel<<<g, 256, 0, stream>>>(status, m, state);
    // rounds until nothing changes; a chain of m candidates settles in m rounds
    for (int32_t r = 0; r <= m; ++r) {
      int32_t changed = 0;
      if (cudaMemsetAsync(words, 0, sizeof(int32_t), stream) != cudaSuccess) return SCHULZE_ECUDA;
      {
        Launch L(ctx, stream, "propagation_round", double(m) * double(m) * 8.0);
        propagate_kernel<<<wb, 32 * kWarps, 0, stream>>>(d, dT, m, mg, state, next, words);
      }
      std::swap(state, next);
      ++rounds;
      if (cudaMemcpyAsync(&changed, words, sizeof(int32_t), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
          cudaStreamSynchronize(stream) != cudaSuccess)
        return SCHULZE_ECUDA;
      if (!changed) break;
    }
    if (cudaMemsetAsync(lose, 0, (size_t(m) + 1) * 4, stream) != cudaSuccess ||
        cudaMemsetAsync(scc_lose, 0, (size_t(m) + 1) * 4, stream) != cudaSuccess)
      return SCHULZE_ECUDA;
    {
      Launch L(ctx, stream, "propagation_marks", double(m) * double(m) * 8.0);
      marks_kernel<<<wb, 32 * kWarps, 0, stream>>>(d, dT, m, mg, state, lose, scc_lose);
    }
    apply_kernel<<<g, 256, 0, stream>>>(state, m, lose, scc_lose, status, words + 1);
    int32_t decided = 0;
    if (cudaMemcpyAsync(&decided, words + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
      return SCHULZE_ECUDA;
    if (decided == 0) return SCHULZE_EDATA;  // never expected: Alg. 4 decides one candidate at least
  }
  if (stats) stats[0] = iterations, stats[1] = rounds;
  return check_launch();
}

}  // namespace schulze
