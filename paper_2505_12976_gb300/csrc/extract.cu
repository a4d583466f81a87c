// Winner and ranking extraction from the widest-path widths (Sect. 2.1):
// j beats i iff p[j][i] > p[i][j]; i is a winner iff nobody beats it. The
// ranking lists the ids sorted by (beaten_by, id), where beaten_by[i] counts
// the candidates that beat i; it extends the strict "beats" relation.
#include <algorithm>

#include "internal.cuh"

namespace schulze {
namespace {

constexpr int kT = 64;         // block of the beaten_by pass
constexpr int kRankChunk = 256;  // keys per shared-memory chunk of the rank pass

// beaten_by over one 64 x 64 block pair (I, J), I <= J (2D grid, the lower
// half exits): p[I, J] and p[J, I] are staged in shared memory, each row of
// both blocks is counted by four threads and added with one atomic per row.
__global__ void __launch_bounds__(256) beaten_by_kernel(const int32_t* __restrict__ p, int32_t m,
                                                        int32_t* __restrict__ bb) {
  const int32_t I = blockIdx.y * kT, J = blockIdx.x * kT;
  if (I > J) return;
  __shared__ int32_t a[kT][kT + 1];  // a[r][c] = p[I + r][J + c]
  __shared__ int32_t b[kT][kT + 1];  // b[r][c] = p[J + r][I + c]
  const int tid = threadIdx.x;
  for (int t = tid; t < kT * kT; t += 256) {
    const int r = t / kT, c = t % kT;
    int32_t i = I + r, j = J + c;
    a[r][c] = (i < m && j < m) ? p[int64_t(i) * m + j] : 0;
    i = J + r, j = I + c;
    b[r][c] = (i < m && j < m) ? p[int64_t(i) * m + j] : 0;
  }
  __syncthreads();
  const int r = tid >> 2, q = tid & 3;  // row r, columns q * 16 .. + 15
  // rows of I: I + r is beaten by J + c when p[J + c][I + r] > p[I + r][J + c]
  int cnt_i = 0, cnt_j = 0;
#pragma unroll
  for (int cc = 0; cc < 16; ++cc) {
    const int c = q * 16 + cc;
    const bool valid = (I + r < m) && (J + c < m) && (I + r != J + c);
    cnt_i += (valid && b[c][r] > a[r][c]) ? 1 : 0;
    // rows of J: J + r is beaten by I + c when p[I + c][J + r] > p[J + r][I + c]
    const bool valid2 = (J + r < m) && (I + c < m) && (I != J);
    cnt_j += (valid2 && a[c][r] > b[r][c]) ? 1 : 0;
  }
  cnt_i += __shfl_xor_sync(0xFFFFFFFFu, cnt_i, 1);
  cnt_i += __shfl_xor_sync(0xFFFFFFFFu, cnt_i, 2);
  cnt_j += __shfl_xor_sync(0xFFFFFFFFu, cnt_j, 1);
  cnt_j += __shfl_xor_sync(0xFFFFFFFFu, cnt_j, 2);
  if (q == 0) {
    if (cnt_i) atomicAdd(&bb[I + r], cnt_i);
    if (cnt_j) atomicAdd(&bb[J + r], cnt_j);
  }
}

__global__ void winners_kernel(const int32_t* __restrict__ bb, int32_t m, int32_t* __restrict__ win) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) win[i] = bb[i] == 0;
}

// pos[i] += #{j in this CTA's chunk : (bb[j], j) < (bb[i], i)}; 2D grid over
// (chunks of i, chunks of j), pos zeroed before.
__global__ void __launch_bounds__(256) rank_count_kernel(const int32_t* __restrict__ bb, int32_t m,
                                                         int32_t* __restrict__ pos) {
  pdl_enter();
  __shared__ int64_t keys[kRankChunk];
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t mine = i < m ? (int64_t(bb[i]) << 32) | uint32_t(i) : INT64_MAX;
  const int32_t j0 = blockIdx.y * kRankChunk;
  const int32_t j = j0 + threadIdx.x;
  keys[threadIdx.x] = j < m ? (int64_t(bb[j]) << 32) | uint32_t(j) : INT64_MAX;
  __syncthreads();
  const int lim = min(kRankChunk, m - j0);
  int32_t c = 0;
  for (int t = 0; t < lim; ++t) c += keys[t] < mine;
  if (i < m && c) atomicAdd(&pos[i], c);
}

// order[pos[i]] = i; with winners, also winners[i] = (bb[i] == 0).
__global__ void rank_scatter_kernel(const int32_t* __restrict__ pos, const int32_t* __restrict__ bb, int32_t m,
                                    int32_t* __restrict__ order, int32_t* __restrict__ winners) {
  pdl_enter();
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    order[pos[i]] = i;
    if (winners) winners[i] = bb[i] == 0;
  }
}

// winners and ranking from beaten_by; pos is scratch [m]
int finish(schulze_ctx* ctx, const int32_t* bb, int32_t* pos, int32_t m, int32_t* winners, int32_t* order,
           cudaStream_t stream) {
  const int g = (m + 255) / 256;
  if (order) {
    ZeroSpans z;
    z.p[0] = reinterpret_cast<uint32_t*>(pos), z.words[0] = m;
    if (int rc = zero_async(ctx, z, stream)) return rc;
    {
      Launch L(ctx, stream, "extract_rank", double(m) * 8.0);
      launch_pdl(rank_count_kernel, dim3(g, (m + kRankChunk - 1) / kRankChunk), dim3(256), 0, stream, false, bb, m,
                 pos);
    }
    Launch L(ctx, stream, "extract_order", double(m) * 8.0);
    launch_pdl(rank_scatter_kernel, dim3(g), dim3(256), 0, stream, false, static_cast<const int32_t*>(pos), bb, m,
               order, winners);
  } else if (winners) {
    Launch L(ctx, stream, "extract_winners", double(m) * 8.0);
    winners_kernel<<<g, 256, 0, stream>>>(bb, m, winners);
  }
  return check_launch();
}

// Iterated winner removal, one level: every candidate not yet placed
// (level 0) that no remaining candidate beats gets level t and is appended
// to placed[1 + ...] (placed[0] counts them). Placed candidates are isolated
// in the working d, so they neither beat nor are beaten.
__global__ void iter_level_kernel(const int32_t* __restrict__ bb, int32_t m, int32_t t, int32_t* __restrict__ level,
                                  int32_t* __restrict__ placed) {
  for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x)
    if (level[c] == 0 && bb[c] == 0) {
      level[c] = t;
      placed[1 + atomicAdd(&placed[0], 1)] = c;
    }
}

// Zeroes row c and column c of the working d for every c placed in this level.
__global__ void iter_isolate_kernel(int32_t* __restrict__ dw, int32_t m, const int32_t* __restrict__ placed) {
  const int32_t cnt = placed[0];
  const int64_t total = int64_t(cnt) * m;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int32_t c = placed[1 + int32_t(e / m)], x = int32_t(e % m);
    dw[int64_t(c) * m + x] = 0;
    dw[int64_t(x) * m + c] = 0;
  }
}

}  // namespace

size_t extract_workspace_bytes(int32_t m) { return 2 * align_up(size_t(m) * 4, 256) + 4096; }

int extract_launch(schulze_ctx* ctx, const int32_t* p, int32_t m, int32_t* winners, int32_t* order,
                   int32_t* beaten_by, void* ws, cudaStream_t stream) {
  Carver cv(ws);
  int32_t* bb = beaten_by ? beaten_by : cv.take<int32_t>(size_t(m));
  int32_t* pos = cv.take<int32_t>(size_t(m));
  if (cudaMemsetAsync(bb, 0, size_t(m) * 4, stream) != cudaSuccess) return SCHULZE_ECUDA;
  const int32_t nbt = (m + kT - 1) / kT;
  {
    Launch L(ctx, stream, "extract_beaten_by", double(m) * double(m) * 4.0);
    beaten_by_kernel<<<dim3(nbt, nbt), 256, 0, stream>>>(p, m, bb);
  }
  if (int rc = check_launch()) return rc;
  return finish(ctx, bb, pos, m, winners, order, stream);
}

int extract_from_beaten_by(schulze_ctx* ctx, const int32_t* beaten_by, int32_t m, int32_t* winners, int32_t* order,
                           void* ws, cudaStream_t stream) {
  Carver cv(ws);
  int32_t* pos = cv.take<int32_t>(size_t(m));
  return finish(ctx, beaten_by, pos, m, winners, order, stream);
}

int iterated_level(schulze_ctx* ctx, const int32_t* bb, int32_t m, int32_t t, int32_t* level, int32_t* placed,
                   int32_t* dw, cudaStream_t stream) {
  if (cudaMemsetAsync(placed, 0, sizeof(int32_t), stream) != cudaSuccess) return SCHULZE_ECUDA;
  const int g = std::max(1, std::min((m + 255) / 256, 1024));
  {
    Launch L(ctx, stream, "iterated_level", double(m) * 8.0);
    iter_level_kernel<<<g, 256, 0, stream>>>(bb, m, t, level, placed);
  }
  Launch L(ctx, stream, "iterated_isolate", 0.0);
  iter_isolate_kernel<<<std::max(1, std::min(m, 2048)), 256, 0, stream>>>(dw, m, placed);
  return check_launch();
}

}  // namespace schulze
