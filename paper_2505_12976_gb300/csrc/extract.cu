// Winner and ranking extraction from the widest-path widths (Sect. 2.1):
// j beats i iff p[j][i] > p[i][j]; i is a winner iff nobody beats it. The
// ranking lists the ids sorted by (beaten_by, id), where beaten_by[i] counts
// the candidates that beat i; it extends the strict "beats" relation.
#include <algorithm>

#include "internal.cuh"

namespace schulze {
namespace {

constexpr int kT = 32;

// beaten_by over one 32 x 32 block pair (I, J) with I <= J: both p[I, J] and
// p[J, I] are staged in shared memory; a warp per row sums its comparisons
// and adds them with one atomic per row (and per column when I < J).
__global__ void beaten_by_kernel(const int32_t* __restrict__ p, int32_t m, int32_t nbt, int32_t* __restrict__ bb) {
  __shared__ int32_t a[kT][kT + 1];  // a[r][c] = p[I + r][J + c]
  __shared__ int32_t b[kT][kT + 1];  // b[r][c] = p[J + r][I + c]
  int32_t t = blockIdx.x, bi = 0;
  while (t >= nbt - bi) {
    t -= nbt - bi;
    ++bi;
  }
  const int32_t bj = bi + t;
  const int32_t I = bi * kT, J = bj * kT;
  const int lane = threadIdx.x, wy = threadIdx.y;  // blockDim = (32, 8)
  for (int r = wy; r < kT; r += blockDim.y) {
    int32_t i = I + r, j = J + lane;
    a[r][lane] = (i < m && j < m) ? p[int64_t(i) * m + j] : 0;
    int32_t i2 = J + r, j2 = I + lane;
    b[r][lane] = (i2 < m && j2 < m) ? p[int64_t(i2) * m + j2] : 0;
  }
  __syncthreads();
  const bool diag = bi == bj;
  // rows of I: beaten by J + c when p[J + c][I + r] > p[I + r][J + c]
  for (int r = wy; r < kT; r += blockDim.y) {
    int32_t i = I + r, j = J + lane;
    int hit = (i < m && j < m && i != j && b[lane][r] > a[r][lane]) ? 1 : 0;
    unsigned bal = __ballot_sync(0xFFFFFFFFu, hit);
    if (lane == 0 && bal && i < m) atomicAdd(&bb[i], __popc(bal));
  }
  if (!diag) {
    // rows of J: J + c beaten by I + r when p[I + r][J + c] > p[J + c][I + r]
    for (int c = wy; c < kT; c += blockDim.y) {
      int32_t j = J + c, i = I + lane;
      int hit = (i < m && j < m && a[lane][c] > b[c][lane]) ? 1 : 0;
      unsigned bal = __ballot_sync(0xFFFFFFFFu, hit);
      if (lane == 0 && bal && j < m) atomicAdd(&bb[j], __popc(bal));
    }
  }
}

__global__ void winners_kernel(const int32_t* __restrict__ bb, int32_t m, int32_t* __restrict__ win) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) win[i] = bb[i] == 0;
}

// order[pos(i)] = i with pos(i) = #{j : (bb[j], j) < (bb[i], i)}.
__global__ void rank_kernel(const int32_t* __restrict__ bb, int32_t m, int32_t* __restrict__ order) {
  __shared__ int64_t keys[1024];
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t mine = i < m ? (int64_t(bb[i]) << 32) | uint32_t(i) : INT64_MAX;
  int32_t pos = 0;
  for (int32_t j0 = 0; j0 < m; j0 += blockDim.x) {
    __syncthreads();
    int32_t j = j0 + threadIdx.x;
    keys[threadIdx.x] = j < m ? (int64_t(bb[j]) << 32) | uint32_t(j) : INT64_MAX;
    __syncthreads();
    const int lim = min(int(blockDim.x), m - j0);
    for (int t = 0; t < lim; ++t) pos += keys[t] < mine;
  }
  if (i < m) order[pos] = i;
}

}  // namespace

size_t extract_workspace_bytes(int32_t m) { return align_up(size_t(m) * 4, 256) + 4096; }

int extract_launch(schulze_ctx* ctx, const int32_t* p, int32_t m, int32_t* winners, int32_t* order,
                   int32_t* beaten_by, void* ws, cudaStream_t stream) {
  Carver cv(ws);
  int32_t* bb = beaten_by ? beaten_by : cv.take<int32_t>(size_t(m));
  if (cudaMemsetAsync(bb, 0, size_t(m) * 4, stream) != cudaSuccess) return SCHULZE_ECUDA;
  const int32_t nbt = (m + kT - 1) / kT;
  const int32_t npairs = nbt * (nbt + 1) / 2;
  {
    Launch L(ctx, stream, "extract_beaten_by", double(m) * double(m) * 4.0);
    beaten_by_kernel<<<npairs, dim3(32, 8), 0, stream>>>(p, m, nbt, bb);
  }
  const int g = (m + 255) / 256;
  if (winners) {
    Launch L(ctx, stream, "extract_winners", double(m) * 8.0);
    winners_kernel<<<g, 256, 0, stream>>>(bb, m, winners);
  }
  if (order) {
    Launch L(ctx, stream, "extract_rank", double(m) * 8.0);
    rank_kernel<<<(m + 255) / 256, 256, 0, stream>>>(bb, m, order);
  }
  return check_launch();
}

}  // namespace schulze
