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
// The closure runs on W in rounds of B = 64 candidates; round r
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
#include <algorithm>
#include <mutex>

#include "internal.cuh"
#include "tiles.cuh"

namespace schulze {
namespace {

using tiles::kB;        // block / tile size
using tiles::kThreads;  // threads per CTA
using tiles::BlockBarrier;
using tiles::Ops;
using tiles::diag_closure;

constexpr uint32_t kNZ = 1u << 30;         // progress word: tile has a nonzero entry
constexpr uint32_t kRoundMask = kNZ - 1u;  // progress word: rounds applied
constexpr long long kSpinLimitCycles = 4000000000LL;  // ~2 s at 2 GHz

// ------------------------------------------------------------ relabel

// rowflag[i] = 1 iff candidate i has an outgoing edge (some j with
// d[i][j] > d[j][i]). One CTA per 32 x 32 block pair (A, B), A <= B, reading
// each d entry once.
__global__ void rowflag_kernel(const int32_t* __restrict__ d, int32_t m, int32_t* __restrict__ rowflag) {
  const int32_t A = blockIdx.y * 32, B = blockIdx.x * 32;
  if (A > B) return;
  __shared__ int32_t t1[32][33], t2[32][33];  // t1 = d[A.., B..], t2 = d[B.., A..]
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int32_t i = A + r, j = B + threadIdx.x;
    t1[r][threadIdx.x] = (i < m && j < m) ? d[int64_t(i) * m + j] : 0;
    i = B + r, j = A + threadIdx.x;
    t2[r][threadIdx.x] = (i < m && j < m) ? d[int64_t(i) * m + j] : 0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    // row A + r: edge to B + c when t1[r][c] > t2[c][r]
    int32_t i = A + r, j = B + threadIdx.x;
    bool e1 = i < m && j < m && i != j && t1[r][threadIdx.x] > t2[threadIdx.x][r];
    if (__any_sync(0xFFFFFFFFu, e1) && threadIdx.x == 0 && i < m) atomicOr(&rowflag[i], 1);
    // row B + r: edge to A + c when t2[r][c] > t1[c][r]
    i = B + r, j = A + threadIdx.x;
    bool e2 = i < m && j < m && i != j && t2[r][threadIdx.x] > t1[threadIdx.x][r];
    if (__any_sync(0xFFFFFFFFu, e2) && threadIdx.x == 0 && i < m) atomicOr(&rowflag[i], 1);
  }
}

// Stable partition: perm[new] = old, candidates with edges first; inv[old] = new.
__global__ void __launch_bounds__(1024) relabel_kernel(const int32_t* __restrict__ rowflag, int32_t m,
                                                       int32_t* __restrict__ perm, int32_t* __restrict__ inv,
                                                       int32_t* __restrict__ warm_out) {
  __shared__ int32_t part[1024];
  const int T = blockDim.x;
  const int per = (m + T - 1) / T;
  const int b = threadIdx.x * per, e = min(m, b + per);
  int32_t s = 0;
  for (int c = b; c < e; ++c) s += rowflag[c] ? 1 : 0;
  part[threadIdx.x] = s;
  __syncthreads();
  for (int o = 1; o < T; o <<= 1) {
    int32_t x = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += x;
    __syncthreads();
  }
  const int32_t warm = part[T - 1];
  if (threadIdx.x == 0) *warm_out = warm;
  int32_t before = threadIdx.x ? part[threadIdx.x - 1] : 0;  // warm candidates before b
  for (int c = b; c < e; ++c) {
    int32_t nw;
    if (rowflag[c]) {
      nw = before++;
    } else {
      nw = warm + (c - before);  // cold ones keep their order after the warm ones
    }
    perm[nw] = c;
    inv[c] = nw;
  }
}

// ---------------------------------------------------------------- pack

// W[a][b] = w[perm[a]][perm[b]] (0 outside m x m, on the diagonal and where
// d does not beat its transpose). One CTA per 32 x 32 block pair (A, B),
// A <= B, writing both W[A][B] and W[B][A]; a warp that writes a nonzero sets
// the nonzero bit of its 64 x 64 tile's progress word.
template <typename E>
__global__ void pack_kernel(const int32_t* __restrict__ d, int32_t m, int32_t mp, int64_t bound,
                            const int32_t* __restrict__ perm, E* __restrict__ W, uint32_t* __restrict__ prog,
                            int32_t nb, int32_t* status) {
  const int32_t A = blockIdx.y * 32, B = blockIdx.x * 32;
  if (A > B) return;
  __shared__ int32_t t1[32][33], t2[32][33];  // t1[r][c] = d[perm[A+r]][perm[B+c]], t2 = (B, A)
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int32_t a = A + r, b = B + threadIdx.x;
    t1[r][threadIdx.x] = (a < m && b < m) ? d[int64_t(perm[a]) * m + perm[b]] : 0;
    a = B + r, b = A + threadIdx.x;
    t2[r][threadIdx.x] = (a < m && b < m) ? d[int64_t(perm[a]) * m + perm[b]] : 0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int32_t a = (side ? B : A) + r, b = (side ? A : B) + threadIdx.x;
      const int32_t x = side ? t2[r][threadIdx.x] : t1[r][threadIdx.x];
      const int32_t y = side ? t1[threadIdx.x][r] : t2[threadIdx.x][r];
      int32_t out = 0;
      if (a < m && b < m) {
        if (x < 0 || int64_t(x) > bound) set_status(status, SCHULZE_EDATA);
        if (a != b && x > y) out = x;
      }
      if (a < mp && b < mp) W[int64_t(a) * mp + b] = E(out);
      if (__any_sync(0xFFFFFFFFu, out != 0) && threadIdx.x == 0)
        atomicOr(&prog[(a / kB) * nb + (b / kB)], kNZ);
      if (A == B) break;  // a diagonal block pair is one block
    }
  }
}

// p[x][y] = W[inv[x]][inv[y]] for x != y < m; p[x][x] = 0.
template <typename E>
__global__ void widen_kernel(const E* __restrict__ W, int32_t mp, int32_t m, const int32_t* __restrict__ inv,
                             int32_t* __restrict__ p) {
  const int32_t x = blockIdx.y;
  const int32_t ix = inv[x];
  const E* wrow = W + int64_t(ix) * mp;
  int32_t* prow = p + int64_t(x) * m;
  for (int32_t y = blockIdx.x * blockDim.x + threadIdx.x; y < m; y += gridDim.x * blockDim.x)
    prow[y] = (y == x) ? 0 : int32_t(wrow[inv[y]]);
}

// ----------------------------------------------------- work queue

enum ItemKind : int32_t { kDiag = 0, kPanel = 1, kTile = 2 };
struct Item {
  int32_t kind, r, i, j;
};

// The candidates with outgoing edges occupy the first nbr tile rows after
// relabeling; the other rows of W are zero and stay zero, and a round over a
// block of them cannot change anything (min(x, 0) = 0). So rounds run over
// r < nbr and only tile rows i < nbr are updated, against all nb tile
// columns: nbr * nbr * nb items in total.
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
    if (clock64() - t0 > kSpinLimitCycles) {
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

template <typename E>
__global__ void __launch_bounds__(kThreads) closure_persistent_kernel(E* __restrict__ W, int32_t ld, int32_t nb,
                                                                       Sync sy) {
  __shared__ __align__(16) typename Ops<E>::Smem sm;
  __shared__ __align__(16) int32_t rowbuf[2][kB];
  __shared__ int32_t s_item[4];
  __shared__ uint32_t s_flags;
  constexpr uint32_t kFail = 0xFFFFFFFFu;
  const int32_t nbr = (*sy.warm + kB - 1) / kB;
  const Shape sh = make_shape(nbr, nb);
  const int64_t total_items = int64_t(nbr) * nbr * nb;
  for (;;) {
    if (threadIdx.x == 0) {
      const int64_t t = int64_t(atomicAdd(sy.head, 1u));
      Item it{-1, 0, 0, 0};
      uint32_t flags = 0;  // bit 0: skip the update; bit 1: tile already nonzero
      if (t < total_items && !*reinterpret_cast<volatile uint32_t*>(sy.abort_flag)) {
        it = decode_item(t, sh);
        const uint32_t r = uint32_t(it.r);
        const uint32_t own = wait_round(sy, it.i * nb + it.j, r);  // rounds 0 .. r-1 applied
        uint32_t ok = own;
        if (own != kFail) {
          if (it.kind == kDiag) {
            if (!(own & kNZ)) flags |= 1u;
          } else if (it.kind == kPanel) {
            const uint32_t dg = wait_round(sy, it.r * nb + it.r, r + 1);
            ok = dg;
            if (dg != kFail && (!(dg & kNZ) || !(own & kNZ))) flags |= 1u;
          } else {
            const uint32_t pa = wait_round(sy, it.i * nb + it.r, r + 1);
            const uint32_t pb = pa != kFail ? wait_round(sy, it.r * nb + it.j, r + 1) : kFail;
            ok = pb;
            if (pb != kFail && (!(pa & kNZ) || !(pb & kNZ))) flags |= 1u;
          }
        }
        if (ok == kFail) {
          it.kind = -1;
        } else {
          __threadfence();
          if (own & kNZ) flags |= 2u;
        }
      }
      s_item[0] = it.kind, s_item[1] = it.r, s_item[2] = it.i, s_item[3] = it.j;
      s_flags = flags;
    }
    __syncthreads();
    const int32_t kind = s_item[0], r = s_item[1], i = s_item[2], j = s_item[3];
    const uint32_t flags = s_flags;
    __syncthreads();
    if (kind < 0) return;
    bool nz = (flags & 2u) != 0;
    if (!(flags & 1u)) {
      if (kind == kDiag)
        nz = diag_closure<E>(W, ld, r, rowbuf, threadIdx.x, BlockBarrier{});
      else
        nz = Ops<E>::update(W, ld, i, j, r, sm, threadIdx.x, BlockBarrier{});
    }
    if (threadIdx.x == 0) {
      publish(sy, i * nb + j, uint32_t(r + 1) | (nz ? kNZ : 0u));
      if (!(flags & 1u)) atomicAdd(&sy.counters[kind == kDiag ? 1 : 0], 1ull);
      atomicAdd(&sy.counters[2], 1ull);
    }
  }
}

template <typename E>
int run_closure(schulze_ctx* ctx, const int32_t* d, int32_t m, int64_t bound, int32_t* p, void* ws,
                cudaStream_t stream) {
  const int32_t mp = int32_t(align_up(size_t(m), kB));
  const int32_t nb = mp / kB;
  Carver cv(ws);
  E* W = cv.take<E>(size_t(mp) * size_t(mp));
  uint32_t* prog = cv.take<uint32_t>(size_t(nb) * size_t(nb) + 2);
  int32_t* rowflag = cv.take<int32_t>(size_t(m));
  int32_t* perm = cv.take<int32_t>(size_t(m));
  int32_t* inv = cv.take<int32_t>(size_t(m));
  int32_t* warm = cv.take<int32_t>(1);
  uint32_t* head = prog + size_t(nb) * size_t(nb);
  uint32_t* abort_flag = head + 1;
  if (cudaMemsetAsync(prog, 0, (size_t(nb) * nb + 2) * 4, stream) != cudaSuccess) return SCHULZE_ECUDA;
  if (cudaMemsetAsync(rowflag, 0, size_t(m) * 4, stream) != cudaSuccess) return SCHULZE_ECUDA;
  const double mm = double(m) * double(m);
  const int32_t nb32 = (m + 31) / 32;
  {
    Launch L(ctx, stream, "closure_rowflags", mm * 4.0);
    rowflag_kernel<<<dim3(nb32, nb32), dim3(32, 8), 0, stream>>>(d, m, rowflag);
  }
  {
    Launch L(ctx, stream, "closure_relabel", double(m) * 12.0);
    relabel_kernel<<<1, 1024, 0, stream>>>(rowflag, m, perm, inv, warm);
  }
  {
    Launch L(ctx, stream, "closure_pack", mm * (4.0 + sizeof(E)));
    const int32_t mp32 = mp / 32;
    pack_kernel<E><<<dim3(mp32, mp32), dim3(32, 8), 0, stream>>>(d, m, mp, bound, perm, W, prog, nb, ctx->status);
  }
  if (int rc = check_launch()) return rc;
  {
    // persistent grid: every CTA resident (cooperative launch)
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, closure_persistent_kernel<E>, kThreads, 0) !=
            cudaSuccess ||
        per_sm < 1)
      return SCHULZE_ECUDA;
    const int sms = ctx->sm_count > 0 ? ctx->sm_count : 1;
    const int64_t max_items = int64_t(nb) * nb * nb;
    const int grid = int(std::min<int64_t>(int64_t(per_sm) * sms, max_items));
    Sync sy{prog, head, abort_flag, ctx->status, warm, ctx->counters};
    E* Wp = W;
    int32_t ldp = mp, nbp = nb;
    void* args[] = {&Wp, &ldp, &nbp, &sy};
    Launch L(ctx, stream, "closure_persistent", double(m) * mm);
    if (cudaLaunchCooperativeKernel(reinterpret_cast<void*>(closure_persistent_kernel<E>), dim3(grid),
                                    dim3(kThreads), args, 0, stream) != cudaSuccess) {
      cudaGetLastError();
      return SCHULZE_ECUDA;
    }
  }
  {
    Launch L(ctx, stream, "closure_widen", mm * (4.0 + sizeof(E)));
    const int32_t gx = std::max(1, std::min<int32_t>((m + 255) / 256, 8));
    widen_kernel<E><<<dim3(gx, m), 256, 0, stream>>>(W, mp, m, inv, p);
  }
  return check_launch();
}

}  // namespace

size_t closure_workspace_bytes(int32_t m, int64_t bound, uint32_t flags) {
  size_t mp = align_up(size_t(m), kB);
  size_t nb = mp / kB;
  return align_up(mp * mp * (use_s16(bound, flags) ? 2 : 4), 256) + align_up((nb * nb + 2) * 4, 256) +
         4 * align_up(size_t(m) * 4, 256) + 4096;
}

int closure_launch(schulze_ctx* ctx, const int32_t* d, int32_t m, int64_t bound, int32_t* p, uint32_t flags,
                   void* ws, cudaStream_t stream) {
  if (use_s16(bound, flags)) return run_closure<int16_t>(ctx, d, m, bound, p, ws, stream);
  return run_closure<int32_t>(ctx, d, m, bound, p, ws, stream);
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
                       int32_t* status, cudaStream_t stream) {
  const int32_t mp = int32_t(align_up(size_t(m), kB));
  const int32_t nb = mp / kB;
  E* W = reinterpret_cast<E*>(base + kStW);
  uint32_t* prog = reinterpret_cast<uint32_t*>(base + kStProg);
  int32_t* rowflag = reinterpret_cast<int32_t*>(base + kStRowflag);
  int32_t* perm = reinterpret_cast<int32_t*>(base + kStPerm);
  int32_t* inv = reinterpret_cast<int32_t*>(base + kStInv);
  int32_t* warm = reinterpret_cast<int32_t*>(base + kStWarm);
  auto* counters = reinterpret_cast<unsigned long long*>(base + kStCounters);
  uint32_t* head = prog + size_t(nb) * size_t(nb);
  uint32_t* abort_flag = head + 1;
  // the array keeps the previous call's contents: reset what must start at zero
  if (cudaMemsetAsync(prog, 0, (size_t(nb) * nb + 2) * 4, stream) != cudaSuccess) return SCHULZE_ECUDA;
  if (cudaMemsetAsync(rowflag, 0, size_t(m) * 4, stream) != cudaSuccess) return SCHULZE_ECUDA;
  const int32_t nb32 = (m + 31) / 32;
  rowflag_kernel<<<dim3(nb32, nb32), dim3(32, 8), 0, stream>>>(d, m, rowflag);
  relabel_kernel<<<1, 1024, 0, stream>>>(rowflag, m, perm, inv, warm);
  const int32_t mp32 = mp / 32;
  pack_kernel<E><<<dim3(mp32, mp32), dim3(32, 8), 0, stream>>>(d, m, mp, bound, perm, W, prog, nb, status);
  if (int rc = check_launch()) return rc;
  int per_sm = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, closure_persistent_kernel<E>, kThreads, 0) !=
          cudaSuccess ||
      per_sm < 1 || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms < 1)
    return SCHULZE_ECUDA;
  const int grid = int(std::min<int64_t>(int64_t(per_sm) * sms, int64_t(nb) * nb * nb));
  Sync sy{prog, head, abort_flag, status, warm, counters};
  E* Wp = W;
  int32_t ldp = mp, nbp = nb;
  void* args[] = {&Wp, &ldp, &nbp, &sy};
  if (cudaLaunchCooperativeKernel(reinterpret_cast<void*>(closure_persistent_kernel<E>), dim3(grid), dim3(kThreads),
                                  args, 0, stream) != cudaSuccess) {
    cudaGetLastError();
    return SCHULZE_ECUDA;
  }
  const int32_t gx = std::max(1, std::min<int32_t>((m + 255) / 256, 8));
  widen_kernel<E><<<dim3(gx, m), 256, 0, stream>>>(W, mp, m, inv, p);
  return check_launch();
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
  if (use_s16(bound, flags)) return run_closure_static<int16_t>(base, device, d, m, bound, p, status, stream);
  return run_closure_static<int32_t>(base, device, d, m, bound, p, status, stream);
}
