// Context, workspace and the public entry points of include/schulze.h.
#include <stdlib.h>

#include <algorithm>
#include <new>

#include "internal.cuh"

namespace schulze {

int side_join(schulze_ctx* ctx, cudaStream_t stream) {
  if (!ctx || !ctx->side_pending) return SCHULZE_OK;
  ctx->side_pending = false;
  return cudaStreamWaitEvent(stream, ctx->side_join, 0) == cudaSuccess ? SCHULZE_OK : SCHULZE_ECUDA;
}

int ensure_workspace(schulze_ctx* ctx, size_t bytes, cudaStream_t stream) {
  if (bytes <= ctx->ws.bytes) return SCHULZE_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess) return SCHULZE_ECUDA;
  if (cs != cudaStreamCaptureStatusNone) return SCHULZE_ERANGE;
  // Grow geometrically so that a sweep of sizes does not reallocate each call.
  size_t want = std::max(bytes, ctx->ws.bytes + ctx->ws.bytes / 2);
  want = align_up(want, size_t(1) << 20);
  if (ctx->ws.base) {
    // Work queued on any stream may still use the old buffer.
    if (cudaDeviceSynchronize() != cudaSuccess) return SCHULZE_ECUDA;
    cudaFree(ctx->ws.base);
    ctx->ws.base = nullptr;
    ctx->ws.bytes = 0;
  }
  void* p = nullptr;
  if (cudaMalloc(&p, want) != cudaSuccess) {
    cudaGetLastError();
    return SCHULZE_ENOMEM;
  }
  ctx->ws.base = p;
  ctx->ws.bytes = want;
  return SCHULZE_OK;
}

bool use_s16(int64_t bound, uint32_t flags) {
  if (flags & SCHULZE_F_FORCE_S32) return false;
  if (flags & SCHULZE_F_FORCE_S16) return true;
  return bound <= 32767;
}

static int set_device(schulze_ctx* ctx) {
  return cudaSetDevice(ctx->device) == cudaSuccess ? SCHULZE_OK : SCHULZE_ECUDA;
}

}  // namespace schulze

using namespace schulze;

// Page-locked host memory (or no buffer): graph copy nodes need it; calls
// with pageable buffers run eagerly.
static bool pinned(const void* ptr) {
  if (!ptr) return true;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

// Makes ctx->host_exec the graph of schulze_run_host's work for `key`,
// capturing enqueue(cap_stream, host_status) when the key changed; false
// when the call cannot be a graph (pageable host buffers, a failed capture)
// and must run eagerly.
template <class Enqueue>
static bool host_graph(schulze_ctx* ctx, const schulze_ctx::HostKey& key, Enqueue&& enqueue) {
  if (!ctx->cap_stream || !ctx->host_status) return false;
  if (ctx->host_exec && ctx->host_key == key) return true;
  if (!pinned(key.ranks) || !pinned(key.winners) || !pinned(key.order)) return false;
  if (ctx->host_exec) {
    cudaGraphExecDestroy(ctx->host_exec);
    ctx->host_exec = nullptr;
    ctx->host_key = schulze_ctx::HostKey{};
  }
  if (cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const int rc = enqueue(ctx->cap_stream, ctx->host_status);
  cudaGraph_t g = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(ctx->cap_stream, &g);
  cudaGraphExec_t exec = nullptr;
  const bool ok = rc == SCHULZE_OK && ec == cudaSuccess && g && cudaGraphInstantiate(&exec, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  if (!ok) {
    cudaGetLastError();
    if (exec) cudaGraphExecDestroy(exec);
    return false;
  }
  ctx->host_exec = exec;
  ctx->host_key = key;
  return true;
}

extern "C" {

int schulze_set_wait_limit(schulze_ctx* ctx, int64_t cycles) {
  if (!ctx || cycles < 1) return SCHULZE_EINVAL;
  if (ctx->wait_limit_cycles != cycles && ctx->host_exec) {
    // schulze_run_host's cached graph holds the old limit in its launches
    if (cudaSetDevice(ctx->device) != cudaSuccess) return SCHULZE_ECUDA;
    cudaGraphExecDestroy(ctx->host_exec);
    ctx->host_exec = nullptr;
    ctx->host_key = schulze_ctx::HostKey{};
  }
  ctx->wait_limit_cycles = cycles;
  return SCHULZE_OK;
}

const char* schulze_strerror(int code) {
  switch (code) {
    case SCHULZE_OK: return "ok";
    case SCHULZE_EINVAL: return "invalid argument";
    case SCHULZE_ENOMEM: return "out of device memory for the workspace";
    case SCHULZE_ECUDA: return "CUDA runtime or launch failure";
    case SCHULZE_EDATA: return "invalid data: ballot id out of range or repeated, or count out of range";
    case SCHULZE_ETIMEOUT: return "a bounded device wait gave up";
    case SCHULZE_ERANGE: return "workspace too small during stream capture (call schulze_reserve first)";
    case SCHULZE_ETOOBIG: return "m above 1024, the limit of the allocation-free schulze_strongest_paths_static";
    default: return "unknown status";
  }
}

int schulze_ctx_create(int device, schulze_ctx** out) {
  if (!out) return SCHULZE_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return device < 0 ? SCHULZE_EINVAL : SCHULZE_ECUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return SCHULZE_ECUDA;
  schulze_ctx* c = new (std::nothrow) schulze_ctx();
  if (!c) return SCHULZE_ENOMEM;
  c->device = device;
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  c->smem_optin = size_t(optin);
  // one small device block: status word, then the closure work counters
  if (cudaMalloc(&c->status, 64) != cudaSuccess || cudaMemset(c->status, 0, 64) != cudaSuccess) {
    cudaGetLastError();
    if (c->status) cudaFree(c->status);
    delete c;
    return SCHULZE_ENOMEM;
  }
  c->counters = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(c->status) + 8);
  // schulze_run_host's graph: its capture stream and page-locked status word
  // (without them that call runs eagerly)
  if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMallocHost(&c->host_status, sizeof(int32_t)) != cudaSuccess) {
    cudaGetLastError();
    c->host_status = nullptr;
  }
  // the side stream of schulze_run (without it p is written on the call's
  // stream)
  if (cudaStreamCreateWithFlags(&c->side_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->side_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->side_join, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    if (c->side_stream) cudaStreamDestroy(c->side_stream);
    if (c->side_fork) cudaEventDestroy(c->side_fork);
    if (c->side_join) cudaEventDestroy(c->side_join);
    c->side_stream = nullptr, c->side_fork = nullptr, c->side_join = nullptr;
  }
  *out = c;
  return SCHULZE_OK;
}

int schulze_ctx_destroy(schulze_ctx* ctx) {
  if (!ctx) return SCHULZE_EINVAL;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  if (ctx->ws.base) cudaFree(ctx->ws.base);
  if (ctx->status) cudaFree(ctx->status);
  if (ctx->host_exec) cudaGraphExecDestroy(ctx->host_exec);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->side_stream) cudaStreamDestroy(ctx->side_stream);
  if (ctx->side_fork) cudaEventDestroy(ctx->side_fork);
  if (ctx->side_join) cudaEventDestroy(ctx->side_join);
  if (ctx->host_status) cudaFreeHost(ctx->host_status);
  delete ctx;
  return SCHULZE_OK;
}

size_t schulze_workspace_bytes(const schulze_ctx* ctx) { return ctx ? ctx->ws.bytes : 0; }

int schulze_reserve(schulze_ctx* ctx, int32_t m_max, int64_t n_max, int32_t k_max) {
  if (!ctx || m_max < 1 || m_max > kMaxM || n_max < 0 || k_max < 0 || k_max > m_max) return SCHULZE_EINVAL;
  if (int rc = set_device(ctx)) return rc;
  size_t t = std::max(tally_workspace_bytes(n_max, m_max, k_max, 0),
                      std::max(tally_workspace_bytes(n_max, m_max, k_max, SCHULZE_F_TALLY_DENSE),
                               tally_workspace_bytes(n_max, m_max, k_max, SCHULZE_F_TALLY_SPARSE)));
  size_t c = std::max(closure_workspace_bytes(m_max, n_max, 0), closure_workspace_bytes(m_max, 1, 0));
  size_t x = extract_workspace_bytes(m_max);
  // schulze_run keeps the tally's warm flags (with their relabeling) and
  // beaten_by after the stages, then the extraction's scratch
  const size_t mv = align_up(size_t(m_max) * 4, 256), hv = align_up(hint_words(m_max) * 4, 256);
  size_t need = align_up(std::max(t, c), 256) + hv + mv + 256 + x;
  // schulze_run_host keeps ranks, d, p, three vectors and the hint words
  // next to the stages
  size_t host_path = align_up(size_t(n_max) * size_t(k_max) * 4, 256) +
                     2 * align_up(size_t(m_max) * size_t(m_max) * 4, 256) + 3 * mv + hv + 512 + need + 4096;
  need = std::max(need, host_path);
  int rc = ensure_workspace(ctx, need, nullptr);
  if (rc) return rc;
  return cudaDeviceSynchronize() == cudaSuccess ? SCHULZE_OK : SCHULZE_ECUDA;
}

int schulze_get_status(schulze_ctx* ctx, int32_t* status, schulze_stream_t stream) {
  if (!ctx || !status) return SCHULZE_EINVAL;
  if (int rc = set_device(ctx)) return rc;
  int32_t h = 0;
  if (cudaMemcpyAsync(&h, ctx->status, sizeof(int32_t), cudaMemcpyDeviceToHost, stream) != cudaSuccess)
    return SCHULZE_ECUDA;
  if (cudaMemsetAsync(ctx->status, 0, sizeof(int32_t), stream) != cudaSuccess) return SCHULZE_ECUDA;
  if (cudaStreamSynchronize(stream) != cudaSuccess) return SCHULZE_ECUDA;
  *status = h;
  return SCHULZE_OK;
}

int schulze_tally(schulze_ctx* ctx, const int32_t* ranks, int64_t n, int32_t m, int32_t k, int32_t* d,
                  uint32_t flags, schulze_stream_t stream) {
  AbiRange abi_range("schulze_tally");
  if (!ctx || !d || m < 1 || m > kMaxM || k < 0 || k > m || n < 0 || n >= (int64_t(1) << 31) ||
      uint64_t(n) * uint64_t(k) >= (uint64_t(1) << 32) || (n > 0 && k > 0 && !ranks))
    return SCHULZE_EINVAL;
  if ((flags & SCHULZE_F_TALLY_DENSE) && (flags & SCHULZE_F_TALLY_SPARSE)) return SCHULZE_EINVAL;
  if (int rc = set_device(ctx)) return rc;
  if (int rc = ensure_workspace(ctx, tally_workspace_bytes(n, m, k, flags), stream)) return rc;
  return tally_launch(ctx, ranks, n, m, k, d, flags, ctx->ws.base, stream);
}

int schulze_tally_positions(schulze_ctx* ctx, const int32_t* pos, int64_t n, int32_t m, int32_t* d,
                            schulze_stream_t stream) {
  AbiRange abi_range("schulze_tally_positions");
  if (!ctx || !d || m < 1 || m > kMaxM || n < 0 || n >= (int64_t(1) << 31) ||
      uint64_t(n) * uint64_t(m) >= (uint64_t(1) << 40) || (n > 0 && !pos))
    return SCHULZE_EINVAL;
  if (int rc = set_device(ctx)) return rc;
  if (int rc = ensure_workspace(ctx, tally_positions_workspace_bytes(n, m), stream)) return rc;
  return tally_positions_launch(ctx, pos, n, m, d, ctx->ws.base, stream);
}

int schulze_strongest_paths(schulze_ctx* ctx, const int32_t* d, int32_t m, int64_t bound, int32_t* p,
                            uint32_t flags, schulze_stream_t stream) {
  AbiRange abi_range("schulze_strongest_paths");
  if (!ctx || !d || !p || d == p || m < 1 || m > kMaxM || bound < 0) return SCHULZE_EINVAL;
  if ((flags & SCHULZE_F_FORCE_S16) && ((flags & SCHULZE_F_FORCE_S32) || bound > 32767)) return SCHULZE_EINVAL;
  if (int rc = set_device(ctx)) return rc;
  if (int rc = ensure_workspace(ctx, closure_workspace_bytes(m, bound, flags), stream)) return rc;
  return closure_launch(ctx, d, m, bound, p, flags, ctx->ws.base, stream);
}

int schulze_winners(schulze_ctx* ctx, const int32_t* p, int32_t m, int32_t* winners, schulze_stream_t stream) {
  AbiRange abi_range("schulze_winners");
  if (!ctx || !p || !winners || m < 1 || m > kMaxM) return SCHULZE_EINVAL;
  if (int rc = set_device(ctx)) return rc;
  if (int rc = ensure_workspace(ctx, extract_workspace_bytes(m), stream)) return rc;
  return extract_launch(ctx, p, m, winners, nullptr, nullptr, ctx->ws.base, stream);
}

int schulze_ranking(schulze_ctx* ctx, const int32_t* p, int32_t m, int32_t* order, int32_t* beaten_by,
                    schulze_stream_t stream) {
  AbiRange abi_range("schulze_ranking");
  if (!ctx || !p || !order || m < 1 || m > kMaxM) return SCHULZE_EINVAL;
  if (int rc = set_device(ctx)) return rc;
  if (int rc = ensure_workspace(ctx, extract_workspace_bytes(m), stream)) return rc;
  return extract_launch(ctx, p, m, nullptr, order, beaten_by, ctx->ws.base, stream);
}

int schulze_ranking_iterated(schulze_ctx* ctx, const int32_t* d, int32_t m, int64_t bound, int32_t k_top,
                             int32_t* level, int32_t* levels, uint32_t flags, schulze_stream_t stream) {
  AbiRange abi_range("schulze_ranking_iterated");
  if (!ctx || !d || !level || m < 1 || m > kMaxM || bound < 0 || k_top < 1) return SCHULZE_EINVAL;
  if ((flags & SCHULZE_F_FORCE_S16) && ((flags & SCHULZE_F_FORCE_S32) || bound > 32767)) return SCHULZE_EINVAL;
  if (int rc = set_device(ctx)) return rc;
  const size_t mm = align_up(size_t(m) * size_t(m) * 4, 256), mv = align_up(size_t(m + 1) * 4, 256);
  const size_t cws = align_up(closure_workspace_bytes(m, bound, flags), 256);
  if (int rc = ensure_workspace(ctx, cws + 2 * mm + 2 * mv + 256, stream)) return rc;
  char* base = static_cast<char*>(ctx->ws.base);
  int32_t* dw = reinterpret_cast<int32_t*>(base + cws);
  int32_t* p = reinterpret_cast<int32_t*>(base + cws + mm);
  int32_t* bb = reinterpret_cast<int32_t*>(base + cws + 2 * mm);
  int32_t* placed = reinterpret_cast<int32_t*>(base + cws + 2 * mm + mv);
  if (cudaMemsetAsync(level, 0, size_t(m) * 4, stream) != cudaSuccess ||
      cudaMemcpyAsync(dw, d, size_t(m) * size_t(m) * 4, cudaMemcpyDeviceToDevice, stream) != cudaSuccess)
    return SCHULZE_ECUDA;
  const int32_t target = std::min(k_top, m);
  int32_t total = 0, t = 0;
  while (total < target) {
    ++t;
    if (int rc = closure_launch(ctx, dw, m, bound, p, flags, ctx->ws.base, stream, bb)) return rc;
    if (int rc = iterated_level(ctx, bb, m, t, level, placed, dw, stream)) return rc;
    int32_t now = 0;
    if (cudaMemcpyAsync(&now, placed, sizeof(int32_t), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
      return SCHULZE_ECUDA;
    if (now <= 0) return SCHULZE_EDATA;  // a nonempty winner set is guaranteed for valid data
    total += now;
  }
  if (levels) *levels = t;
  return SCHULZE_OK;
}

int schulze_winners_propagation(schulze_ctx* ctx, const int32_t* d, int32_t m, uint32_t flags, int32_t* winners,
                                int32_t* stats, schulze_stream_t stream) {
  AbiRange abi_range("schulze_winners_propagation");
  if (!ctx || !d || !winners || m < 1 || m > kMaxM) return SCHULZE_EINVAL;
  if (int rc = set_device(ctx)) return rc;
  if (int rc = ensure_workspace(ctx, propagation_workspace_bytes(m), stream)) return rc;
  return winners_propagation_launch(ctx, d, m, (flags & SCHULZE_F_MARGIN) != 0, winners, stats, ctx->ws.base,
                                    stream);
}

int schulze_run(schulze_ctx* ctx, const int32_t* ranks, int64_t n, int32_t m, int32_t k, int32_t* d, int32_t* p,
                int32_t* winners, int32_t* order, int32_t* beaten_by, uint32_t flags, schulze_stream_t stream) {
  AbiRange abi_range("schulze_run");
  if (!ctx || !d || !p || d == p || m < 1 || m > kMaxM || k < 0 || k > m || n < 0 ||
      n >= (int64_t(1) << 31) || uint64_t(n) * uint64_t(k) >= (uint64_t(1) << 32) || (n > 0 && k > 0 && !ranks))
    return SCHULZE_EINVAL;
  if ((flags & SCHULZE_F_TALLY_DENSE) && (flags & SCHULZE_F_TALLY_SPARSE)) return SCHULZE_EINVAL;
  if ((flags & SCHULZE_F_FORCE_S16) && ((flags & SCHULZE_F_FORCE_S32) || n > 32767)) return SCHULZE_EINVAL;
  if (int rc = set_device(ctx)) return rc;
  // workspace: the stages' scratch (tally, then closure, from the start),
  // then the tally's warm flags with their relabeling and beaten_by (kept
  // across the stages), then the extraction's scratch (the winners and the
  // ranking are extracted while p is still being written from the closure's
  // scratch on the side stream)
  const size_t mv = align_up(size_t(m) * 4, 256), hv = align_up(hint_words(m) * 4, 256);
  const size_t keep = std::max(align_up(tally_workspace_bytes(n, m, k, flags), 256),
                               align_up(closure_workspace_bytes(m, n, flags), 256));
  const size_t xoff = keep + hv + mv + 256;
  if (int rc = ensure_workspace(ctx, xoff + extract_workspace_bytes(m), stream)) return rc;
  char* tail = static_cast<char*>(ctx->ws.base) + keep;
  int32_t* hint = reinterpret_cast<int32_t*>(tail);
  int32_t* hint_valid = reinterpret_cast<int32_t*>(tail + hv);
  int32_t* bb = beaten_by ? beaten_by : reinterpret_cast<int32_t*>(tail + hv + 256);
  void* xws = static_cast<char*>(ctx->ws.base) + xoff;
  if (int rc = tally_launch(ctx, ranks, n, m, k, d, flags, ctx->ws.base, stream, hint, hint_valid)) return rc;
  const bool ext = winners || order || beaten_by;
  int rc = closure_launch(ctx, d, m, n, p, flags, ctx->ws.base, stream, ext ? bb : nullptr, hint, hint_valid, true);
  if (!rc && ext && (winners || order)) rc = extract_from_beaten_by(ctx, bb, m, winners, order, xws, stream);
  const int rj = side_join(ctx, stream);  // also after an error: a capture must end with the fork joined
  return rc ? rc : rj;
}

int schulze_run_host(schulze_ctx* ctx, const int32_t* ranks_host, int64_t n, int32_t m, int32_t k,
                     int32_t* winners_host, int32_t* order_host, uint32_t flags, schulze_stream_t stream) {
  AbiRange abi_range("schulze_run_host");
  if (!ctx || m < 1 || m > kMaxM || k < 0 || k > m || n < 0 || n >= (int64_t(1) << 31) ||
      uint64_t(n) * uint64_t(k) >= (uint64_t(1) << 32) || (n > 0 && k > 0 && !ranks_host))
    return SCHULZE_EINVAL;
  if (int rc = set_device(ctx)) return rc;
  size_t rbytes = size_t(n) * size_t(k) * sizeof(int32_t);
  size_t mm = size_t(m) * size_t(m) * sizeof(int32_t);
  // (the extraction's scratch after the closure's: they run side by side)
  size_t stage = align_up(std::max(tally_workspace_bytes(n, m, k, flags), closure_workspace_bytes(m, n, flags)), 256) +
                 extract_workspace_bytes(m);
  size_t head = align_up(rbytes, 256) + 2 * align_up(mm, 256) + 3 * align_up(size_t(m) * 4, 256) +
                align_up(hint_words(m) * 4, 256) + 512;
  if (int rc = ensure_workspace(ctx, head + stage + 4096, stream)) return rc;
  Carver cv(ctx->ws.base);
  int32_t* ranks = cv.take<int32_t>(size_t(n) * size_t(k));
  int32_t* d = cv.take<int32_t>(size_t(m) * size_t(m));
  int32_t* p = cv.take<int32_t>(size_t(m) * size_t(m));
  int32_t* win = cv.take<int32_t>(size_t(m));
  int32_t* ord = cv.take<int32_t>(size_t(m));
  int32_t* bb = cv.take<int32_t>(size_t(m));
  int32_t* hint = cv.take<int32_t>(hint_words(m));
  int32_t* hint_valid = cv.take<int32_t>(1);
  void* rest = cv.take<char>(0);
  void* xrest = static_cast<char*>(rest) +
                align_up(std::max(tally_workspace_bytes(n, m, k, flags), closure_workspace_bytes(m, n, flags)), 256);
  // the call's work on stream s, the status word copied to *st
  auto enqueue = [&](cudaStream_t s, int32_t* st) -> int {
    if (rbytes && cudaMemcpyAsync(ranks, ranks_host, rbytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return SCHULZE_ECUDA;
    if (int rc = tally_launch(ctx, ranks, n, m, k, d, flags, rest, s, hint, hint_valid)) return rc;
    const bool ext = winners_host || order_host;
    int rc = closure_launch(ctx, d, m, n, p, flags, rest, s, ext ? bb : nullptr, hint, hint_valid, true);
    if (!rc && ext) rc = extract_from_beaten_by(ctx, bb, m, win, ord, xrest, s);
    const int rj = side_join(ctx, s);
    if (rc || rj) return rc ? rc : rj;
    if (winners_host && cudaMemcpyAsync(winners_host, win, size_t(m) * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return SCHULZE_ECUDA;
    if (order_host && cudaMemcpyAsync(order_host, ord, size_t(m) * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return SCHULZE_ECUDA;
    if (cudaMemcpyAsync(st, ctx->status, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return SCHULZE_ECUDA;
    return SCHULZE_OK;
  };
  int32_t st = 0;
  if (host_graph(ctx, {ranks_host, winners_host, order_host, ctx->ws.base, n, m, k, flags}, enqueue)) {
    if (cudaGraphLaunch(ctx->host_exec, stream) != cudaSuccess || cudaStreamSynchronize(stream) != cudaSuccess)
      return SCHULZE_ECUDA;
    st = *ctx->host_status;
  } else {
    if (int rc = enqueue(stream, &st)) return rc;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return SCHULZE_ECUDA;
  }
  if (st != 0) {
    cudaMemsetAsync(ctx->status, 0, sizeof(int32_t), stream);
    cudaStreamSynchronize(stream);
    return st;
  }
  return SCHULZE_OK;
}

}  // extern "C"
