// Launch accounting, optional per-kernel event timing, the zeroing kernel
// of the path's scratch, and the integer min/max issue-rate probe
// (include/schulze_profile.h).
#include <string.h>

#include <algorithm>

#include "count.cuh"
#include "internal.cuh"

namespace schulze {

static int class_index(schulze_ctx* ctx, const char* name) {
  for (size_t i = 0; i < ctx->prof_classes.size(); ++i)
    if (ctx->prof_classes[i].name == name) return int(i);
  ProfClass c;
  c.name = name;
  ctx->prof_classes.push_back(c);
  return int(ctx->prof_classes.size()) - 1;
}

static cudaEvent_t get_event(schulze_ctx* ctx) {
  if (!ctx->prof_free_events.empty()) {
    cudaEvent_t e = ctx->prof_free_events.back();
    ctx->prof_free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

Launch::Launch(schulze_ctx* ctx, cudaStream_t stream, const char* name, double work) : ctx_(ctx), stream_(stream) {
  if (!ctx) return;  // callers without a context (no counting, no profiling)
  ctx->launches += 1;
  if (!ctx->profiling) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return;
  }
  ProfRecord r;
  r.cls = class_index(ctx, name);
  r.start = get_event(ctx);
  r.stop = get_event(ctx);
  r.work = work;
  if (!r.start || !r.stop) return;
  cudaEventRecord(r.start, stream);
  ctx->prof_pending.push_back(r);
  rec_ = int(ctx->prof_pending.size()) - 1;
}

Launch::~Launch() {
  if (rec_ >= 0) cudaEventRecord(ctx_->prof_pending[rec_].stop, stream_);
}

static void drain(schulze_ctx* ctx) {
  for (ProfRecord& r : ctx->prof_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.start, r.stop) == cudaSuccess) {
      ProfClass& c = ctx->prof_classes[r.cls];
      c.launches += 1;
      c.ms += ms;
      c.work += r.work;
    } else {
      cudaGetLastError();
    }
    ctx->prof_free_events.push_back(r.start);
    ctx->prof_free_events.push_back(r.stop);
  }
  ctx->prof_pending.clear();
}

// ----------------------------------------------------------- zeroing

namespace {
__global__ void __launch_bounds__(256) zero_kernel(ZeroSpans z) {
  pdl_enter();
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
#pragma unroll
  for (int s = 0; s < 4; ++s)
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < z.words[s]; i += stride) z.p[s][i] = 0u;
}
}  // namespace

int zero_async(schulze_ctx* ctx, const ZeroSpans& z, cudaStream_t stream) {
  int64_t most = 0;
  for (int s = 0; s < 4; ++s)
    if (z.p[s]) most = std::max(most, z.words[s]);
  if (most == 0) return SCHULZE_OK;
  const int sms = ctx && ctx->sm_count > 0 ? ctx->sm_count : 148;
  const int grid = int(std::max<int64_t>(1, std::min<int64_t>((most + 255) / 256, int64_t(sms) * 4)));
  ZeroSpans zz = z;
  for (int s = 0; s < 4; ++s)
    if (!zz.p[s]) zz.words[s] = 0;
  Launch L(ctx, stream, "zero", double(most) * 4.0);
  if (launch_pdl(zero_kernel, dim3(grid), dim3(256), 0, stream, false, zz) != cudaSuccess) {
    cudaGetLastError();
    return SCHULZE_ECUDA;
  }
  return SCHULZE_OK;
}

// ----------------------------------------------------------- probe

template <int KIND>
__global__ void __launch_bounds__(256) minmax_probe_kernel(int iters, uint32_t seed, uint32_t* sink) {
  constexpr int C = 16;
  uint32_t c[C], a[C];
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
  for (int q = 0; q < C; ++q) {
    c[q] = (t * 2654435761u + q * 40503u + seed) & 0x3FFF3FFFu;
    a[q] = (t * 97u + q * 7919u + seed * 3u) & 0x3FFF3FFFu;
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < C; ++q) {
      // a[] stays fixed; the other operand is another chain's running value,
      // so nothing can be hoisted out of the loop
      const uint32_t b = c[(q + 5) % C];
      if (KIND == 0) {
        c[q] = uint32_t(max(int32_t(c[q]), min(int32_t(a[q]), int32_t(b))));
      } else if (KIND == 1) {
        c[q] = __vmaxs2(c[q], __vmins2(a[q], b));
      } else if (KIND == 2) {
        c[q] = __vimax3_s16x2(c[q], __vmins2(a[q], b), __vmins2(a[(q + 1) % C], c[(q + 9) % C]));
      } else {
        c[q] = uint32_t(__vimax3_s32(int32_t(c[q]), min(int32_t(a[q]), int32_t(b)),
                                     min(int32_t(a[(q + 1) % C]), int32_t(c[(q + 9) % C]))));
      }
    }
  }
  uint32_t s = 0;
#pragma unroll
  for (int q = 0; q < C; ++q) s ^= c[q];
  if (s == 0x12345678u) sink[0] = s;
}

// Float lanes: KIND 4 fp32 max(c, min(a, b)); KIND 5 fp32 three-input max
// folding two updates; KIND 6 half the chains int32 three-input max, half
// fp32 three-input max (do the two pipes add up?).
template <int KIND>
__global__ void __launch_bounds__(256) minmax_probe_f32_kernel(int iters, uint32_t seed, uint32_t* sink) {
  constexpr int C = 16;
  float c[C], a[C];
  int32_t ci[C], ai[C];
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
  for (int q = 0; q < C; ++q) {
    ci[q] = int32_t((t * 2654435761u + q * 40503u + seed) & 0xFFFFFu);
    ai[q] = int32_t((t * 97u + q * 7919u + seed * 3u) & 0xFFFFFu);
    c[q] = float(ci[q]);
    a[q] = float(ai[q]);
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < C; ++q) {
      if (KIND == 4) {
        c[q] = fmaxf(c[q], fminf(a[q], c[(q + 5) % C]));
      } else if (KIND == 5) {
        c[q] = max3f(c[q], fminf(a[q], c[(q + 5) % C]), fminf(a[(q + 1) % C], c[(q + 9) % C]));
      } else if (q & 1) {  // KIND 6: odd chains read odd chains only (all updated every step)
        c[q] = max3f(c[q], fminf(a[q], c[(q + 2) % C]), fminf(a[(q + 4) % C], c[(q + 6) % C]));
      } else {  // even chains read even chains only
        ci[q] = __vimax3_s32(ci[q], min(ai[q], ci[(q + 2) % C]), min(ai[(q + 4) % C], ci[(q + 6) % C]));
      }
    }
  }
  uint32_t s = 0;
#pragma unroll
  for (int q = 0; q < C; ++q) s ^= __float_as_uint(c[q]) ^ uint32_t(ci[q]);
  if (s == 0x12345678u) sink[0] = s;
}

// Probes on non-negative int32 bit patterns, the integer and the fp32
// min/max units sharing one set of values (see fmin_bits). KIND 7: the two
// mins on the fp32 unit, the three-input max on the integer unit; KIND 8:
// the reverse; KIND 9: a third of the chains all-integer, the rest
// all-fp32; KIND 10: two thirds all-integer; KIND 11: half and half (as
// KIND 6, on the bit patterns the closure would use).
template <int KIND>
__global__ void __launch_bounds__(256) minmax_probe_bits_kernel(int iters, uint32_t seed, uint32_t* sink) {
  constexpr int C = 18;  // a multiple of 2 and 3
  uint32_t c[C], a[C];
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
  for (int q = 0; q < C; ++q) {
    c[q] = (t * 2654435761u + q * 40503u + seed) & 0xFFFFFu;
    a[q] = (t * 97u + q * 7919u + seed * 3u) & 0xFFFFFu;
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < C; ++q) {
      // chains of one kind read chains of the same kind (KIND 9-11), all
      // updated every step; q + 6, q + 12 keep the residue mod 2 and 3
      const uint32_t b1 = c[(q + 6) % C], b2 = c[(q + 12) % C], a2 = a[(q + 6) % C];
      bool intchain = false;
      if (KIND == 9) intchain = (q % 3) == 0;
      if (KIND == 10) intchain = (q % 3) != 0;
      if (KIND == 11) intchain = (q & 1) == 0;
      if (KIND == 7) {
        c[q] = imax3_bits(c[q], fmin_bits(a[q], b1), fmin_bits(a2, b2));
      } else if (KIND == 8) {
        c[q] = fmax3_bits(c[q], imin_bits(a[q], b1), imin_bits(a2, b2));
      } else if (intchain) {
        c[q] = imax3_bits(c[q], imin_bits(a[q], b1), imin_bits(a2, b2));
      } else {
        c[q] = fmax3_bits(c[q], fmin_bits(a[q], b1), fmin_bits(a2, b2));
      }
    }
  }
  uint32_t s = 0;
#pragma unroll
  for (int q = 0; q < C; ++q) s ^= c[q];
  if (s == 0x12345678u) sink[0] = s;
}

// KIND 12: the tally's guard-bit compare-and-count on two 16-bit lanes
// (count_lt2): per chain step, two position compares.
__global__ void __launch_bounds__(256) compare_probe_kernel(int iters, uint32_t seed, uint32_t* sink) {
  constexpr int C = 16;
  uint32_t acc[C], a[C];
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
  for (int q = 0; q < C; ++q) {
    acc[q] = (t * 2654435761u + q * 40503u + seed) & 0x3FFF3FFFu;
    a[q] = ((t * 97u + q * 7919u + seed * 3u) & 0x3FFF3FFFu) | kGuard2;
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < C; ++q) acc[q] = count_lt2(acc[q], a[q], acc[(q + 5) % C] & 0x3FFF3FFFu);
  }
  uint32_t s = 0;
#pragma unroll
  for (int q = 0; q < C; ++q) s ^= acc[q];
  if (s == 0x12345678u) sink[0] = s;
}

}  // namespace schulze

using namespace schulze;

extern "C" {

int schulze_profile_enable(schulze_ctx* ctx, int enable) {
  if (!ctx) return SCHULZE_EINVAL;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return SCHULZE_ECUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return SCHULZE_ECUDA;
  drain(ctx);
  ctx->prof_classes.clear();
  ctx->profiling = enable != 0;
  return SCHULZE_OK;
}

int schulze_profile_read(schulze_ctx* ctx, schulze_kernel_stats* out, int max, int* count) {
  if (!ctx || !count || (max > 0 && !out)) return SCHULZE_EINVAL;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return SCHULZE_ECUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return SCHULZE_ECUDA;
  drain(ctx);
  int n = int(ctx->prof_classes.size());
  for (int i = 0; i < n && i < max; ++i) {
    const ProfClass& c = ctx->prof_classes[i];
    memset(out[i].name, 0, sizeof(out[i].name));
    strncpy(out[i].name, c.name.c_str(), sizeof(out[i].name) - 1);
    out[i].launches = c.launches;
    out[i].ms = c.ms;
    out[i].work = c.work;
  }
  *count = n;
  return SCHULZE_OK;
}

int64_t schulze_launch_count(const schulze_ctx* ctx) { return ctx ? ctx->launches : -1; }

int schulze_closure_counters(schulze_ctx* ctx, int64_t* tile_updates, int64_t* diag_closures, int64_t* items) {
  if (!ctx || !tile_updates || !diag_closures || !items) return SCHULZE_EINVAL;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return SCHULZE_ECUDA;
  unsigned long long h[3] = {0, 0, 0};
  if (cudaDeviceSynchronize() != cudaSuccess ||
      cudaMemcpy(h, ctx->counters, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess)
    return SCHULZE_ECUDA;
  *tile_updates = int64_t(h[0]);
  *diag_closures = int64_t(h[1]);
  *items = int64_t(h[2]);
  return SCHULZE_OK;
}

int schulze_probe_minmax(int device, int kind, int blocks, int iters, double* seconds, double* updates) {
  if (kind < 0 || kind > 12 || blocks < 1 || iters < 1 || !seconds || !updates) return SCHULZE_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return SCHULZE_ECUDA;
  uint32_t* sink = nullptr;
  if (cudaMalloc(&sink, 4) != cudaSuccess) return SCHULZE_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto launch = [&](int it) {
    if (kind == 0) minmax_probe_kernel<0><<<blocks, 256>>>(it, 1u, sink);
    else if (kind == 1) minmax_probe_kernel<1><<<blocks, 256>>>(it, 1u, sink);
    else if (kind == 2) minmax_probe_kernel<2><<<blocks, 256>>>(it, 1u, sink);
    else if (kind == 3) minmax_probe_kernel<3><<<blocks, 256>>>(it, 1u, sink);
    else if (kind == 4) minmax_probe_f32_kernel<4><<<blocks, 256>>>(it, 1u, sink);
    else if (kind == 5) minmax_probe_f32_kernel<5><<<blocks, 256>>>(it, 1u, sink);
    else if (kind == 6) minmax_probe_f32_kernel<6><<<blocks, 256>>>(it, 1u, sink);
    else if (kind == 7) minmax_probe_bits_kernel<7><<<blocks, 256>>>(it, 1u, sink);
    else if (kind == 8) minmax_probe_bits_kernel<8><<<blocks, 256>>>(it, 1u, sink);
    else if (kind == 9) minmax_probe_bits_kernel<9><<<blocks, 256>>>(it, 1u, sink);
    else if (kind == 10) minmax_probe_bits_kernel<10><<<blocks, 256>>>(it, 1u, sink);
    else if (kind == 11) minmax_probe_bits_kernel<11><<<blocks, 256>>>(it, 1u, sink);
    else compare_probe_kernel<<<blocks, 256>>>(it, 1u, sink);
  };
  launch(16);  // warm-up
  cudaEventRecord(e0);
  launch(iters);
  cudaEventRecord(e1);
  int rc = SCHULZE_OK;
  if (cudaEventSynchronize(e1) != cudaSuccess) rc = SCHULZE_ECUDA;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  *seconds = double(ms) * 1e-3;
  // (max, min) updates per chain step: one, or two when a three-input max
  // folds two steps, times the lanes per word
  static const double per_step[13] = {1.0, 2.0, 4.0, 2.0, 1.0, 2.0, 2.0, 2.0, 2.0, 2.0, 2.0, 2.0, 2.0};
  const double lanes = per_step[kind];
  const double chains = (kind >= 7 && kind <= 11) ? 18.0 : 16.0;
  *updates = double(blocks) * 256.0 * double(iters) * chains * lanes;
  return rc;
}

}  // extern "C"
