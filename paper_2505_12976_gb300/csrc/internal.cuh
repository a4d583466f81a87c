// Internal declarations shared by the CUDA translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/schulze.h"
#include "../../include/schulze_profile.h"

namespace schulze {

constexpr int kMaxM = 65535;

// Non-negative int32 values read as fp32 bit patterns keep their order
// (sign bit clear; below 2^23 they are subnormals, which min and max without
// flush-to-zero compare exactly), so a (max, min) update on such values may
// run on the floating-point min/max unit instead of the integer one. Bit
// patterns at or above 0x7F800000 would be infinities or NaNs: callers use
// these only when every value is below that.
__device__ __forceinline__ float max3f(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
__device__ __forceinline__ uint32_t fmin_bits(uint32_t a, uint32_t b) {
  return __float_as_uint(fminf(__uint_as_float(a), __uint_as_float(b)));
}
__device__ __forceinline__ uint32_t fmax3_bits(uint32_t a, uint32_t b, uint32_t c) {
  return __float_as_uint(max3f(__uint_as_float(a), __uint_as_float(b), __uint_as_float(c)));
}
__device__ __forceinline__ uint32_t imax3_bits(uint32_t a, uint32_t b, uint32_t c) {
  return uint32_t(__vimax3_s32(int32_t(a), int32_t(b), int32_t(c)));
}
__device__ __forceinline__ uint32_t imin_bits(uint32_t a, uint32_t b) { return uint32_t(min(int32_t(a), int32_t(b))); }

// Names one C-ABI call as a range on the host timeline of profilers that
// read NVTX annotations (header-only NVTX: a no-op when no tool is attached).
struct AbiRange {
  explicit AbiRange(const char* name) { nvtxRangePushA(name); }
  ~AbiRange() { nvtxRangePop(); }
  AbiRange(const AbiRange&) = delete;
  AbiRange& operator=(const AbiRange&) = delete;
};

// Device status word helpers: the first error recorded wins.
__device__ __forceinline__ void set_status(int32_t* status, int32_t code) {
  if (status) atomicCAS(status, 0, code);
}

struct Workspace {
  void* base = nullptr;
  size_t bytes = 0;
};

}  // namespace schulze

namespace schulze {
// One profiled launch: event pair plus the class it belongs to.
struct ProfRecord {
  int cls;
  cudaEvent_t start, stop;
  double work;
};
struct ProfClass {
  std::string name;
  int64_t launches = 0;
  double ms = 0.0, work = 0.0;
};
}  // namespace schulze

struct schulze_ctx {
  int device = 0;
  int32_t* status = nullptr;                // device word
  unsigned long long* counters = nullptr;   // device: closure tile updates, diagonal closures, items
  schulze::Workspace ws;
  int sm_count = 0;
  size_t smem_optin = 0;
  int64_t launches = 0;
  bool profiling = false;
  // bound on each device-side wait of the persistent closure, in SM clock
  // cycles (schulze_set_wait_limit)
  long long wait_limit_cycles = 4000000000LL;
  std::vector<schulze::ProfRecord> prof_pending;
  std::vector<schulze::ProfClass> prof_classes;
  std::vector<cudaEvent_t> prof_free_events;
  // schulze_run_host: the whole call (copies in, path, copies out) captured
  // once as a CUDA graph on cap_stream and replayed while the arguments,
  // the workspace and the host buffers (page-locked) stay the same
  cudaStream_t cap_stream = nullptr;
  // schulze_run / schulze_run_host: the closure writes p on side_stream
  // (forked from the call's stream with side_fork) while the winners and
  // the ranking are extracted; side_join is recorded after it and the
  // call's stream waits on it before the call returns (side_pending)
  cudaStream_t side_stream = nullptr;
  cudaEvent_t side_fork = nullptr, side_join = nullptr;
  bool side_pending = false;
  cudaGraphExec_t host_exec = nullptr;
  int32_t* host_status = nullptr;  // page-locked word receiving the device status
  struct HostKey {
    const void* ranks = nullptr;
    const void* winners = nullptr;
    const void* order = nullptr;
    const void* ws = nullptr;
    int64_t n = -1;
    int32_t m = -1, k = -1;
    uint32_t flags = 0;
    bool operator==(const HostKey& o) const {
      return ranks == o.ranks && winners == o.winners && order == o.order && ws == o.ws && n == o.n && m == o.m &&
             k == o.k && flags == o.flags;
    }
  } host_key;
};

namespace schulze {

// Make sure ctx->ws holds at least `bytes`; may cudaMalloc unless the stream
// is capturing (then SCHULZE_ERANGE).
int ensure_workspace(schulze_ctx* ctx, size_t bytes, cudaStream_t stream);

constexpr inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Rows of an int32 [m, m] caller matrix at `ptr` may be moved with 16-byte
// accesses only when every row starts on a 16-byte boundary: m a multiple of
// 4 and the base itself aligned. Caller pointers need only 4-byte alignment
// (an int32 tensor with an odd storage offset, say), so kernels take this as
// an argument instead of deciding from m alone.
inline int rows_vec16(const void* ptr, int32_t m) {
  return ((m & 3) == 0 && (reinterpret_cast<uintptr_t>(ptr) & 15u) == 0) ? 1 : 0;
}

// Carves aligned sub-buffers out of the workspace.
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base(static_cast<char*>(b)) {}
  template <class T>
  T* take(size_t count) {
    off = align_up(off, 256);
    T* p = reinterpret_cast<T*>(base + off);
    off += count * sizeof(T);
    return p;
  }
};

// Workspace sizes (bytes) of each stage, for ensure_workspace and reserve.
size_t tally_workspace_bytes(int64_t n, int32_t m, int32_t k, uint32_t flags);
size_t closure_workspace_bytes(int32_t m, int64_t bound, uint32_t flags);
size_t extract_workspace_bytes(int32_t m);

size_t tally_positions_workspace_bytes(int64_t n, int32_t m);

// Stage launchers operating on caller-provided workspace (no allocation).
// With hint / hint_valid (hint_words(m) int32 words and one word, outside
// ws), a top-k tally also reports which candidates have an outgoing edge:
// when some candidate is listed on no ballot, exactly the listed ones do
// (each beats every unlisted one, and an unlisted one prefers nobody).
// *hint_valid is set to 1 when hint holds them, else 0. Layout of hint:
// flags [m], then the closure's warm-first relabeling of those flags, perm
// [m] (new -> old), inv [m] (old -> new) and the warm count [1], which the
// tally's plan pass writes so that the closure need not scan the flags.
inline size_t hint_words(int32_t m) { return 3 * size_t(m) + 1; }
int tally_launch(schulze_ctx* ctx, const int32_t* ranks, int64_t n, int32_t m, int32_t k, int32_t* d,
                 uint32_t flags, void* ws, cudaStream_t stream, int32_t* hint = nullptr,
                 int32_t* hint_valid = nullptr);
// Tally of weak-order ballots given as int32 positions [n, m].
int tally_positions_launch(schulze_ctx* ctx, const int32_t* pos, int64_t n, int32_t m, int32_t* d, void* ws,
                           cudaStream_t stream);

// With beaten_by non-null the closure also fills it (int32 [m]) from its
// warm rows, so extract_from_beaten_by can finish without reading p. With
// hint / hint_valid (from tally_launch, outside ws) the closure takes the
// warm flags and their relabeling from the tally when *hint_valid is set,
// skipping its own pass over d (and that pass's bound check, which the
// tally's d meets); otherwise it writes its relabeling into hint's perm,
// inv and warm words. With side (and beaten_by) p is written on the
// context's side stream while beaten_by is extracted on stream; the caller
// ends with side_join(ctx, stream) before it returns (and before anything
// on stream reuses the closure's scratch).
int closure_launch(schulze_ctx* ctx, const int32_t* d, int32_t m, int64_t bound, int32_t* p, uint32_t flags,
                   void* ws, cudaStream_t stream, int32_t* beaten_by = nullptr, int32_t* hint = nullptr,
                   const int32_t* hint_valid = nullptr, bool side = false);
// stream waits for the side stream's work if closure_launch forked any
int side_join(schulze_ctx* ctx, cudaStream_t stream);
int extract_launch(schulze_ctx* ctx, const int32_t* p, int32_t m, int32_t* winners, int32_t* order,
                   int32_t* beaten_by, void* ws, cudaStream_t stream);
// Winners by the paper's vertex-centric algorithm on the dense tally;
// stats (host, may be null): [0] while-loop iterations, [1] rounds.
size_t propagation_workspace_bytes(int32_t m);
int winners_propagation_launch(schulze_ctx* ctx, const int32_t* d, int32_t m, bool margin, int32_t* winners,
                               int32_t* stats, void* ws, cudaStream_t stream);
// One level of the iterated-removal ranking: candidates with level 0 and
// beaten_by 0 get level t (listed in placed[1..], counted in placed[0]) and
// are isolated in the working tally dw.
int iterated_level(schulze_ctx* ctx, const int32_t* bb, int32_t m, int32_t t, int32_t* level, int32_t* placed,
                   int32_t* dw, cudaStream_t stream);
// Winners (beaten_by == 0) and the ranking from a filled beaten_by.
int extract_from_beaten_by(schulze_ctx* ctx, const int32_t* beaten_by, int32_t m, int32_t* winners, int32_t* order,
                           void* ws, cudaStream_t stream);

// Brackets one kernel launch: counts it and, when profiling is on, records
// CUDA events around it on `stream`, filed under `name` with `work` units.
class Launch {
 public:
  Launch(schulze_ctx* ctx, cudaStream_t stream, const char* name, double work);
  ~Launch();

 private:
  schulze_ctx* ctx_;
  cudaStream_t stream_;
  int rec_ = -1;
};

// Programmatic dependent launch. A kernel launched with launch_pdl may start
// while its predecessor on the stream is still running: pdl_enter(), the
// first statement of such a kernel, waits until the predecessor has finished
// and its writes are visible, then lets the successor start launching.
// Without a programmatic dependency (a plain launch) both are no-ops.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
// The same for kernels that usually return at once (the alternatives the
// device decides against): the successor may start launching before the
// wait, so a returning kernel adds little to the chain. The successor still
// waits for this kernel's completion, which follows the predecessor's.
__device__ __forceinline__ void pdl_enter_early() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                              bool cooperative, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  attr[1].id = cudaLaunchAttributeCooperative;
  attr[1].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = cooperative ? 2 : 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Zeroes up to four spans of 32-bit words in one kernel launched with
// launch_pdl (where a memset would end the programmatic chain); spans with a
// null pointer or no words are skipped.
struct ZeroSpans {
  uint32_t* p[4] = {nullptr, nullptr, nullptr, nullptr};
  int64_t words[4] = {0, 0, 0, 0};
};
int zero_async(schulze_ctx* ctx, const ZeroSpans& z, cudaStream_t stream);

inline int check_launch() {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SCHULZE_OK : SCHULZE_ECUDA;
}

bool use_s16(int64_t bound, uint32_t flags);

}  // namespace schulze
