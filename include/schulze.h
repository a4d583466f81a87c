/*
 * schulze.h -- C ABI of the GB300 (sm_103a) Schulze hot path.
 *
 * The Schulze method (Csar, Lackner, Pichler, "Computing the Schulze Method
 * for Large-Scale Preference Data Sets", arXiv 2505.12976, Sect. 2.1) ranks
 * candidates by widest paths in the weighted majority graph. The calls below
 * cover its data-parallel path: the pairwise tally, the all-pairs widest-path
 * closure in the (max, min) semiring (the classical Floyd-Warshall route of
 * Sect. 1 and Sect. 4), and winner and ranking extraction.
 *
 * Conventions shared by every call
 *  - All array arguments are DEVICE pointers (cudaMalloc / torch CUDA memory)
 *    owned by the caller, unless a call says "host". The library never frees
 *    them and keeps no reference after the call returns.
 *  - Matrices are dense, row-major, leading dimension m, int32. Device
 *    pointers need only the 4-byte alignment of int32; rows that start on
 *    16-byte boundaries (m a multiple of 4 and a 16-byte aligned base) are
 *    moved with 16-byte accesses, others element by element.
 *  - Calls are asynchronous and ordered on `stream` (a cudaStream_t; NULL is
 *    the legacy default stream). Outputs are valid once the stream reaches
 *    the end of the call's work.
 *  - Return value: SCHULZE_OK or a negative code detected on the host
 *    (bad argument, launch failure, allocation failure). Problems found by
 *    the kernels in the data itself (an out-of-range or repeated id in a
 *    ballot, a negative count) are recorded in the context's device status
 *    word and read back by schulze_get_status(); outputs are then unspecified.
 *  - A context owns its workspace and status word. Calls that share a
 *    context must be ordered on one stream (they reuse the workspace);
 *    create one context per concurrent stream.
 *  - A call grows the workspace with cudaMalloc when it is too small. During
 *    CUDA stream capture it does not allocate and returns SCHULZE_ERANGE
 *    instead; call schulze_reserve() with the largest sizes first.
 */
#ifndef SCHULZE_H
#define SCHULZE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* schulze_stream_t; /* same type as cudaStream_t */
typedef struct schulze_ctx schulze_ctx;

enum schulze_status {
  SCHULZE_OK = 0,
  SCHULZE_EINVAL = -1,   /* null pointer, size out of range, bad flag combination */
  SCHULZE_ENOMEM = -2,   /* workspace allocation failed */
  SCHULZE_ECUDA = -3,    /* a CUDA runtime call or kernel launch failed */
  SCHULZE_EDATA = -4,    /* (device status) bad ballot id, repeated id, negative or too large count */
  SCHULZE_ETIMEOUT = -5, /* (device status) a bounded device wait gave up */
  SCHULZE_ERANGE = -6,   /* workspace too small while the stream is being captured */
  SCHULZE_ETOOBIG = -7   /* size beyond the fixed scratch of schulze_strongest_paths_static */
};

/* Closure flags (schulze_strongest_paths, schulze_run). */
#define SCHULZE_F_AUTO 0u         /* 16-bit packed closure when bound <= 32767, else int32 */
#define SCHULZE_F_FORCE_S32 1u    /* always the int32 closure */
#define SCHULZE_F_FORCE_S16 2u    /* always the 16-bit closure; EINVAL if bound > 32767 */
#define SCHULZE_F_MARGIN 32u      /* edge weights are the margins d[i][j] - d[j][i] > 0 (Sect. 2.1)
                                     instead of winning votes */
/* Tally flags (schulze_tally, schulze_run). */
#define SCHULZE_F_TALLY_DENSE 4u  /* position-compare tally, O(n m^2) */
#define SCHULZE_F_TALLY_SPARSE 8u /* pair-count tally, O(n k^2) */
#define SCHULZE_F_TALLY_GROUPED 16u /* pair-count tally without the listed-candidate compaction */

/* Human-readable text for a status code (static storage). */
const char* schulze_strerror(int code);

/* Create a context on `device` (made current for the call). *out receives it. */
int schulze_ctx_create(int device, schulze_ctx** out);

/* Free the workspace and the context. Waits for the device first. */
int schulze_ctx_destroy(schulze_ctx* ctx);

/* Size the workspace for elections up to m_max candidates and n_max ballots
 * of at most k_max entries, so that later calls (and stream capture) do not
 * allocate. Synchronous. */
int schulze_reserve(schulze_ctx* ctx, int32_t m_max, int64_t n_max, int32_t k_max);

/* Bytes of workspace currently held by the context. */
size_t schulze_workspace_bytes(const schulze_ctx* ctx);

/* Wait for `stream`, then copy the device status word to *status (host) and
 * reset it to SCHULZE_OK. */
int schulze_get_status(schulze_ctx* ctx, int32_t* status, schulze_stream_t stream);

/* Bound on each device-side wait of the closure's persistent kernel (a CTA
 * waiting for the tiles an item depends on), in SM clock cycles; default
 * 4e9, about 2 s at 2 GHz. A wait that runs out records SCHULZE_ETIMEOUT in
 * the status word and raises an abort flag that every CTA checks in its
 * waits and before its next item, so the launch always ends; that call's
 * outputs are then unspecified and the next call starts afresh. Applies to
 * calls issued after it (a graph captured earlier keeps the limit it was
 * captured with). cycles >= 1, else SCHULZE_EINVAL. */
int schulze_set_wait_limit(schulze_ctx* ctx, int64_t cycles);

/*
 * Pairwise tally (Sect. 2.1: the counts behind the majority margin
 * mu(a,b) = d[a][b] - d[b][a]).
 *   ranks  [n, k] int32 device, row v lists candidate ids best first; every
 *          id in [0, m) and distinct within its row; k == m is a full
 *          ranking, and with k < m the unlisted candidates are tied below
 *          all listed ones.
 *   d      [m, m] int32 device output: d[i][j] = #voters preferring i to j,
 *          d[i][i] = 0. Overwritten completely.
 *   flags  0 (choose by cost), SCHULZE_F_TALLY_DENSE or SCHULZE_F_TALLY_SPARSE;
 *          SCHULZE_F_TALLY_GROUPED keeps the pair-count tally on its grouped
 *          form even when few candidates are listed (same result).
 * Sizes: 1 <= m <= 65535, 0 <= k <= m, 0 <= n < 2^31, n*k < 2^32.
 * Bad ids are reported as SCHULZE_EDATA through schulze_get_status().
 */
int schulze_tally(schulze_ctx* ctx, const int32_t* ranks, int64_t n, int32_t m, int32_t k, int32_t* d,
                  uint32_t flags, schulze_stream_t stream);

/*
 * Pairwise tally of weak-order ballots (Sect. 2.1: a voter may rank
 * candidates equally), given in position form.
 *   pos    [n, m] int32 device, pos[v][c] = position of candidate c on ballot
 *          v: smaller is better, equal positions are tied (a tied pair counts
 *          for neither); every position in [0, 65534]. An unranked candidate
 *          is simply given a position behind the ranked ones.
 *   d      [m, m] int32 device output: d[i][j] = #{v : pos[v][i] < pos[v][j]},
 *          d[i][i] = 0. Overwritten completely. O(n m^2) position compares.
 * Sizes: 1 <= m <= 65535, 0 <= n < 2^31, n*m < 2^40. A position out of range
 * is reported as SCHULZE_EDATA through schulze_get_status() (d unspecified).
 */
int schulze_tally_positions(schulze_ctx* ctx, const int32_t* pos, int64_t n, int32_t m, int32_t* d,
                            schulze_stream_t stream);

/*
 * Widest paths (Sect. 2.1: p(a,b) = the largest width min over the edges of
 * a path from a to b; Sect. 4: all pairs by Floyd-Warshall). Edge weights
 * are winning votes: w[i][j] = d[i][j] if d[i][j] > d[j][i], else 0.
 *   d      [m, m] int32 device input (e.g. from schulze_tally); read only.
 *   bound  an upper bound on every entry of d (n for a tally of n ballots);
 *          it selects the 16-bit packed closure when <= 32767. A d entry
 *          above it, or below 0, is reported as SCHULZE_EDATA.
 *   p      [m, m] int32 device output: p[i][j] = widest-path width from i to
 *          j, 0 if j is unreachable, p[i][i] = 0. May not alias d.
 *   flags  SCHULZE_F_AUTO, SCHULZE_F_FORCE_S32 or SCHULZE_F_FORCE_S16, plus
 *          SCHULZE_F_MARGIN for the paper's margin weights
 *          w[i][j] = d[i][j] - d[j][i] when positive (same edges).
 */
int schulze_strongest_paths(schulze_ctx* ctx, const int32_t* d, int32_t m, int64_t bound, int32_t* p,
                            uint32_t flags, schulze_stream_t stream);

/*
 * Same result as schulze_strongest_paths, without any device allocation.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc -- code whose device memory is owned entirely by
 * another allocator (a framework's caching pool, an arena reserved at
 * start-up), or that runs under a rule forbidding allocation once set up
 * (latency-critical serving loops). It needs no context either.
 *   d, bound, p, flags  as for schulze_strongest_paths; 1 <= m <= 1024,
 *          larger m returns SCHULZE_ETOOBIG.
 *   status a device int32 where data errors found by the kernels are
 *          recorded (SCHULZE_EDATA, SCHULZE_ETIMEOUT; the first one wins; the
 *          caller zeroes it), or NULL to not record them. When status would
 *          hold an error, p is unspecified; with NULL such an error goes
 *          unnoticed (the call still returns SCHULZE_OK), so pass a status
 *          word unless d is known to be valid.
 * Scratch: one file-scope device array of about 4.1 MB (W for m <= 1024 in
 * int32, progress words, relabeling), present on every GPU that loads the
 * library until the process exits. The call runs on the calling thread's
 * current device; its first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) and caches it, so make that first call
 * before any stream capture. The cache assumes one primary context per
 * device for the life of the process: after cudaDeviceReset() the cached
 * address is stale, so do not call this entry point again in that process. The call resets the parts of the array that
 * must start at zero; all calls share the one array, so calls that overlap
 * on the GPU (other streams, other host threads) race and corrupt each
 * other's results: order them on one stream.
 */
int schulze_strongest_paths_static(const int32_t* d, int32_t m, int64_t bound, int32_t* p, uint32_t flags,
                                   int32_t* status, schulze_stream_t stream);

/*
 * Winners (Sect. 2.1): i is a winner iff no j beats it, i.e. p[i][j] >=
 * p[j][i] for all j.
 *   p        [m, m] int32 device input.
 *   winners  [m] int32 device output, 1 for a winner, 0 otherwise. At least
 *            one entry is 1 when p comes from schulze_strongest_paths.
 */
int schulze_winners(schulze_ctx* ctx, const int32_t* p, int32_t m, int32_t* winners, schulze_stream_t stream);

/*
 * Ranking (Sect. 2.1, the relation p(a,b) >= p(b,a)). With ties that
 * relation need not be transitive, so the output is the linear order of ids
 * sorted by (beaten_by, id), where beaten_by[i] = #{j : p[j][i] > p[i][j]};
 * it extends the strict relation "a beats b".
 *   order      [m] int32 device output: candidate ids, best first.
 *   beaten_by  [m] int32 device output, or NULL.
 */
int schulze_ranking(schulze_ctx* ctx, const int32_t* p, int32_t m, int32_t* order, int32_t* beaten_by,
                    schulze_stream_t stream);

/*
 * Top-k ranking by iterated winner removal (Sect. 4, closing remark: run the
 * method again after removing the Schulze winners). Level t is the winner
 * set of the profile restricted to the candidates not placed in levels
 * 1 .. t-1 (pairwise counts do not depend on the other candidates).
 *   d       [m, m] int32 device tally (read only); bound as for
 *           schulze_strongest_paths; flags may add SCHULZE_F_MARGIN.
 *   k_top   levels are assigned until at least min(k_top, m) candidates are
 *           placed (k_top >= 1).
 *   level   [m] int32 device output: the level (>= 1) of each placed
 *           candidate, 0 for the others.
 *   levels  host int32, may be NULL: number of levels assigned.
 * Synchronous on `stream` (one host round trip per level; not for capture).
 * Each level runs the closure on a working copy of d in which the placed
 * candidates are isolated.
 */
int schulze_ranking_iterated(schulze_ctx* ctx, const int32_t* d, int32_t m, int64_t bound, int32_t k_top,
                             int32_t* level, int32_t* levels, uint32_t flags, schulze_stream_t stream);

/*
 * Winners only, by the paper's vertex-centric algorithm (Sect. 4, Alg. 1-4:
 * initial loser filter, then while some candidate is undecided: forward and
 * backward propagation of the smallest source / target id with the widest
 * width, and the SCC rules of the postprocessing), restated on the dense
 * tally. The same winner set as schulze_winners on the closure; provided as
 * a comparator for the paper's own method.
 *   d        [m, m] int32 device tally (read only); flags: 0 or
 *            SCHULZE_F_MARGIN (edge weights as in schulze_strongest_paths).
 *   winners  [m] int32 device output, 1 for a winner.
 *   stats    host int32 [2], may be NULL: while-loop iterations, propagation
 *            rounds in total.
 * Synchronous on `stream` (host round trips per round; not for capture).
 */
int schulze_winners_propagation(schulze_ctx* ctx, const int32_t* d, int32_t m, uint32_t flags, int32_t* winners,
                                int32_t* stats, schulze_stream_t stream);

/*
 * The whole path for one election: tally, widest paths, winners and ranking
 * in one call (device buffers). d and p are written as by the calls above;
 * winners, order and beaten_by may each be NULL. `flags` combines the tally
 * and closure flags. The closure bound is n.
 */
int schulze_run(schulze_ctx* ctx, const int32_t* ranks, int64_t n, int32_t m, int32_t k, int32_t* d, int32_t* p,
                int32_t* winners, int32_t* order, int32_t* beaten_by, uint32_t flags, schulze_stream_t stream);

/*
 * Same as schulze_run with HOST buffers: copies ranks to the device, runs the
 * path on workspace memory and copies winners and order (each may be NULL)
 * back to the host. Synchronous on `stream`. Device d and p stay inside the
 * context. Returns SCHULZE_EDATA directly when the ballots are invalid.
 * When every host buffer is page-locked, the call's work (copies included)
 * is captured once as a CUDA graph and replayed by later calls with the same
 * buffers and sizes (the ballots are read afresh each call); pageable
 * buffers run the same work eagerly.
 */
int schulze_run_host(schulze_ctx* ctx, const int32_t* ranks_host, int64_t n, int32_t m, int32_t k,
                     int32_t* winners_host, int32_t* order_host, uint32_t flags, schulze_stream_t stream);

/*
 * Batched elections: E independent elections (each 1 <= m <= 1024) run in
 * one persistent launch, one election per CTA at a time, longest first.
 * Every election goes through the same path as schulze_run (Sect. 2.1:
 * tally, winning-votes weights, widest paths, winners, ranking).
 *
 * Layout: the elections are packed back to back in the caller's order.
 * Ballots of election e start at element ranks_off[e] = sum_{f<e} n_f k_f of
 * `ranks`; its d and p start at mat_off[e] = sum_{f<e} m_f^2 (row-major,
 * leading dimension m_e); its winners, order and beaten_by at vec_off[e] =
 * sum_{f<e} m_f. schulze_batch_layout reports these offsets and the totals.
 */
typedef struct schulze_batch schulze_batch;

/* Plan a batch from HOST arrays n[E], m[E], k[E]: computes the layout and the
 * job order, uploads the job table and reserves per-CTA scratch (allocates;
 * call before any stream capture). */
int schulze_batch_create(schulze_ctx* ctx, int32_t E, const int32_t* n, const int32_t* m, const int32_t* k,
                         schulze_batch** out);

/* Free the plan (waits for the device). */
int schulze_batch_destroy(schulze_batch* b);

/* Totals (elements) and per-election offsets (host arrays of E, or NULL). */
int schulze_batch_layout(const schulze_batch* b, int64_t* ranks_elems, int64_t* mat_elems, int64_t* vec_elems,
                         int64_t* ranks_off, int64_t* mat_off, int64_t* vec_off);

/* Run every election of the plan. ranks: device ballots in the plan's
 * layout. d, p, winners, order, beaten_by: device outputs in the plan's
 * layout, each may be NULL (not written). Allocates nothing, so a run can be
 * captured in a CUDA graph and replayed. Bad ballots are reported as
 * SCHULZE_EDATA in the context's status word. */
int schulze_batch_run(schulze_batch* b, const int32_t* ranks, int32_t* d, int32_t* p, int32_t* winners,
                      int32_t* order, int32_t* beaten_by, schulze_stream_t stream);

/* The batch from HOST buffers, end to end: ranks_host in the plan's layout
 * (page-locked memory gives the copies full speed; any host memory works),
 * winners_host / order_host (host int32 [vec_elems], either may be NULL)
 * receive the results. The caller's elections are cut into up to eight
 * segments of about equal ballot bytes; each segment's ballots are copied on
 * the plan's own copy stream while the previous segment is computed, and
 * each segment runs as one launch (its elections longest first, the plan's
 * schedule). The first call allocates the plan's device copy of the ballots
 * and its output buffers (ranks_elems + 2 vec_elems int32), kept until
 * schulze_batch_destroy. Synchronous: returns once the results are on the
 * host. Bad ballots are reported as SCHULZE_EDATA in the context's status
 * word. */
int schulze_batch_run_host(schulze_batch* b, const int32_t* ranks_host, int32_t* winners_host, int32_t* order_host,
                           schulze_stream_t stream);

/* Schedule knobs: tally_policy 0 stages each election's ballots in steps of
 * its m-bucket's size (schulze_batch_set_bucket_chunk, the autotuner), 1
 * stages eight everywhere; order_policy 0 runs the longest elections first,
 * 1 the caller's order. Synchronous. */
int schulze_batch_set_schedule(schulze_batch* b, int32_t tally_policy, int32_t order_policy);

/* Elections are grouped by m into five buckets (m <= 64, 128, 256, 512,
 * 1024); the tally of an election stages `chunk` ballots per step as position
 * rows in shared memory (8, 16, 32 or 64; a power of two that fits: chunk *
 * ceil64(m) * 6 bytes within the CTA's shared memory and chunk * m <= 8192),
 * set here per bucket (EINVAL for a size that does not fit the bucket's
 * largest m). Synchronous. */
int schulze_batch_set_bucket_chunk(schulze_batch* b, int32_t bucket, int32_t chunk);

/* The tally of an election covers d in 64 x 64 tiles, worked on by the four
 * 128-thread tile groups of a CTA; groups_per_tile (1, 2 or 4) groups share
 * one tile, each counting every groups_per_tile-th staged ballot (so an
 * election of one or two tiles still keeps all four busy), set here per
 * bucket (EINVAL otherwise). Synchronous. */
int schulze_batch_set_bucket_tiles(schulze_batch* b, int32_t bucket, int32_t groups_per_tile);

/* The per-bucket schedule: largest m of each bucket, its ballots per step
 * and the number of the plan's elections in it (host int32 [5] each, any may
 * be NULL). */
int schulze_batch_bucket_schedule(const schulze_batch* b, int32_t* bucket_max_m, int32_t* chunks,
                                  int32_t* elections);

/* Groups per tally tile of each bucket (host int32 [5], not NULL). */
int schulze_batch_bucket_tiles(const schulze_batch* b, int32_t* groups_per_tile);

/* Autotuner: for every m-bucket with elections, times the bucket's elections
 * alone (one launch over them, three runs, the best of the last two) with
 * every ballots-per-step size that fits times every number of groups per
 * tally tile (1, 2, 4) and keeps the fastest pair; then times both election
 * orders on the whole batch. best_tally receives 0 (the per-bucket
 * schedule), best_order the order policy. With cache_path, a result already
 * recorded for the same GPU and bucket (election count and mean ballot
 * count; value chunk * 8 + groups per tile) or batch signature is reused,
 * and new ones are appended, one "<key> <value>" line each. */
int schulze_batch_autotune(schulze_batch* b, const int32_t* ranks, const char* cache_path, int32_t* best_tally,
                           int32_t* best_order, schulze_stream_t stream);

/*
 * Learned winner proposal with exact certification. The paper has no learned
 * component: a small MLP (16 -> 64 -> 64 -> 1, ReLU, FP32) proposes likely
 * winners, and each proposal is certified with the definitions of Sect. 2.1
 * (c wins iff p(c, j) >= p(j, c) for every j) by single-source and
 * single-sink widest paths; the full closure decides when no proposal
 * certifies. The winner set never depends on the model.
 *
 * Parameters: 5313 floats, W1 [64][16] at 0, b1 [64] at 1024, W2 [64][64] at
 * 1088, b2 [64] at 5184, W3 [64] at 5248, b3 at 5312 (device memory).
 */

/* 16 FP32 features per candidate from d and the ballot count n (feat is
 * [m, 16] row-major, device): Copeland wins / losses / ties over m-1;
 * row and column sums of d over n(m-1); largest outgoing and incoming
 * winning-votes edge over n; the loser filter of Sect. 4 (1 if the largest
 * incoming edge is heavier); their difference; outgoing and incoming edge
 * sums; smallest and largest margin; largest d[c][j]; the ranks of the row
 * sum and of wins - losses among the candidates (0 = best, over m-1). d is
 * a tally of n ballots: its entries are counts in [0, n] (sums and ranks
 * are exact under that bound, not for arbitrary matrices). */
int schulze_features(schulze_ctx* ctx, const int32_t* d, int32_t m, int64_t n, float* feat, schulze_stream_t stream);

/* score[c] = MLP(feat[c]) for N candidates (device arrays). */
int schulze_mlp_forward(schulze_ctx* ctx, const float* params, const float* feat, int32_t N, float* score,
                        schulze_stream_t stream);

/* One training step on N candidates from nseg elections: election e owns
 * candidates seg_off[e] .. seg_off[e+1]-1 (device int32 [nseg+1]); label[c]
 * is 1 for a winner, else 0. Loss: listwise softmax cross-entropy with equal
 * target mass on an election's winners, averaged over elections. Then one
 * Adam step (beta1 0.9, beta2 0.999, eps 1e-8, 1-based `step`) updates params
 * and the moments adam_m, adam_v in place. loss (device float [1]) and grad
 * (device float [5313]) may be NULL. Gradients are summed in a fixed order
 * (deterministic). */
int schulze_mlp_train_step(schulze_ctx* ctx, float* params, float* adam_m, float* adam_v, int64_t step,
                           const float* feat, const int32_t* label, const int32_t* seg_off, int32_t nseg, int32_t N,
                           float lr, float* loss, float* grad, schulze_stream_t stream);

/* Certify proposals cand[0..ncand-1] (device int32, ncand <= 8) for the
 * election with tally d: winners (device int32 [m]) receives the exact
 * winner set when result[0] == 1 (device int32 [4]: [0] 1 if certified, 0 if
 * the closure must decide; [1] index of the certified proposal or -1; [2]
 * tied candidates checked; [3] widest-path relaxation rounds). Handles up to
 * 2048 candidates with outgoing edges; beyond that result[0] is 0. */
int schulze_certify(schulze_ctx* ctx, const int32_t* d, int32_t m, int64_t n, const int32_t* cand, int32_t ncand,
                    int32_t* winners, int32_t* result, schulze_stream_t stream);

/* Winners of the election with tally d: features, proposals (the MLP with
 * `params`, or the Copeland score wins - losses when params is NULL), the
 * `top` best (<= 8) certified in order. When none certifies, the full
 * closure decides; when the warm set is too large to certify (more than
 * 2048 candidates with outgoing edges), the paper's propagation algorithm
 * (Sect. 4, Alg. 1-4, as schulze_winners_propagation) decides instead.
 * Synchronous on `stream`. winners: device int32 [m]. stats (HOST int32 [4],
 * may be NULL): [0] index of the proposal that certified (-1 if none), [1] 0
 * if a proposal certified, 1 if the closure decided, 2 if the propagation
 * did, [2] ties checked, [3] relaxation rounds. */
int schulze_winners_fast(schulze_ctx* ctx, const int32_t* d, int32_t m, int64_t n, const float* params, int32_t top,
                         int32_t* winners, int32_t* stats, schulze_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* SCHULZE_H */
