/*
 * schulze_profile.h -- measurement hooks of the GB300 Schulze library.
 *
 * Not part of the method: these calls let a benchmark time the library's own
 * kernels on the stream they run on, count launches, and measure the integer
 * min/max issue rate the widest-path closure is bound by.
 */
#ifndef SCHULZE_PROFILE_H
#define SCHULZE_PROFILE_H

#include <stdint.h>

#include "schulze.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Per kernel class: launches, summed device time, summed algorithmic work
 * (the class's own unit: min/max updates for the closure, bytes for the
 * tally and extraction stages). */
typedef struct {
  char name[32];
  int64_t launches;
  double ms;
  double work;
} schulze_kernel_stats;

/* enable != 0: from now on every kernel launch of this context records a CUDA
 * event pair on its stream (cleared statistics); enable == 0: stop. */
int schulze_profile_enable(schulze_ctx* ctx, int enable);

/* Synchronizes the device, then writes up to `max` classes to out[] and
 * their number to *count. Statistics keep accumulating until re-enabled. */
int schulze_profile_read(schulze_ctx* ctx, schulze_kernel_stats* out, int max, int* count);

/* Kernel launches issued by this context since it was created. */
int64_t schulze_launch_count(const schulze_ctx* ctx);

/* Work the widest-path closure kernel actually executed on this context
 * since it was created (synchronizes the device): 64 x 64 x 64 tile updates
 * computed (skipped all-zero updates not counted), 64 x 64 diagonal-tile
 * closures computed, and work items taken from the queue. */
int schulze_closure_counters(schulze_ctx* ctx, int64_t* tile_updates, int64_t* diag_closures, int64_t* items);

/*
 * Integer min/max issue-rate probe: a grid of `blocks` x 256 threads runs
 * `iters` iterations of 16 independent (max, min) chains per thread in the
 * given lane format (kind 0: int32, 2 instructions per update; kind 1: packed
 * int16x2, 2 instructions per 2 updates; kind 2: packed int16x2 with a
 * three-input max folding two updates, 3 instructions per 4 updates; kind 3:
 * int32 with a three-input max, 3 instructions per 2 updates; kind 4: fp32
 * lanes; kind 5: fp32 with a three-input max; kind 6: half the chains as
 * kind 3, half as kind 5; kinds 7-11 work on non-negative int32 bit patterns
 * read as fp32 where a float unit is used, as a closure sharing one matrix
 * between the two units would: kind 7 fp32 mins with an int32 three-input
 * max, kind 8 int32 mins with an fp32 three-input max, kind 9 a third of the
 * chains as kind 3 and the rest in fp32, kind 10 two thirds as kind 3, kind
 * 11 half and half; kind 12 the tally's guard-bit compare-and-count of two
 * 16-bit position lanes, counting lane compares as updates). *seconds
 * receives the kernel time (CUDA events) and *updates the number of
 * (max, min) lane updates done.
 * Synchronous.
 */
int schulze_probe_minmax(int device, int kind, int blocks, int iters, double* seconds, double* updates);

#ifdef __cplusplus
}
#endif

#endif /* SCHULZE_PROFILE_H */
