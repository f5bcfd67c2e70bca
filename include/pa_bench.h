/* pa_bench.h — integer-throughput probes of libpa.so (measurement support).
 *
 * These probes have no counterpart in the paper: they measure the integer
 * issue rates that bound the Metropolis sweep (a Philox4x32-10 word per site
 * update plus a few bitwise operations), so that the sweep kernel's speed can
 * be stated as a fraction of what this GPU can issue.
 *
 * pa_bench_int_throughput(kind, ...) launches `blocks` x `threads` threads, each
 * running `iters` iterations of 8 independent dependency chains of one operation:
 *   PA_BENCH_LOP3      lop3.b32 (3-input XOR)                  1 op per chain step
 *   PA_BENCH_IADD      add.u32                                  1 op
 *   PA_BENCH_IMAD      mad.lo.u32                               1 op
 *   PA_BENCH_MULWIDE   mul.wide.u32 + lop3 (fold hi into lo)    2 ops
 *   PA_BENCH_PHILOX    one Philox4x32-10 block (4 words)        counted as 4 words
 *   PA_BENCH_MULWIDE_ADD  mul.wide.u32 + add.u32 (hi + lo)      2 ops
 *   PA_BENCH_LOP3_IADD    lop3.b32 + add.u32                    2 ops
 *   PA_BENCH_PHILOX_LOP3  one Philox4x32-10 block + 16 independent lop3.b32 on
 *                         other registers                      counted as 4 words
 *                         (against PA_BENCH_PHILOX: whether logic work overlaps
 *                         the multiplies or adds its own time)
 * The pairs tell how the issue of a wide multiply (or a 3-input logic op) and a
 * full-rate add share one scheduler: with no sharing a pair costs the slower of
 * the two, with full sharing the sum.
 * On return *ms is the device time (CUDA events, after one warm-up launch) and
 * *ops the number of operations (words for PA_BENCH_PHILOX) executed.  Runs on
 * the current device, legacy default stream; allocates and frees a small
 * output buffer.  Returns 0 or a negative pa.h status. */
#ifndef PA_BENCH_H
#define PA_BENCH_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PA_BENCH_LOP3 0
#define PA_BENCH_IADD 1
#define PA_BENCH_IMAD 2
#define PA_BENCH_MULWIDE 3
#define PA_BENCH_PHILOX 4
#define PA_BENCH_MULWIDE_ADD 5
#define PA_BENCH_LOP3_IADD 6
#define PA_BENCH_PHILOX_LOP3 7

int pa_bench_int_throughput(int kind, int64_t iters, int blocks, int threads, double* ms, double* ops);

#ifdef __cplusplus
}
#endif
#endif
