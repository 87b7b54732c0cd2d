/*
 * Launch-shape and measurement entry points of the GB300 generator library
 * (companions of rng.h used by the autotuner and the benchmark).  The paper
 * tunes the block size (128/256/512 threads, occupancy-calculator choice in
 * the MWC and XorShift kernel sections) and measures the achievable memory
 * bandwidth with a separate benchmark (Sec. "Discussion"); these are the
 * GB300 counterparts.
 */
#ifndef GBRNG_RNG_TUNE_H
#define GBRNG_RNG_TUNE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Launch shape of the vector-store generate kernel for (kind, fmt):
 * v = groups of four streams per thread (1 or 2), block = threads per CTA
 * (power of two, 32..512), hint = 1 for streaming (evict-first) stores,
 * 0 for default stores, 2 for rows staged in shared memory and written by
 * TMA bulk copies (32-byte aligned rows only; v and block then unused:
 * CTAs of 256 threads, 1024 streams each).  Applies to later rng_generate calls in this process
 * on every device; does not change any output.  Returns 0 or RNG_ERR_ARG. */
int gbrng_set_launch(int kind, int fmt, int v, int block, int hint);
int gbrng_get_launch(int kind, int fmt, int *v, int *block, int *hint);

/* The same per size class: class 0 holds the shapes of calls of fewer than
 * 2^21 streams, class 1 those of the rest (the class gbrng_set_launch and
 * gbrng_get_launch address).  Returns 0 or RNG_ERR_ARG. */
int gbrng_set_launch_class(int kind, int fmt, int size_class, int v, int block, int hint);
int gbrng_get_launch_class(int kind, int fmt, int size_class, int *v, int *block, int *hint);

/* One CTA per SM (1) or as many as fit (0) for the aligned vector kernel of
 * (kind, fmt) in a size class (as gbrng_set_launch_class): with 1, a
 * shared-memory reservation keeps a second CTA off each SM whenever the
 * call runs CTAs of the shape's size.  gbrng_set_launch(_class) leave it
 * as it is.  Outputs never change.  Returns 0 or RNG_ERR_ARG. */
int gbrng_set_launch_ctas(int kind, int fmt, int size_class, int ctas_per_sm);
int gbrng_get_launch_ctas(int kind, int fmt, int size_class, int *ctas_per_sm);

/* CTAs per SM of the kernels for rows that are 16- but not 32-byte aligned
 * (realigned = 0) and for rows that are not 16-byte aligned (realigned = 1),
 * per (kind, fmt): 1 = one CTA of 512 threads per SM (a shared-memory
 * reservation keeps a second one off the SM), 0 = as many as fit.  Outputs
 * never change.  Returns 0 or RNG_ERR_ARG. */
int gbrng_set_row_ctas(int kind, int fmt, int realigned, int ctas_per_sm);
int gbrng_get_row_ctas(int kind, int fmt, int realigned, int *ctas_per_sm);

/* Sequence splitting of few-stream calls (rng_generate, rng_generate_reduce):
 * `log2_rows` is log2 of the fewest rows a segment may have for `kind`
 * (1..30); 0 turns splitting off for the kind.  A split generate call takes
 * as many segments as bring its threads up to 2048 per SM (1024 for a
 * consumer call), each a power-of-two number of rows no smaller than that.
 * Outputs never change. */
int gbrng_set_split(int kind, int log2_rows);
int gbrng_get_split(int kind, int *log2_rows);

/* Write-only bandwidth probe: fills `bytes` (a multiple of 16) of the DEVICE
 * buffer `dst` with 16-byte stores from a grid of `blocks` x `threads`
 * (grid-stride), on `cuda_stream`, `reps` times back to back.  hint as
 * above.  Asynchronous.  The paper measured its card's achievable bandwidth
 * the same way, with writes only (Sec. "Discussion"). */
int gbrng_probe_write(void *dst, uint64_t bytes, int blocks, int threads, int hint,
                      int reps, void *cuda_stream);

/* Integer-pipe probe: every thread runs `iters` iterations of `op` on each
 * of 8 independent chains (op 0 = 32x32->64 multiply-add as in one MWC step,
 * 2 instructions; op 1 = 32-bit multiply-add as in the LCG, 1; op 2 =
 * shift + xor as in a xorshift step, 2; op 3 = 32-bit add, 1), each written
 * as volatile inline PTX so that none is folded or dropped, and writes one
 * word per thread to `sink` (DEVICE, blocks*threads uint32).  Asynchronous.
 * Used to measure the integer throughput the generators can reach (the
 * paper's U_ops, Eq. 9). */
int gbrng_probe_int(int op, uint32_t *sink, int blocks, int threads, uint64_t iters,
                    void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* GBRNG_RNG_TUNE_H */
