/*
 * C-ABI of the GB300 library for the Marsaglia generators of Hissoiny,
 * Despres and Ozell, "Using graphics processing units to generate random
 * numbers" (arXiv:1101.1846): many independent generator streams, each with
 * its own parameters and seeds (Sec. "Parallelizing RNGs", parametrisation),
 * writing uint32 or single-precision uniforms to device memory (Sec.
 * "Performance evaluation").
 *
 * Generators (kind):
 *   RNG_MWC32  multiply-with-carry, base 2^32 (Eq. 2-3):
 *              t = a*x + c (64-bit); x' = t mod 2^32; c' = t >> 32; out = x'.
 *              Stream s has multiplier a = the (s+1)-th largest a < 2^32 with
 *              a*2^32 - 1 a safe prime (background MWC section).
 *   RNG_XOR128 Marsaglia's xor128 XorShift (4 x 32-bit words; the paper's
 *              XorShift reference, Marsaglia 2003): t = x ^ (x << 11);
 *              (x, y, z) = (y, z, w); w = w ^ (w >> 19) ^ t ^ (t >> 8); out = w.
 *   RNG_KISS   KISS (Sec. "KISS"): one MWC32 step (as above), one xorshift32
 *              step y ^= y<<13; y ^= y>>17; y ^= y<<5 (Eq. 6) and one LCG
 *              step z = 69069 z + 1234567 mod 2^32 (Eq. 7); out is the sum
 *              of the three new values mod 2^32.
 *   The paper's own generators:
 *   RNG_MWC16X2  two base-2^16 MWCs (Methods / MWC), each kept as one word
 *              z = x + c 2^16 and stepped as z' = a (z & 0xFFFF) + (z >> 16);
 *              out = (z' << 16) + w' mod 2^32.  Stream s has the s-th pair
 *              (i < j, lexicographic) of the 392 multipliers a < 2^16 with
 *              a 2^16 - 1 a safe prime (largest first): a1 = table[i] for z,
 *              a2 = table[j] for w.
 *   RNG_XORSHIFT8  Panneton's r = 8, s = 7 XorShift (Eq. 5): words
 *              (v_{n-8} .. v_{n-1}); v_n = (I+L^9)(I+L^13) v_{n-1} +
 *              (I+L^7) v_{n-4} + (I+R^3) v_{n-5} + (I+R^10) v_{n-7} +
 *              (I+L^24)(I+R^7) v_{n-8} (xor; products applied right to left);
 *              out = v_n.
 *   RNG_KISS_XOR  KISS in the paper's form: ((MWC16X2 xor LCG) + xorshift32)
 *              mod 2^32, with the MWC pair, Eq. 6 and Eq. 7 as above.
 * Formats (fmt):
 *   RNG_U32    the 32-bit output.
 *   RNG_F32    (float)(u >> 8) * 2^-24, exactly; in [0, 1 - 2^-24]
 *              (the uniform variant of Sec. "Performance evaluation").
 *
 * Seeding: stream s of a generator created with `seed` draws from
 * splitmix64 started at seed + s (mod 2^64): MWC (x, c) = (lo32, hi32 mod a)
 * of a draw, redrawn while (x, c) is (0, 0) or (2^32 - 1, a - 1); xor128
 * words = lo32, hi32 of two draws, redrawn while all zero; KISS (x, c) as
 * MWC, then y = lo32 and z = hi32 of the next draw, y redrawn (lo32 of
 * further draws) while zero.  MWC16X2: from one draw r, part 1 x = bits
 * 0-15, c = bits 16-31 mod a1, part 2 x = bits 32-47, c = bits 48-63 mod a2,
 * redrawn while either part is a fixed point; XORSHIFT8: the eight words are
 * lo32, hi32 of four draws, redrawn while all zero; KISS_XOR: the MWC pair as
 * MWC16X2, then y and the LCG word as KISS.
 *
 * Output layout (stream-interleaved): output j (0-based, counted from the
 * start of the call) of stream s is element out[j * n_streams + s].  Each
 * call continues every stream where the previous call on the handle left it
 * (the state is written back after every call, Sec. "Performance
 * evaluation").
 *
 * Conventions for every call:
 *   - Return 0 (RNG_OK) on success or a negative rng_status.  rng_create
 *     returns NULL on failure.  The status of the last failing call on the
 *     calling host thread is kept for rng_last_error().
 *   - Device work is enqueued on the handle's CUDA stream (default: the
 *     legacy default stream; see rng_set_stream) and the call returns
 *     without waiting, except where a call says it synchronises.
 *   - A failed call leaves the generator state unchanged, except after
 *     RNG_ERR_CUDA from an already-launched kernel (the CUDA context is then
 *     in an error state).
 *   - A handle is not thread-safe: use each one from one host thread at a
 *     time.  Different handles are independent.
 *   - The device is the one current on the calling thread at rng_create;
 *     later calls on the handle make it current themselves.
 */
#ifndef GBRNG_RNG_H
#define GBRNG_RNG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rng_gen *rng_handle;

enum rng_kind {
    RNG_MWC32 = 0,
    RNG_XOR128 = 1,
    RNG_KISS = 2,
    RNG_MWC16X2 = 3,
    RNG_XORSHIFT8 = 4,
    RNG_KISS_XOR = 5
};
enum rng_fmt { RNG_U32 = 0, RNG_F32 = 1 };

enum rng_status {
    RNG_OK = 0,
    RNG_ERR_ARG = -1,     /* invalid argument (kind, fmt, size, pointer)    */
    RNG_ERR_OOM = -2,     /* device or host allocation failed               */
    RNG_ERR_CUDA = -3,    /* a CUDA runtime call or kernel launch failed    */
    RNG_ERR_TIMEOUT = -4, /* a bounded device-side wait gave up             */
    RNG_ERR_BUSY = -5,    /* admission refused: over the stated budget      */
    RNG_ERR_NODEV = -6    /* no CUDA device, or not an sm_103 device        */
};

/* Largest stream count of an MWC32 or KISS generator: the size of the
 * multiplier table (valid multipliers exist for about 5.6 million a < 2^32;
 * this bound keeps the device search to a = 1.05e9 and above). */
#define RNG_MAX_STREAMS_MWC ((uint64_t)1 << 22)
/* Largest stream count of an xor128 generator (no multiplier table). */
#define RNG_MAX_STREAMS_XOR ((uint64_t)1 << 30)
/* Largest stream count of an MWC16X2 or KISS_XOR generator: the number of
 * distinct pairs of the 392 base-2^16 multipliers. */
#define RNG_MAX_STREAMS_MWC16 ((uint64_t)392 * 391 / 2)
/* Largest stream count of an XORSHIFT8 generator (8 GiB of state). */
#define RNG_MAX_STREAMS_XS8 ((uint64_t)1 << 28)

/* Creates a generator of `kind` with n_streams independent streams seeded
 * from `seed` (header comment).  Allocates the per-stream state (and, for
 * MWC32/KISS, the stream multipliers) on the current device, builds the
 * device multiplier table if it is not yet long enough (once per device and
 * process; synchronises), and seeds every stream on the device.  Returns
 * NULL with rng_last_error() = RNG_ERR_ARG for a bad kind or n_streams of 0
 * or above the kind's maximum, RNG_ERR_OOM, RNG_ERR_CUDA or RNG_ERR_NODEV.
 * Paper: per-thread multipliers and seeds (MWC and KISS kernel sections;
 * Sec. "Parallelizing RNGs"). */
rng_handle rng_create(int kind, uint64_t n_streams, uint64_t seed);

/* Creates a generator that holds streams s_begin .. s_begin + n_streams - 1
 * of the generator rng_create(kind, s_begin + n_streams, seed) would make:
 * its stream s gets global stream s_begin + s's multiplier (or pair) and
 * its seed, splitmix64 started at seed + s_begin + s.  Every output and
 * state is then equal to that stream of the one large generator, so a
 * stream range can live on its own device (one range per GPU) and no call
 * ever exchanges data between ranges.  RNG_ERR_ARG when s_begin + n_streams
 * exceeds the kind's maximum stream count; other errors as rng_create.
 * Paper: parametrisation, each stream its own multiplier and seeds
 * (Sec. "Parallelizing RNGs"). */
rng_handle rng_create_range(int kind, uint64_t s_begin, uint64_t n_streams, uint64_t seed);

/* Releases the handle and its device memory (waits for its stream first).
 * NULL is ignored. */
void rng_destroy(rng_handle h);

/* Makes the handle enqueue its work on `cuda_stream` (a cudaStream_t; NULL
 * = the legacy default stream).  The caller keeps ownership of the stream
 * and must not destroy it while work of the handle is pending. */
int rng_set_stream(rng_handle h, void *cuda_stream);

/* Number of streams and of 32-bit state words per stream (2 for MWC32 and
 * MWC16X2, 8 for XORSHIFT8, 4 for the others). */
uint64_t rng_n_streams(rng_handle h);
int rng_state_words(rng_handle h);

/* The hot path.  Advances every stream n_per_stream times and writes the
 * outputs, stream-interleaved (header comment), to `out`: a DEVICE pointer,
 * caller-owned, with room for n_streams * n_per_stream 4-byte elements,
 * 4-byte aligned.  With n_streams % 4 == 0 and 16-byte alignment every row
 * is 16-byte aligned; otherwise the rows are realigned in registers and
 * still written with 16-byte stores, and the last n_streams % 4 streams
 * use 4-byte stores; the results are the same.  Calls longer than 2^31
 * steps run as several launches.  fmt is RNG_U32 or RNG_F32.  n_per_stream = 0 does
 * nothing and returns RNG_OK.  Asynchronous on the handle's stream.
 * Errors: RNG_ERR_ARG (NULL handle or out, bad fmt, misaligned out),
 * RNG_ERR_CUDA (launch failure).
 * Paper: the generation kernels of Sec. "GPU implementations" (MWC, XorShift
 * registers variant, KISS) and the uniform variant of Sec. "Performance
 * evaluation". */
int rng_generate(rng_handle h, uint64_t n_per_stream, void *out, int fmt);
/* Few streams with long sequences: when n_streams is too small to fill the
 * device and rows are 32-byte aligned, rng_generate cuts each stream's
 * outputs into segments of 2^l rows (l chosen per kind; gbrng_set_split),
 * starts every segment from the state jumped ahead to it (rng_jump) and
 * runs the segments side by side; the final state goes through a scratch
 * buffer allocated with the handle.  For MWC32 and KISS the segments' MWC
 * jumps come from a per-handle table of multipliers (8 bytes per stream and
 * segment), allocated by the first split call that needs it and grown when
 * a call needs more segments: that call synchronises the device and returns
 * RNG_ERR_OOM if the allocation fails.  A split call captured in a CUDA
 * graph never allocates; it powers the multipliers in the kernel instead.
 * The outputs and the state are those of the plain sequence (sequence
 * splitting, Sec. "Parallelizing RNGs"). */

/* Advances only streams [s_begin, s_end) (0 <= s_begin < s_end <= n_streams)
 * n_per_stream times; the other streams keep their state.  Output j of
 * stream s goes to out[j * ld + (s - s_begin)]: `out` is a DEVICE pointer to
 * the element of stream s_begin in row 0, 4-byte aligned, and ld >=
 * s_end - s_begin is the row stride in elements (ld = n_streams and the full
 * range give rng_generate).  A serving layer uses this to continue a
 * stream-interleaved sequence from the middle of a row.  Asynchronous.
 * Errors: RNG_ERR_ARG (bad range, ld or pointer), RNG_ERR_CUDA.
 * Paper: the per-thread generators of Sec. "Parallelizing RNGs" advanced
 * independently. */
int rng_generate_range(rng_handle h, uint64_t s_begin, uint64_t s_end,
                       uint64_t n_per_stream, void *out, uint64_t ld, int fmt);

/* Same outputs as rng_generate, delivered to HOST memory: `host_out` has
 * room for n_streams * n_per_stream 4-byte elements in the same layout.
 * The library generates blocks of rows into its own device staging buffers
 * (allocated on first use, kept with the handle) and copies each block to
 * the host while the next is generated.  Page-locked host memory is
 * copied asynchronously; pageable memory works but is slower.  SYNCHRONISES
 * the handle's stream before returning.  Errors as rng_generate, plus
 * RNG_ERR_OOM for the staging buffers.
 * Paper: the generated numbers stay in device memory for later kernels or
 * are copied to host memory afterwards (Sec. "Performance evaluation"). */
int rng_generate_host(rng_handle h, uint64_t n_per_stream, void *host_out,
                      int fmt);

/* Copies the state to/from HOST memory: word w of stream s at
 * buf[w * n_streams + s] (uint32), rng_state_words(h) words per stream, so
 * `bytes` must be exactly 4 * words * n_streams.  Both synchronise the
 * handle's stream.  rng_set_state rejects (RNG_ERR_ARG, state unchanged) an
 * MWC or KISS state whose carry is not below its multiplier or that is an
 * MWC fixed point, an all-zero xor128 state and a zero KISS xorshift word.
 * Paper: the state is written back to global memory after each call so that
 * the sequence can continue (Sec. "Performance evaluation"). */
int rng_get_state(rng_handle h, void *host_buf, size_t bytes);
int rng_set_state(rng_handle h, const void *host_buf, size_t bytes);

/* Inline consumers (op) of rng_generate_reduce. */
enum rng_reduce_op {
    RNG_SUM_U32 = 0, /* sum of the outputs, mod 2^64                          */
    RNG_SUM_U24 = 1, /* sum of u >> 8: exactly 2^24 x the sum of the uniforms  */
    RNG_DISC = 2     /* outputs taken in consecutive pairs (u0, u1) as points
                        (x, y) of their uniforms: the number of points with
                        x^2 + y^2 < 1, tested exactly as
                        (u0>>8)^2 + (u1>>8)^2 < 2^48; an unpaired last output
                        is drawn and ignored.  4 x count / pairs estimates pi */
};

/* Advances every stream n_per_stream times, exactly as rng_generate does
 * (same state afterwards), but writes no outputs: each output is consumed
 * where it is made, and out[s] receives the consumer `op` applied to
 * stream s's outputs of this call.  `out` is a DEVICE pointer, caller-owned,
 * n_streams uint64 values, 8-byte aligned.  Asynchronous on the handle's
 * stream.  Errors: RNG_ERR_ARG (NULL handle or out, bad op, misaligned
 * out), RNG_ERR_OOM (the split scratch, below), RNG_ERR_CUDA.
 * Few streams with long sequences are split like rng_generate's (each
 * stream's outputs cut into segments that start from jumped states; the
 * segment results are added, which is exact in integers).
 * Paper: the generators timed without writing the numbers back, only the
 * final state (Sec. "Performance evaluation"; Tables I-III). */
int rng_generate_reduce(rng_handle h, uint64_t n_per_stream, int op, void *out);

/* Advances every stream by k steps without computing the outputs in
 * between, in O(log k) work per stream: MWC by modular exponentiation
 * (with p = a 2^32 - 1 and t = a x + c, one step maps t to a t mod p), the
 * xorshift parts by powers of their GF(2) matrices (tables of M^(2^m) built
 * once per device on first use; synchronises then), the LCG by composing
 * its affine map.  The state afterwards equals k single steps.
 * Asynchronous on the handle's stream.  Errors: RNG_ERR_ARG, RNG_ERR_OOM,
 * RNG_ERR_CUDA.
 * Paper: sequence splitting needs the i-th number without the ones before
 * it (Sec. "Parallelizing RNGs"). */
int rng_jump(rng_handle h, uint64_t k);

/* Most birthday-spacings samples rng_battery takes (2^21, a bound on the
 * work; the statistics compare the repeat counts with their distribution at
 * 512 days in a year of 2^24, which holds at millions of samples). */
#define RNG_BATTERY_BIRTHDAY_MAX ((uint64_t)1 << 21)

/* Counts of a small statistical battery (rng_battery). */
typedef struct rng_battery_counts {
    uint64_t n_outputs;        /* outputs counted                              */
    uint64_t ones;             /* monobit: one bits in all outputs             */
    uint64_t bytes[256];       /* frequency: outputs by their top 8 bits       */
    uint64_t serial[256];      /* serial: non-overlapping pairs (u_2k, u_2k+1)
                                  of a stream by (u_2k >> 28) * 16 + (u_2k+1 >> 28) */
    uint64_t birthday_samples; /* birthday spacings: samples of 512
                                  consecutive outputs of a stream; sample i is
                                  block i / n_streams of stream i % n_streams,
                                  for i < min(floor(n_per_stream / 512) *
                                  n_streams, RNG_BATTERY_BIRTHDAY_MAX)       */
    uint64_t birthday[16];     /* samples by repeated spacings (15: 15 or more):
                                  days = top 24 bits, sorted; spacings = the
                                  first day and neighbour differences, sorted;
                                  repeats = spacings equal to the one before.
                                  Asymptotically Poisson with mean
                                  512^3 / (4 * 2^24) = 2                      */
} rng_battery_counts;

/* Counts the battery over generator outputs in device memory: `dev_u`
 * (DEVICE, uint32, 4-byte aligned) holds n_per_stream rows of n_streams
 * outputs, output j of stream s at dev_u[j * n_streams + s] (rng_generate's
 * layout); the counts go to *host_counts (HOST).  Runs on cuda_stream and
 * SYNCHRONISES it; allocates a few KB of device memory for the call.
 * Errors: RNG_ERR_ARG, RNG_ERR_OOM, RNG_ERR_CUDA.
 * Paper: the generators' randomness is assessed with DIEHARD and TestU01
 * (Sec. "Performance evaluation"); these four tests come from those
 * families (monobit, frequency, serial, Marsaglia's birthday spacings). */
int rng_battery(const void *dev_u, uint64_t n_streams, uint64_t n_per_stream,
                rng_battery_counts *host_counts, void *cuda_stream);

/* Where a handle's state lives, for kernels that step the streams
 * themselves (include/gbrng_device.cuh, Engine<KIND>). */
typedef struct rng_device_view {
    int kind;            /* rng_kind                                         */
    int device;          /* CUDA device of the handle                        */
    int state_words;     /* 2 (MWC32) or 4                                   */
    uint64_t n_streams;
    void *state;         /* DEVICE uint32: word w of stream s at
                            state[w * n_streams + s]; owned by the handle    */
    const void *mult;    /* DEVICE uint32 multiplier of stream s at mult[s]
                            (MWC32, KISS); NULL for xor128                   */
} rng_device_view;

/* Fills *view.  The pointers stay valid until rng_destroy.  A kernel that
 * reads or writes the state must be ordered with the handle's own work
 * (enqueue it on the handle's stream).  Errors: RNG_ERR_ARG. */
int rng_get_device_view(rng_handle h, rng_device_view *view);

/* Writes the first k stream multipliers (the MWC32/KISS table: a < 2^32,
 * largest first, a*2^32 - 1 a safe prime) to `dev_out` (DEVICE pointer,
 * caller-owned, k uint32).  Builds the table on the current device if it is
 * not yet long enough; SYNCHRONISES the device.  k <= RNG_MAX_STREAMS_MWC.
 * Paper: the multiplier condition of the background MWC section. */
int rng_multipliers(uint64_t k, uint32_t *dev_out);

/* Writes the first k multiplier pairs of MWC16X2 / KISS_XOR streams, packed
 * a1 | a2 << 16, to `dev_out` (DEVICE, caller-owned, k uint32); k <=
 * RNG_MAX_STREAMS_MWC16.  Builds the 392-entry base-2^16 table on the
 * current device on first use; SYNCHRONISES the device.
 * Paper: pairs of the 392 multipliers, one pair per thread (Methods / MWC). */
int rng_mwc16_pairs(uint64_t k, uint32_t *dev_out);

/* One entry of a batched launch: generator h advances streams
 * [s_begin, s_end) n_per_stream times and writes output j of stream s to
 * out[j * ld + (s - s_begin)] (DEVICE pointer, 4-byte aligned) in format
 * fmt.  s_end = 0 means n_streams, ld = 0 means n_streams; with both 0 and
 * s_begin = 0 the item is rng_generate(h, n_per_stream, out, fmt). */
typedef struct rng_batch_item {
    rng_handle h;
    uint64_t n_per_stream;
    void *out;
    int fmt;
    uint64_t s_begin;
    uint64_t s_end;
    uint64_t ld;
} rng_batch_item;

typedef struct rng_plan *rng_plan_handle;

/* Builds a batched launch over many generators of mixed kinds, stream
 * counts, lengths and formats: the streams of every item are cut into tiles
 * of 4 * threads streams when its rows are 16-byte aligned, else of
 * 4 * (31 * threads / 32 + 1) streams (the last (s_end - s_begin) % 4
 * streams of such an item run in the last warp of its last tile when that
 * warp holds no group, else in a tile of their own), the tiles are ordered
 * by length, largest first, and
 * the work list is copied to the device (synchronises).  threads = CTA size
 * (power of two, 32..512; 0 = 512), ctas_per_sm = resident CTAs the
 * persistent grid puts on each SM (1..32; 0 = as many as fit); both 0 = the
 * default shape, CTAs of 512 threads, one per SM (the fastest measured on
 * GB300).  With ctas_per_sm = 1 the launch reserves more than half an SM's
 * shared memory (unused) so that no SM takes a second CTA.  Items of the
 * same handle must cover disjoint stream ranges (they then run side by
 * side); items with n_per_stream = 0 are
 * skipped.  The plan refers to the handles' device
 * memory and the out pointers: it must not outlive them.  Items must be
 * of the kinds RNG_MWC32, RNG_XOR128 or RNG_KISS (the persistent kernel
 * carries the bodies of those three only, so that the paper's larger-state
 * variants do not cost the common case registers).  Returns NULL with
 * rng_last_error() = RNG_ERR_ARG (bad item or kind, duplicate handle, handles
 * on different devices, n_per_stream >= 2^32), RNG_ERR_OOM or RNG_ERR_CUDA.
 * Paper: none; the parametrised streams of Sec. "Parallelizing RNGs" served
 * as one launch. */
rng_plan_handle rng_plan_create(const rng_batch_item *items, size_t n_items,
                                int threads, int ctas_per_sm);

/* Enqueues the plan on `cuda_stream`: a counter reset and ONE persistent
 * kernel whose CTAs take tiles from the work list through an atomic counter
 * (no device-side waits).  Outputs and state afterwards are bit-identical to
 * calling rng_generate on each item in turn; launching again continues every
 * stream, like a second rng_generate.  No host synchronisation, so the call
 * can be captured in a CUDA graph and replayed.  Two launches of the same
 * plan must not overlap on the device. */
int rng_plan_launch(rng_plan_handle p, void *cuda_stream);

/* Replaces the plan's work list with the tiles of a new set of items (same
 * rules as rng_plan_create; the CTA size and grid stay), enqueueing the copy
 * to the device on `cuda_stream`: a later rng_plan_launch on the same stream
 * runs the new list, and a launch still in flight on that stream finishes
 * with the old one.  The tiles keep the items' order (no length ordering),
 * so that a serving loop can rebuild a plan every tick cheaply.  Allocates
 * device memory only when the list outgrows every earlier one (after waiting
 * for `cuda_stream`).  The tiles are written to one of two pinned host lists
 * owned by the plan, used in turn, and copied without the call waiting; a
 * refill waits only if the copy out of its list (two refills earlier) has not
 * finished.  `items` may be reused as soon as the call returns.
 * Errors: RNG_ERR_ARG (as rng_plan_create, or items on another device),
 * RNG_ERR_OOM, RNG_ERR_CUDA. */
int rng_plan_refill(rng_plan_handle p, const rng_batch_item *items, size_t n_items,
                    void *cuda_stream);

/* Tiles in the plan, and its CTA size and persistent grid size. */
uint64_t rng_plan_tiles(rng_plan_handle p);
int rng_plan_shape(rng_plan_handle p, int *threads, int *grid);

/* Frees the plan (waits for its device work first).  NULL is ignored. */
void rng_plan_destroy(rng_plan_handle p);

/* Convenience: create a plan with the default shape, launch it on
 * `cuda_stream`, wait for it, and free it.  SYNCHRONISES. */
int rng_generate_batch(const rng_batch_item *items, size_t n_items,
                       void *cuda_stream);

/* ---------------------------------------------------------------------
 * Serving engine: many clients, each with its own device-resident
 * generator of streams_per_client streams (seeded with seed_base + client
 * id), answering requests for the next N samples of the client's sequence.
 * Sample g of a client's sequence (g = 0, 1, ...) is output number
 * g / streams_per_client of stream g % streams_per_client, so a client's
 * sequence is the stream-interleaved output of its generator read row by
 * row, and requests of one client take consecutive ranges of it in the
 * order they were submitted.  Results are the same whatever other requests
 * share the device (each is a function of its client and range only).
 *
 * The engine keeps submitted requests in a FIFO and admits a request when
 * its output fits in the device arena (the HBM budget minus the generators'
 * state; first fit).  On every tick the engine runs one batched launch (a
 * refilled plan) that advances every client with admitted work by one piece
 * of at most chunk_rows rows of its sequence: the piece starts at the
 * client's first unfinished request and runs on through the admitted
 * requests after it, each request's part going to that request's output in
 * its own format.  Requests that arrive while others run join the next tick
 * (continuous batching); while a tick runs, a lane waits for a quarter of
 * the target tick size (rng_server_set_tick_bytes) before it launches the
 * next one.  Clients are split into two
 * lanes (even and odd ids) with a CUDA stream each, so that one lane's tick
 * overlaps the other's; up to two ticks per lane are in flight.  A request's output (uint32 or
 * float, N elements, contiguous, in sequence order) stays in the arena until
 * it is released; it starts at a word index congruent to its first sample's
 * index in the client's sequence modulo 8 (so 4-byte aligned, and 16-byte
 * aligned only when that index is a multiple of 4).  Not thread-safe: drive one engine from one host thread.
 * Paper: none; the parametrised generators of Sec. "Parallelizing RNGs"
 * served on demand.
 * ------------------------------------------------------------------- */
typedef struct rng_server *rng_server_handle;

/* kind: RNG_MWC32, RNG_XOR128 or RNG_KISS (the engine batches through the
 * persistent kernel of rng_plan_create); n_clients >= 1; streams_per_client
 * within the kind's maximum; budget_bytes: device memory for state plus outputs;
 * chunk_rows >= 1.  Allocates everything up front (synchronises).  NULL on
 * failure (rng_last_error(): RNG_ERR_ARG, RNG_ERR_OOM when the budget does
 * not cover the state, RNG_ERR_CUDA, RNG_ERR_NODEV). */
rng_server_handle rng_server_create(int kind, uint32_t n_clients,
                                    uint64_t streams_per_client, uint64_t seed_base,
                                    uint64_t budget_bytes, uint32_t chunk_rows);

/* Queues a request for the next n_samples samples of `client` in format
 * fmt; *req_id receives its id (ids count up from 0).  The request's range
 * of the client's sequence is fixed here, at submission.  RNG_ERR_ARG for a
 * bad client or fmt, n_samples = 0, or an output larger than the arena less
 * the 28 bytes of room its placement may need. */
int rng_server_submit(rng_server_handle s, uint32_t client, uint64_t n_samples, int fmt,
                      uint64_t *req_id);

/* rng_server_submit for n requests at once (arrays of clients, sizes and
 * formats; ids written to req_ids if not NULL), in array order.  Checks all
 * of them first: nothing is queued if any is invalid. */
int rng_server_submit_many(rng_server_handle s, const uint32_t *clients,
                           const uint64_t *n_samples, const int *fmts, size_t n,
                           uint64_t *req_ids);

/* Does the engine's work without blocking: retires finished ticks, admits
 * queued requests that now fit, and launches the next tick when fewer than
 * two are in flight.  Returns the number of requests completed so far
 * (ready to be taken), or a negative status. */
int rng_server_progress(rng_server_handle s);

/* Blocks until every submitted request has completed (driving progress). */
int rng_server_drain(rng_server_handle s);

/* Takes up to `cap` completed requests: ids[i] and done_ms[i], the device
 * time of completion in milliseconds since the engine was created (from
 * CUDA events).  Returns how many were taken. */
int rng_server_take(rng_server_handle s, uint64_t *ids, double *done_ms, int cap);

/* Where a completed (not yet released) request's output is: *dev_ptr (in
 * the arena), *n_samples, *fmt, *client, *start (its first sample index in
 * the client's sequence).  RNG_ERR_ARG for an unknown or released id. */
int rng_server_result(rng_server_handle s, uint64_t req_id, void **dev_ptr,
                      uint64_t *n_samples, int *fmt, uint32_t *client, uint64_t *start);

/* Copies elements [offset, offset + count) of a completed request's output
 * to dst (device or host memory) on cuda_stream, a cudaStream_t (NULL: the
 * legacy default stream, as everywhere in this library).  The tick that
 * produced a completed request has finished, so any stream may be used.
 * Asynchronous: the caller synchronises cuda_stream (or orders its own work
 * after the copy on it), and releases the request only after the copy is
 * done. */
int rng_server_copy(rng_server_handle s, uint64_t req_id, void *dst, uint64_t offset,
                    uint64_t count, void *cuda_stream);

/* Returns a completed request's output space to the arena. */
int rng_server_release(rng_server_handle s, uint64_t req_id);

/* rng_server_release for n requests; returns the first error, after
 * releasing every valid id. */
int rng_server_release_many(rng_server_handle s, const uint64_t *req_ids, size_t n);

/* Counters: [0] submitted, [1] admitted, [2] completed, [3] ticks,
 * [4] samples generated, [5] arena bytes in use, [6] arena bytes total,
 * [7] requests waiting for admission. */
int rng_server_stats(rng_server_handle s, uint64_t *out8);

/* Sizes ticks by output bytes: each tick gives every client with admitted
 * work an equal share of `bytes` (at least one row, at most chunk_rows
 * rows), so that ticks stay short under light load (latency) and grow under
 * a backlog (throughput).  0 (the default) gives every client chunk_rows
 * rows per tick. */
int rng_server_set_tick_bytes(rng_server_handle s, uint64_t bytes);

/* Shape of the engine's persistent kernel, as rng_plan_create's `threads`
 * (a power of two in [32, 512]; default 512) and `ctas_per_sm` (0 = as many
 * as fit; default 1).  Synchronises the engine's streams if ticks have run;
 * the next tick of each lane uses the new shape.  Output is the same for any shape.
 * RNG_ERR_ARG outside those ranges. */
int rng_server_set_plan_shape(rng_server_handle s, int threads, int ctas_per_sm);

/* Waits for the engine's work and frees everything.  NULL is ignored. */
void rng_server_destroy(rng_server_handle s);

/* Allocation-free variant of rng_generate_batch, for callers that cannot
 * allocate device memory when they need samples: an application whose own
 * pool allocator holds the whole device budget, or a latency-sensitive loop
 * that must not pay for, or be synchronised by, cudaMalloc and cudaFree.
 * Same outputs and state afterwards as rng_generate_batch on the same items
 * (same work list and kernel, CTA size 128).  The work list and its tile
 * counter live in one fixed device array inside the library, of 256 bytes
 * plus 32768 tiles of 64 bytes (2 MB, held by every GPU that loads the library
 * until the process exits): a call may cover at most 4096 items and 32768
 * tiles (an item of c = s_end - s_begin streams takes ceil(c / 512) tiles
 * when its rows are 16-byte aligned, else ceil((c - c % 4) / 500) tiles plus
 * at most one when c % 4 != 0); more returns RNG_ERR_ARG and launches nothing.  No cudaMalloc, cudaFree or other allocating routine is
 * called.  The first call on a device looks up the device address of that
 * array (once per device), so make the first call before any stream capture.
 * That address is kept until the process exits, like the library's other
 * per-device tables: cudaDeviceReset is not supported while the library is
 * in use.
 * Asynchronous on `cuda_stream`: the work list is copied from library host
 * memory before the call returns.  Every call shares the one array, which
 * keeps the last call's contents; calls whose kernels overlap on the GPU
 * race and give wrong results, so order them on one stream or with events.
 * Errors as rng_generate_batch.  The paper has no counterpart. */
int rng_generate_batch_noalloc(const rng_batch_item *items, size_t n_items,
                               void *cuda_stream);

/* Status of the last failing call on this host thread (RNG_OK if none);
 * and a static description of a status code. */
int rng_last_error(void);
const char *rng_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* GBRNG_RNG_H */
