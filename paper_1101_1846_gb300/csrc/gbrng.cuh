// Internal declarations of the GB300 generator library (not installed; the
// public interface is include/rng.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gbrng_device.cuh"
#include "rng.h"

namespace gbrng {

// The recurrences (mwc_step, xor128_step, xorshift32_step, lcg_step,
// kiss_step, unit_f32) are defined once, in the public device header; every
// kernel of the library uses them.

// ------------------------------------------------------------- handles
struct Gen {
    int kind = 0;
    int device = 0;
    uint64_t n = 0;          // streams
    uint64_t seed = 0;
    int words = 0;           // state words per stream
    uint32_t *d_state = nullptr;  // SoA: word w of stream s at d_state[w*n + s]
    uint32_t *d_a = nullptr;      // multipliers (MWC32, KISS), n entries
    cudaStream_t stream = nullptr;
    // Split calls (few streams, long sequences; allocated at creation when
    // n <= kSplitMaxStreams):
    uint32_t *d_split = nullptr;  // final state stash, same layout as d_state
    uint32_t *d_cnt = nullptr;    // arrival counters, n entries, zero between calls
    uint64_t *d_jmul = nullptr;   // MWC jump multipliers: a^(y*jmul_rows) mod p in
                                  // Montgomery form at d_jmul[y*n + s], y < jmul_cap;
                                  // allocated by the first split call that needs it
    uint64_t jmul_rows = 0;       // rows per segment the table was built for (0: none)
    uint32_t jmul_cap = 0;        // segments the table holds
    uint32_t jmul_segs = 0;       // most segments a split call of this handle has
    // staging for rng_generate_host
    void *d_stage[2] = {nullptr, nullptr};
    size_t stage_bytes = 0;
    cudaEvent_t stage_ev[2] = {nullptr, nullptr};
};

// Launch parameters of one generate call (host side).
struct GenLaunch {
    uint32_t *state;      // SoA base, stride n
    const uint32_t *a;    // multipliers or nullptr
    uint64_t n;           // streams of the generator
    uint64_t s_begin;     // first stream advanced by this call
    uint64_t s_end;       // one past the last
    uint64_t steps;       // outputs per stream in this call
    void *out;            // device output: element (j, s) at out[j*ld + s - s_begin]
    uint64_t ld;          // row stride in elements
    Gen *owner = nullptr;  // handle whose split buffers a split call uses;
                           // nullptr: never split
};

int set_error(int status);
int cuda_status(cudaError_t e);

// multipliers.cu: makes the device table at least k long; returns its base.
int multiplier_table(uint64_t k, const uint32_t **table);
// The packed base-2^16 multiplier pairs of MWC16X2 / KISS_XOR streams (all
// RNG_MAX_STREAMS_MWC16 of them, built once per device; synchronises then).
int mwc16_pair_table(uint64_t k, const uint32_t **pairs);

// seed.cu
int launch_seed(Gen *g, cudaStream_t st);

constexpr int kKinds = 6;

// generate.cu: the launch shape of the vector kernels per (kind, fmt)
// (gbrng_set_launch), and one generate call of any kind.
struct LaunchShape {
    int v;      // groups of four streams per thread
    int block;  // CTA size
    int hint;   // streaming stores
    int one;    // one CTA per SM
};
// The shape for a call of `streams` streams (its size class).
LaunchShape launch_shape(int kind, int fmt, uint64_t streams);
// CTAs per SM of the barrier-synced kernels for rows that are not 32-byte
// aligned (realigned: rows not 16-byte aligned): 1, or 0 for as many as fit.
int row_ctas(int kind, int fmt, bool realigned);
// Dynamic shared memory that keeps `kernel`, launched with `threads`
// threads, to one CTA per SM: more than half an SM's shared memory (nothing
// is stored there; the reservation only bars a second CTA).  0 when the
// device cannot tell or the kernel would not fit; sets the kernel's limit.
int one_cta_smem(const void *kernel, int threads);
int launch_generate(int kind, int fmt, const GenLaunch &p, cudaStream_t st);
// generate_paper.cu: the same for RNG_MWC16X2, RNG_XORSHIFT8, RNG_KISS_XOR.
int launch_generate_paper(int kind, int fmt, const GenLaunch &p, cudaStream_t st);
// Segments of a split call: rows per segment (a power of two) and count
// (at most max_segments); returns false when the call should run unsplit.
// `streams` are the streams the call advances, `streams_per_thread` how many
// of them one thread takes.
// fill_threads: the threads the segments should add up to (split_fill).
bool split_plan(int kind, uint64_t streams, uint64_t steps, uint64_t streams_per_thread,
                uint64_t max_segments, uint64_t fill_threads, uint64_t *rows,
                uint64_t *segments);
// Threads a split call aims for: generate calls, or consumer
// (rng_generate_reduce) calls.
uint64_t split_fill(bool reduce);

// jump.cu: device tables of the GF(2) and affine jumps, built on first use
// on the current device (synchronises then).
struct JumpTables {
    const uint4 *xor128;      // [m][j]: column j of M^(2^m), M = one xor128 step
    const uint32_t *xs32;     // [m][j]: column j of X^(2^m), X = one xorshift32 step
    const uint2 *lcg;         // [m]: (A, C) of the LCG map applied 2^m times
    const uint4 *xs8;         // [m][2j], [m][2j+1]: column j of Y^(2^m), Y = one
                              // XORSHIFT8 step (words 0-3, 4-7)
};
int jump_tables(JumpTables *t);
int launch_jump(Gen *g, uint64_t k, cudaStream_t st);
// The handle's MWC jump multipliers for `segs` segments of `rows` rows,
// rebuilt on `st` when `rows` differs from the table's (MWC32 and KISS
// handles only).  The table is allocated, or grown, when a call needs more
// segments than it holds (synchronises then; never inside a capture).
int mwc_jump_table(Gen *g, uint64_t rows, uint64_t segs, cudaStream_t st,
                   const uint64_t **table);
// Most segments a split call on a handle of n streams can have.
uint32_t split_max_segments(uint64_t n);

inline int words_of(int kind)
{
    return kind == RNG_MWC32 || kind == RNG_MWC16X2 ? 2 : kind == RNG_XORSHIFT8 ? 8 : 4;
}
inline bool has_mult(int kind) { return kind != RNG_XOR128 && kind != RNG_XORSHIFT8; }
// Kinds whose split jumps use the handle's table of Montgomery powers.
inline bool mont_table(int kind) { return kind == RNG_MWC32 || kind == RNG_KISS; }
// Kinds that need the device jump tables (GF(2) or affine parts).
inline bool needs_jump_tables(int kind) { return kind != RNG_MWC32 && kind != RNG_MWC16X2; }

// Mapped tiles of the batched kernel: each output's format and place come
// from its tile's output map (gen_body.cuh, OutMap).  kFmtMixed is the
// format value of such tiles; kFmtEnd ends a map.
constexpr int kFmtMixed = 2;
constexpr uint32_t kFmtEnd = 0xFFFFFFFFu;

// batch.cu: refills a plan (rng_plan_refill) with tiles whose outputs are
// placed and encoded by output maps (OutMap layout, in host words `maps`;
// item i's map starts at word map_off[i], its origin a device address), and
// makes its launches run the mapped-tile kernel.  The items' fmt fields are
// ignored; each item's out pointer is its place in the map's virtual window.
// Same rules and errors as rng_plan_refill.
int plan_refill_mixed(rng_plan_handle p, const rng_batch_item *items, size_t n_items,
                      const uint64_t *map_off, const uint32_t *maps, uint64_t map_words,
                      cudaStream_t stream);

// Handles with at most this many streams keep a split scratch (split calls
// only happen for stream counts well below it).
constexpr uint64_t kSplitMaxStreams = (uint64_t)1 << 19;

}  // namespace gbrng
