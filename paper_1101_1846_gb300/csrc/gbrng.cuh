// Internal declarations of the GB300 generator library (not installed; the
// public interface is include/rng.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rng.h"

namespace gbrng {

// ---------------------------------------------------------------- steps
// One step of each generator on registers.  These are the only definitions
// of the recurrences in the library; every kernel uses them.

// Eq. 2-3 with b = 2^32: t = a*x + c as a 64-bit value, x' = low word,
// c' = high word.  Written as a multiply-add of the low words that sets the
// carry flag and a multiply-add of the high words that consumes it, which is
// the same 64-bit sum in fewer instructions than a widened add.
__device__ __forceinline__ uint32_t mwc_step(uint32_t a, uint32_t &x, uint32_t &c)
{
    uint32_t lo, hi;
    asm("mad.lo.cc.u32 %0, %2, %3, %4;\n\t"
        "madc.hi.u32 %1, %2, %3, 0;"
        : "=&r"(lo), "=r"(hi)  // lo is written before a and x are read again
        : "r"(a), "r"(x), "r"(c));
    x = lo;
    c = hi;
    return lo;
}

// xor128 (Marsaglia 2003); the four words are renamed in registers.
__device__ __forceinline__ uint32_t xor128_step(uint32_t &s0, uint32_t &s1,
                                                uint32_t &s2, uint32_t &s3)
{
    uint32_t t = s0 ^ (s0 << 11);
    s0 = s1;
    s1 = s2;
    s2 = s3;
    s3 = s3 ^ (s3 >> 19) ^ t ^ (t >> 8);
    return s3;
}

// Eq. 6 applied as <<13, >>17, <<5.
__device__ __forceinline__ uint32_t xorshift32_step(uint32_t &y)
{
    y ^= y << 13;
    y ^= y >> 17;
    y ^= y << 5;
    return y;
}

// Eq. 7 with a = 69069, c = 1234567; mod 2^32 by wrap-around.
__device__ __forceinline__ uint32_t lcg_step(uint32_t &z)
{
    z = 69069u * z + 1234567u;
    return z;
}

// KISS: sum of the three new values mod 2^32.
__device__ __forceinline__ uint32_t kiss_step(uint32_t a, uint32_t &x, uint32_t &c,
                                              uint32_t &y, uint32_t &z)
{
    return mwc_step(a, x, c) + xorshift32_step(y) + lcg_step(z);
}

// (u >> 8) * 2^-24: a 24-bit integer converts exactly and the scaling is a
// power of two, so the result does not depend on the rounding mode.
__device__ __forceinline__ float unit_f32(uint32_t u)
{
    return __uint2float_rn(u >> 8) * 5.9604644775390625e-8f;
}

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
};

int set_error(int status);
int cuda_status(cudaError_t e);

// multipliers.cu: makes the device table at least k long; returns its base.
int multiplier_table(uint64_t k, const uint32_t **table);

// seed.cu
int launch_seed(Gen *g, cudaStream_t st);

// generate.cu
int launch_generate(int kind, int fmt, const GenLaunch &p, cudaStream_t st);

inline int words_of(int kind) { return kind == RNG_MWC32 ? 2 : 4; }

}  // namespace gbrng
