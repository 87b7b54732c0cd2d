/*
 * Device-side interface of the GB300 generator library: the recurrences as
 * inline device functions, and Engine<KIND>, one stream's state in
 * registers, for kernels that use the numbers where they are made instead
 * of reading them back from memory (the paper's inline use, in which only
 * the final state is stored: Sec. "Performance evaluation").
 *
 * The library's own kernels are built from these same definitions, so a
 * user kernel that steps a stream through Engine produces exactly the
 * outputs rng_generate would have written, and leaves exactly the state.
 *
 * Use:
 *   rng_device_view v;  rng_get_device_view(h, &v);   // host, once
 *   my_kernel<<<...>>>(v, ...);                       // on the handle's stream
 *
 *   __global__ void my_kernel(rng_device_view v, ...) {
 *       uint64_t s = ...;                              // one stream per thread
 *       gbrng::Engine<RNG_KISS> e;
 *       e.load(v, s);
 *       for (...) { float u = e.next_f32(); ... }
 *       e.store(v, s);                                 // state carries on
 *   }
 *
 * A stream's state must be loaded and stored by one thread at a time, and
 * the user kernel must be ordered with the library's own work on the
 * handle (same CUDA stream, or events).
 */
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rng.h"

namespace gbrng {

// ---------------------------------------------------------------- steps

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

// ------------------------------------------------------------- engines
// One stream's state in registers.  load()/store() read and write word w of
// stream s at view.state[w * n_streams + s] (the handle's layout).
template <int KIND>
struct Engine;

template <>
struct Engine<RNG_MWC32> {
    uint32_t a, x, c;
    __device__ __forceinline__ void load(const rng_device_view &v, uint64_t s)
    {
        const uint32_t *st = static_cast<const uint32_t *>(v.state);
        a = static_cast<const uint32_t *>(v.mult)[s];
        x = st[s];
        c = st[v.n_streams + s];
    }
    __device__ __forceinline__ void store(const rng_device_view &v, uint64_t s) const
    {
        uint32_t *st = static_cast<uint32_t *>(v.state);
        st[s] = x;
        st[v.n_streams + s] = c;
    }
    __device__ __forceinline__ uint32_t next() { return mwc_step(a, x, c); }
    __device__ __forceinline__ float next_f32() { return unit_f32(next()); }
};

template <>
struct Engine<RNG_XOR128> {
    uint32_t s0, s1, s2, s3;
    __device__ __forceinline__ void load(const rng_device_view &v, uint64_t s)
    {
        const uint32_t *st = static_cast<const uint32_t *>(v.state);
        const uint64_t n = v.n_streams;
        s0 = st[s];
        s1 = st[n + s];
        s2 = st[2 * n + s];
        s3 = st[3 * n + s];
    }
    __device__ __forceinline__ void store(const rng_device_view &v, uint64_t s) const
    {
        uint32_t *st = static_cast<uint32_t *>(v.state);
        const uint64_t n = v.n_streams;
        st[s] = s0;
        st[n + s] = s1;
        st[2 * n + s] = s2;
        st[3 * n + s] = s3;
    }
    __device__ __forceinline__ uint32_t next() { return xor128_step(s0, s1, s2, s3); }
    __device__ __forceinline__ float next_f32() { return unit_f32(next()); }
};

template <>
struct Engine<RNG_KISS> {
    uint32_t a, x, c, y, z;
    __device__ __forceinline__ void load(const rng_device_view &v, uint64_t s)
    {
        const uint32_t *st = static_cast<const uint32_t *>(v.state);
        const uint64_t n = v.n_streams;
        a = static_cast<const uint32_t *>(v.mult)[s];
        x = st[s];
        c = st[n + s];
        y = st[2 * n + s];
        z = st[3 * n + s];
    }
    __device__ __forceinline__ void store(const rng_device_view &v, uint64_t s) const
    {
        uint32_t *st = static_cast<uint32_t *>(v.state);
        const uint64_t n = v.n_streams;
        st[s] = x;
        st[n + s] = c;
        st[2 * n + s] = y;
        st[3 * n + s] = z;
    }
    __device__ __forceinline__ uint32_t next() { return kiss_step(a, x, c, y, z); }
    __device__ __forceinline__ float next_f32() { return unit_f32(next()); }
};

}  // namespace gbrng
