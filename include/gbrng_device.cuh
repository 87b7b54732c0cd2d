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

// The paper's own MWC (Methods / MWC): two base-2^16 MWCs with 16-bit
// multipliers a1 = a_pair & 0xFFFF, a2 = a_pair >> 16, each kept as one word
// x + c 2^16; a step of Eq. 2-3 maps it to a (z mod 2^16) + (z div 2^16),
// and the output joins the new words as (z << 16) + w mod 2^32.
__device__ __forceinline__ uint32_t mwc16x2_step(uint32_t a_pair, uint32_t &z, uint32_t &w)
{
    z = (a_pair & 0xFFFFu) * (z & 0xFFFFu) + (z >> 16);
    w = (a_pair >> 16) * (w & 0xFFFFu) + (w >> 16);
    return (z << 16) + w;
}

// Eq. 5, Panneton's XorShift with r = 8, s = 7: v0..v7 = v_{n-8}..v_{n-1};
// v_n = (I+L^9)(I+L^13) v_{n-1} + (I+L^7) v_{n-4} + (I+R^3) v_{n-5}
//     + (I+R^10) v_{n-7} + (I+L^24)(I+R^7) v_{n-8}, products applied right
// to left; the words shift down and v_n (the output) enters at the top.
__device__ __forceinline__ uint32_t xorshift8_step(uint32_t &v0, uint32_t &v1, uint32_t &v2,
                                                   uint32_t &v3, uint32_t &v4, uint32_t &v5,
                                                   uint32_t &v6, uint32_t &v7)
{
    uint32_t t1 = v7 ^ (v7 << 13);
    t1 ^= t1 << 9;
    uint32_t t8 = v0 ^ (v0 >> 7);
    t8 ^= t8 << 24;
    const uint32_t v = t1 ^ v4 ^ (v4 << 7) ^ v3 ^ (v3 >> 3) ^ v1 ^ (v1 >> 10) ^ t8;
    v0 = v1;
    v1 = v2;
    v2 = v3;
    v3 = v4;
    v4 = v5;
    v5 = v6;
    v6 = v7;
    v7 = v;
    return v;
}

// KISS in the paper's form (Background / KISS): (MWC xor LCG) + xorshift32
// mod 2^32, with the two-part MWC above.
__device__ __forceinline__ uint32_t kiss_xor_step(uint32_t a_pair, uint32_t &z, uint32_t &w,
                                                  uint32_t &y, uint32_t &l)
{
    const uint32_t m = mwc16x2_step(a_pair, z, w);
    return (m ^ lcg_step(l)) + xorshift32_step(y);
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

template <>
struct Engine<RNG_MWC16X2> {
    uint32_t a, z, w;  // a = packed multiplier pair
    __device__ __forceinline__ void load(const rng_device_view &v, uint64_t s)
    {
        const uint32_t *st = static_cast<const uint32_t *>(v.state);
        a = static_cast<const uint32_t *>(v.mult)[s];
        z = st[s];
        w = st[v.n_streams + s];
    }
    __device__ __forceinline__ void store(const rng_device_view &v, uint64_t s) const
    {
        uint32_t *st = static_cast<uint32_t *>(v.state);
        st[s] = z;
        st[v.n_streams + s] = w;
    }
    __device__ __forceinline__ uint32_t next() { return mwc16x2_step(a, z, w); }
    __device__ __forceinline__ float next_f32() { return unit_f32(next()); }
};

template <>
struct Engine<RNG_XORSHIFT8> {
    uint32_t v[8];
    __device__ __forceinline__ void load(const rng_device_view &view, uint64_t s)
    {
        const uint32_t *st = static_cast<const uint32_t *>(view.state);
#pragma unroll
        for (int k = 0; k < 8; ++k)
            v[k] = st[k * view.n_streams + s];
    }
    __device__ __forceinline__ void store(const rng_device_view &view, uint64_t s) const
    {
        uint32_t *st = static_cast<uint32_t *>(view.state);
#pragma unroll
        for (int k = 0; k < 8; ++k)
            st[k * view.n_streams + s] = v[k];
    }
    __device__ __forceinline__ uint32_t next()
    {
        return xorshift8_step(v[0], v[1], v[2], v[3], v[4], v[5], v[6], v[7]);
    }
    __device__ __forceinline__ float next_f32() { return unit_f32(next()); }
};

template <>
struct Engine<RNG_KISS_XOR> {
    uint32_t a, z, w, y, l;
    __device__ __forceinline__ void load(const rng_device_view &v, uint64_t s)
    {
        const uint32_t *st = static_cast<const uint32_t *>(v.state);
        const uint64_t n = v.n_streams;
        a = static_cast<const uint32_t *>(v.mult)[s];
        z = st[s];
        w = st[n + s];
        y = st[2 * n + s];
        l = st[3 * n + s];
    }
    __device__ __forceinline__ void store(const rng_device_view &v, uint64_t s) const
    {
        uint32_t *st = static_cast<uint32_t *>(v.state);
        const uint64_t n = v.n_streams;
        st[s] = z;
        st[n + s] = w;
        st[2 * n + s] = y;
        st[3 * n + s] = l;
    }
    __device__ __forceinline__ uint32_t next() { return kiss_xor_step(a, z, w, y, l); }
    __device__ __forceinline__ float next_f32() { return unit_f32(next()); }
};

}  // namespace gbrng
