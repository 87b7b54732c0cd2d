// Jump-ahead on the device: the state of a stream k steps later without
// the steps in between (sequence splitting, Sec. "Parallelizing RNGs").
//
//   MWC     With p = a 2^32 - 1 and t = a x + c (0 < t < p), one step maps t
//           to a t mod p (a = 2^-32 mod p; the step is Lehmer's generator
//           in disguise), so k steps multiply t by a^k mod p.  In Montgomery
//           form with R = 2^64, a R = 2^32 (mod p) since a 2^32 = p + 1, and
//           -p^-1 = 1 + a 2^32 (mod 2^64) since p (1 + a 2^32) = a^2 2^64 - 1:
//           no division or inversion is needed to set up the powering.
//           Multiplying a residue X = h 2^32 + l by a is a l + h (< p): one
//           MWC step applied to X.
//   xor128, xorshift32
//           GF(2)-linear: k steps apply M^k, the product of the tables'
//           M^(2^m) over the set bits m of k (powers of one matrix commute).
//   LCG     affine: the composed maps (A_m, C_m) of 2^m steps.
//   MWC16X2 each base-2^16 part by the same Lehmer argument with
//           p = a 2^16 - 1 < 2^32, in plain 64-bit arithmetic.
//   XORSHIFT8  GF(2) with 256 x 256 matrices (the tables' third part).
#pragma once

#include "gen_body.cuh"
#include "modarith.cuh"

namespace gbrng {

__device__ __forceinline__ uint64_t mwc_mul_a(uint64_t X, uint32_t a)
{
    return (uint64_t)a * (uint32_t)X + (X >> 32);
}

// a^k mod p in Montgomery form, k >= 1.
__device__ __forceinline__ uint64_t mwc_power(uint32_t a, uint64_t k)
{
    const uint64_t p = ((uint64_t)a << 32) - 1;
    const uint64_t ninv = ((uint64_t)a << 32) + 1;
    uint64_t A = (uint64_t)1 << 32;  // a^1 in Montgomery form: the top bit of k
    for (int bit = 62 - __clzll((long long)k); bit >= 0; --bit) {
        A = mont_mul(A, A, p, ninv);
        if ((k >> bit) & 1)
            A = mwc_mul_a(A, a);
    }
    return A;
}

// (x, c) <- the state whose t is A t mod p, for A = a^k in Montgomery form.
__device__ __forceinline__ void mwc_apply(uint64_t A, uint32_t a, uint32_t &x, uint32_t &c)
{
    const uint64_t p = ((uint64_t)a << 32) - 1;
    const uint64_t ninv = ((uint64_t)a << 32) + 1;
    const uint64_t t = mont_mul(A, (uint64_t)a * x + c, p, ninv);  // a^k t mod p
    x = (uint32_t)(t / a);
    c = (uint32_t)(t - (uint64_t)x * a);
}

__device__ __forceinline__ void mwc_jump(uint32_t a, uint32_t &x, uint32_t &c, uint64_t k)
{
    if (k != 0)
        mwc_apply(mwc_power(a, k), a, x, c);
}

// One base-2^16 part packed as z = x | c << 16, multiplier a < 2^16: k steps
// multiply t = a x + c by a^k mod p (p = a 2^16 - 1); then x = t div a,
// c = t mod a.  The power is taken in Montgomery form with R = 2^32, where
// a is 2^16 (a 2^16 = 1 mod p, so a R = 2^16 mod p) and -p^-1 mod 2^32 is
// 1 + a 2^16, so nothing needs a division; left to right from k's top bit.
__device__ __forceinline__ void mwc16_jump(uint32_t a, uint32_t &z, uint64_t k)
{
    if (k == 0)
        return;
    const uint32_t p = (a << 16) - 1u;
    const uint32_t ninv = (a << 16) + 1u;
    const uint32_t base = 1u << 16;  // a in Montgomery form
    uint32_t A = base;
    for (int bit = 62 - __clzll((long long)k); bit >= 0; --bit) {
        A = mont_mul32(A, A, p, ninv);
        if ((k >> bit) & 1u)
            A = mont_mul32(A, base, p, ninv);
    }
    // A = a^k R mod p; one more product with t (plain) gives a^k t mod p
    const uint32_t t = mont_mul32(A, a * (z & 0xFFFFu) + (z >> 16), p, ninv);
    z = (t / a) | ((t % a) << 16);
}

// v <- M v for a 128 x 128 GF(2) matrix given by columns (word w of column j
// in col[j]); the four streams of a group share every column load.
template <int G>
__device__ __forceinline__ void gf2_apply128(const uint4 *__restrict__ col,
                                             uint32_t (&w)[kMaxWords][4])
{
    uint32_t r[4][G];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int i = 0; i < G; ++i)
            r[q][i] = 0;
#pragma unroll
    for (int word = 0; word < 4; ++word) {
#pragma unroll 4
        for (int b = 0; b < 32; ++b) {
            const uint4 m = __ldg(col + 32 * word + b);
#pragma unroll
            for (int i = 0; i < G; ++i) {
                const uint32_t mask = 0u - ((w[word][i] >> b) & 1u);
                r[0][i] ^= m.x & mask;
                r[1][i] ^= m.y & mask;
                r[2][i] ^= m.z & mask;
                r[3][i] ^= m.w & mask;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int i = 0; i < G; ++i)
            w[q][i] = r[q][i];
}

// v <- M v for a 256 x 256 GF(2) matrix: column j is col[2j] (words 0-3)
// and col[2j + 1] (words 4-7).
template <int G>
__device__ __forceinline__ void gf2_apply256(const uint4 *__restrict__ col,
                                             uint32_t (&w)[kMaxWords][4])
{
    uint32_t r[8][G];
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
        for (int i = 0; i < G; ++i)
            r[q][i] = 0;
#pragma unroll
    for (int word = 0; word < 8; ++word) {
#pragma unroll 2
        for (int b = 0; b < 32; ++b) {
            const uint4 lo = __ldg(col + 2 * (32 * word + b));
            const uint4 hi = __ldg(col + 2 * (32 * word + b) + 1);
#pragma unroll
            for (int i = 0; i < G; ++i) {
                const uint32_t mask = 0u - ((w[word][i] >> b) & 1u);
                r[0][i] ^= lo.x & mask;
                r[1][i] ^= lo.y & mask;
                r[2][i] ^= lo.z & mask;
                r[3][i] ^= lo.w & mask;
                r[4][i] ^= hi.x & mask;
                r[5][i] ^= hi.y & mask;
                r[6][i] ^= hi.z & mask;
                r[7][i] ^= hi.w & mask;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
        for (int i = 0; i < G; ++i)
            w[q][i] = r[q][i];
}

__device__ __forceinline__ uint32_t gf2_apply32(const uint32_t *__restrict__ col, uint32_t y)
{
    uint32_t r = 0;
#pragma unroll 8
    for (int b = 0; b < 32; ++b)
        r ^= __ldg(col + b) & (0u - ((y >> b) & 1u));
    return r;
}

// Jumps G streams held as w[word][i] (the vector bodies' layout; G = 1 for
// a single stream) with multipliers a[i] by k steps.  With MWC_DONE the
// base-2^32 MWC words are left alone (the caller has applied a tabulated
// multiplier).
template <int KIND, int G, bool MWC_DONE = false>
__device__ __forceinline__ void jump_streams(uint32_t (&w)[kMaxWords][4],
                                             const uint32_t (&a)[4], uint64_t k,
                                             const JumpTables &T)
{
    if (k == 0)
        return;
    if constexpr ((KIND == RNG_MWC32 || KIND == RNG_KISS) && !MWC_DONE) {
#pragma unroll
        for (int i = 0; i < G; ++i)
            mwc_jump(a[i], w[0][i], w[1][i], k);
    }
    if constexpr (KIND == RNG_MWC16X2 || KIND == RNG_KISS_XOR) {
#pragma unroll
        for (int i = 0; i < G; ++i) {
            mwc16_jump(a[i] & 0xFFFFu, w[0][i], k);
            mwc16_jump(a[i] >> 16, w[1][i], k);
        }
    }
    if constexpr (KIND == RNG_XOR128) {
        for (uint64_t r = k; r; r &= r - 1)
            gf2_apply128<G>(T.xor128 + 128 * (__ffsll((long long)r) - 1), w);
    }
    if constexpr (KIND == RNG_XORSHIFT8) {
        for (uint64_t r = k; r; r &= r - 1)
            gf2_apply256<G>(T.xs8 + 512 * (__ffsll((long long)r) - 1), w);
    }
    if constexpr (KIND == RNG_KISS || KIND == RNG_KISS_XOR) {
        for (uint64_t r = k; r; r &= r - 1) {
            const int m = __ffsll((long long)r) - 1;
            const uint2 lc = __ldg(T.lcg + m);
#pragma unroll
            for (int i = 0; i < G; ++i) {
                w[2][i] = gf2_apply32(T.xs32 + 32 * m, w[2][i]);
                w[3][i] = lc.x * w[3][i] + lc.y;
            }
        }
    }
}

// The same for one stream in an Engine.  A != 0 (MWC32, KISS): the MWC part
// is multiplied by A = a^k in Montgomery form (a tabulated power) instead of
// powering.
template <int KIND>
__device__ __forceinline__ void jump_engine(Engine<KIND> &e, uint64_t k, const JumpTables &T,
                                            uint64_t A = 0)
{
    uint32_t w[kMaxWords][4] = {};
    uint32_t a[4] = {};
    if constexpr (KIND == RNG_MWC32) {
        w[0][0] = e.x;
        w[1][0] = e.c;
        a[0] = e.a;
    } else if constexpr (KIND == RNG_XOR128) {
        w[0][0] = e.s0;
        w[1][0] = e.s1;
        w[2][0] = e.s2;
        w[3][0] = e.s3;
    } else if constexpr (KIND == RNG_KISS) {
        w[0][0] = e.x;
        w[1][0] = e.c;
        w[2][0] = e.y;
        w[3][0] = e.z;
        a[0] = e.a;
    } else if constexpr (KIND == RNG_MWC16X2) {
        w[0][0] = e.z;
        w[1][0] = e.w;
        a[0] = e.a;
    } else if constexpr (KIND == RNG_XORSHIFT8) {
#pragma unroll
        for (int q = 0; q < 8; ++q)
            w[q][0] = e.v[q];
    } else {
        w[0][0] = e.z;
        w[1][0] = e.w;
        w[2][0] = e.y;
        w[3][0] = e.l;
        a[0] = e.a;
    }
    if constexpr (KIND == RNG_MWC32 || KIND == RNG_KISS) {
        if (A != 0 && k != 0) {
            mwc_apply(A, a[0], w[0][0], w[1][0]);
            jump_streams<KIND, 1, true>(w, a, k, T);
        } else {
            jump_streams<KIND, 1>(w, a, k, T);
        }
    } else {
        jump_streams<KIND, 1>(w, a, k, T);
    }
    if constexpr (KIND == RNG_MWC32) {
        e.x = w[0][0];
        e.c = w[1][0];
    } else if constexpr (KIND == RNG_XOR128) {
        e.s0 = w[0][0];
        e.s1 = w[1][0];
        e.s2 = w[2][0];
        e.s3 = w[3][0];
    } else if constexpr (KIND == RNG_KISS) {
        e.x = w[0][0];
        e.c = w[1][0];
        e.y = w[2][0];
        e.z = w[3][0];
    } else if constexpr (KIND == RNG_MWC16X2) {
        e.z = w[0][0];
        e.w = w[1][0];
    } else if constexpr (KIND == RNG_XORSHIFT8) {
#pragma unroll
        for (int q = 0; q < 8; ++q)
            e.v[q] = w[q][0];
    } else {
        e.z = w[0][0];
        e.w = w[1][0];
        e.y = w[2][0];
        e.l = w[3][0];
    }
}

}  // namespace gbrng
