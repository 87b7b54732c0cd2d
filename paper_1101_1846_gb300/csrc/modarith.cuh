// Modular arithmetic on the device: Montgomery multiplication with R = 2^64
// and R = 2^32 (Montgomery, "Modular multiplication without trial
// division", Math. Comp. 44, 1985).  Used by the multiplier search
// (Miller-Rabin) and by the MWC jump-ahead.
#pragma once

#include <stdint.h>

namespace gbrng {

// a * b * R^-1 mod n for a, b < n, n odd; ninv = -n^-1 mod 2^64.
__device__ __forceinline__ uint64_t mont_mul(uint64_t a, uint64_t b, uint64_t n,
                                             uint64_t ninv)
{
    uint64_t lo = a * b, hi = __umul64hi(a, b);
    uint64_t m = lo * ninv;
    uint64_t mn_hi = __umul64hi(m, n);
    // lo + lo(m*n) = 0 mod 2^64, so the low word carries exactly when lo != 0.
    uint64_t s = hi + mn_hi;
    bool over = s < hi;
    uint64_t s2 = s + (lo != 0 ? 1u : 0u);
    over |= s2 < s;
    if (over || s2 >= n)
        s2 -= n;  // true sum is < 2n, so one subtraction suffices
    return s2;
}

// a * b * 2^-32 mod n for a, b < n < 2^32, n odd; ninv = -n^-1 mod 2^32.
__device__ __forceinline__ uint32_t mont_mul32(uint32_t a, uint32_t b, uint32_t n, uint32_t ninv)
{
    const uint64_t t = (uint64_t)a * b;
    const uint32_t m = (uint32_t)t * ninv;
    const uint64_t s = t + (uint64_t)m * n;  // divisible by 2^32; true sum < 2^65
    const uint64_t r = (s >> 32) | ((uint64_t)(s < t) << 32);  // < 2n
    return (uint32_t)(r >= n ? r - n : r);
}

}  // namespace gbrng
