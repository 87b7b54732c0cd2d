// 64-bit modular arithmetic on the device: Montgomery multiplication with
// R = 2^64 (Montgomery, "Modular multiplication without trial division",
// Math. Comp. 44, 1985).  Used by the multiplier search (Miller-Rabin) and
// by the MWC jump-ahead.
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

}  // namespace gbrng
