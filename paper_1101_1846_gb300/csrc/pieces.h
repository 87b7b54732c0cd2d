// How the serving engine cuts a client's samples into batch items (host-only,
// tested on the CPU by itself).  Sample g of a client's sequence is output
// g / n of stream g % n.  A piece of m samples starting at sample c covers
// columns 0 .. m-1 of a row-major window whose column `col` belongs to stream
// (c % n + col) % n: columns below m % n get one output more than the
// others.  Each column range maps to at most two contiguous stream ranges
// (the window wraps around stream n-1), so a piece is at most four batch
// items with disjoint stream ranges of one generator.
#pragma once

#include <stdint.h>

#include <algorithm>
#include <vector>

#include "rng.h"

namespace gbrng {

// Appends the items of one piece: m samples of `h` (n streams) from sample c
// on, written to out[0 .. m) in sequence order.
inline void piece_items(rng_handle h, uint64_t n, uint64_t c, uint64_t m, uint32_t *out, int fmt,
                        std::vector<rng_batch_item> &items)
{
    const uint64_t r = c % n, q = m / n, rem = m % n;
    auto columns = [&](uint64_t c0, uint64_t c1, uint64_t rows) {
        if (rows == 0 || c0 >= c1)
            return;
        const uint64_t a1 = std::min(c1, n - r);  // columns [c0, a1): streams r + col
        if (c0 < a1)
            items.push_back(rng_batch_item{h, rows, out + c0, fmt, r + c0, r + a1, n});
        const uint64_t b0 = std::max(c0, n - r);  // columns [b0, c1): streams col - (n - r)
        if (b0 < c1)
            items.push_back(
                rng_batch_item{h, rows, out + b0, fmt, b0 - (n - r), c1 - (n - r), n});
    };
    columns(0, rem, q + 1);
    columns(rem, n, q);
}

}  // namespace gbrng
