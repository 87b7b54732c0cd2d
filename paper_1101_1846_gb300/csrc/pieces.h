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

// Splits items[first ..) at multiples of 8 streams, where that makes their
// middles 32-byte aligned: an item whose row stride is a multiple of 8 and
// whose output of stream s sits at a word address congruent to s modulo 8
// (the serving engine places every output so) becomes up to three items: the
// streams before the first multiple of 8, the streams from there to the last
// multiple of 8 (aligned rows: the batched kernel's barrier-free vector
// tiles), and the rest.  Other items stay as they are.  The stream ranges
// stay disjoint and every output keeps its place.
inline void split_aligned(std::vector<rng_batch_item> &items, size_t first)
{
    const size_t end = items.size();
    for (size_t i = first; i < end; ++i) {
        const rng_batch_item it = items[i];
        const uint64_t w = (uint64_t)(reinterpret_cast<uintptr_t>(it.out) / 4);
        if (it.ld % 8 != 0 || (w - it.s_begin) % 8 != 0)
            continue;
        const uint64_t a = std::min((it.s_begin + 7) / 8 * 8, it.s_end);
        const uint64_t b = std::max(a, it.s_end / 8 * 8);
        if (b == a || (a == it.s_begin && b == it.s_end))
            continue;  // nothing aligned to split off, or aligned already
        auto part = [&](uint64_t s0, uint64_t s1) {
            rng_batch_item q = it;
            q.s_begin = s0;
            q.s_end = s1;
            q.out = static_cast<uint32_t *>(it.out) + (s0 - it.s_begin);
            return q;
        };
        items[i] = part(a, b);
        if (it.s_begin < a)
            items.push_back(part(it.s_begin, a));
        if (b < it.s_end)
            items.push_back(part(b, it.s_end));
    }
}

}  // namespace gbrng
