// Prints the batch items the serving engine makes for pieces read from
// stdin ("n c m split" per line; split = 1 also runs split_aligned with the
// window placed at word phase c mod 8): one line per piece, "count" then,
// per item, "s_begin s_end rows offset ld" with offset = item.out - out.
#include <cinttypes>
#include <cstdio>
#include <vector>

#include "pieces.h"

int main()
{
    uint64_t n = 0, c = 0, m = 0;
    int split = 0;
    std::vector<uint32_t> buf(64);
    while (std::scanf("%" SCNu64 " %" SCNu64 " %" SCNu64 " %d", &n, &c, &m, &split) == 4) {
        // the window's first element at a word address congruent to c mod 8
        uint32_t *out = buf.data() + 16;
        out -= (reinterpret_cast<uintptr_t>(out) / 4 - c) % 8;
        std::vector<rng_batch_item> items;
        gbrng::piece_items(nullptr, n, c, m, out, 0, items);
        if (split)
            gbrng::split_aligned(items, 0);
        std::printf("%zu", items.size());
        for (const rng_batch_item &it : items)
            std::printf(" %" PRIu64 " %" PRIu64 " %" PRIu64 " %td %" PRIu64, it.s_begin, it.s_end,
                        it.n_per_stream, static_cast<uint32_t *>(it.out) - out, it.ld);
        std::printf("\n");
    }
    return 0;
}
