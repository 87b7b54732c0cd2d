// Prints the batch items the serving engine makes for pieces read from
// stdin ("n c m" per line): one line per piece, "count" then, per item,
// "s_begin s_end rows offset ld" with offset = item.out - out.
#include <cinttypes>
#include <cstdio>
#include <vector>

#include "pieces.h"

int main()
{
    uint64_t n = 0, c = 0, m = 0;
    std::vector<uint32_t> out(1);
    while (std::scanf("%" SCNu64 " %" SCNu64 " %" SCNu64, &n, &c, &m) == 3) {
        std::vector<rng_batch_item> items;
        gbrng::piece_items(nullptr, n, c, m, out.data(), 0, items);
        std::printf("%zu", items.size());
        for (const rng_batch_item &it : items)
            std::printf(" %" PRIu64 " %" PRIu64 " %" PRIu64 " %td %" PRIu64, it.s_begin, it.s_end,
                        it.n_per_stream, static_cast<uint32_t *>(it.out) - out.data(), it.ld);
        std::printf("\n");
    }
    return 0;
}
