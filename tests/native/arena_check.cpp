// Drives the serving arena (paper_1101_1846_gb300/csrc/arena.h) from a
// script on stdin: "size granule" first, then "a BYTES" (alloc: prints
// "1 OFFSET" or "0 0") and "r OFFSET BYTES" (release: prints the bytes in
// use, the free blocks and the largest of them), so that a test can compare
// it with a model.
#include <cinttypes>
#include <cstdio>

#include "arena.h"

int main()
{
    uint64_t size = 0, granule = 0;
    if (std::scanf("%" SCNu64 " %" SCNu64, &size, &granule) != 2 || granule == 0)
        return 2;
    gbrng::Arena a(size, granule);
    std::printf("%" PRIu64 "\n", a.size());
    char op = 0;
    while (std::scanf(" %c", &op) == 1) {
        if (op == 'a') {
            uint64_t bytes = 0, off = 0;
            if (std::scanf("%" SCNu64, &bytes) != 1)
                return 2;
            const bool ok = a.alloc(bytes, &off);
            std::printf("%d %" PRIu64 " %" PRIu64 "\n", ok ? 1 : 0, ok ? off : 0, a.used());
        } else if (op == 'r') {
            uint64_t off = 0, bytes = 0;
            if (std::scanf("%" SCNu64 " %" SCNu64, &off, &bytes) != 2)
                return 2;
            a.release(off, bytes);
            std::printf("%" PRIu64 " %zu %" PRIu64 "\n", a.used(), a.free_blocks(), a.largest());
        } else {
            return 2;
        }
    }
    return 0;
}
