// Drives the serving engine's placement rule and piece builder
// (paper_1101_1846_gb300/csrc/runs.h) from a script on stdin, so that a test
// can check them:
//   a BLOCK START    placement_pad: prints the pad in bytes
//   q CAP COUNT (OFF N DONE FMT) x COUNT
//                    run_piece: prints "origin m touched nseg (b fmt shift) x nseg"
#include <cinttypes>
#include <cstdio>
#include <vector>

#include "runs.h"

int main()
{
    char op = 0;
    while (std::scanf(" %c", &op) == 1) {
        if (op == 'a') {
            uint64_t block = 0, start = 0;
            if (std::scanf("%" SCNu64 " %" SCNu64, &block, &start) != 2)
                return 2;
            std::printf("%" PRIu64 "\n", gbrng::placement_pad(block, start));
        } else if (op == 'q') {
            uint64_t cap = 0;
            size_t count = 0;
            if (std::scanf("%" SCNu64 " %zu", &cap, &count) != 2 || count == 0)
                return 2;
            std::vector<gbrng::RunReq> reqs(count);
            for (auto &q : reqs)
                if (std::scanf("%" SCNu64 " %" SCNu64 " %" SCNu64 " %d", &q.off, &q.n, &q.done,
                               &q.fmt) != 4)
                    return 2;
            const gbrng::RunPiece p = gbrng::run_piece(reqs.data(), count, cap);
            std::printf("%" PRIu64 " %" PRIu64 " %zu %zu", p.origin, p.m, p.touched,
                        p.segs.size());
            for (const gbrng::Seg &g : p.segs)
                std::printf(" %u %d %" PRId64, g.b, g.fmt, g.shift);
            std::printf("\n");
        } else {
            return 2;
        }
    }
    return 0;
}
