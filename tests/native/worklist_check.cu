// Host-only driver of the batched launch's work-list builder: includes the
// library's batch.cu to reach fill_units and order_units, builds the work
// list of items read from stdin (no CUDA call is made), and prints the tiles.
// Input: "threads n_items", then per item "kind fmt n s_begin s_end ld
// out_words steps" (out_words: the output's offset in 4-byte words from a
// 256-byte aligned base).  Output per tile: "item mode s0 count tail
// out_words steps".
#include <cinttypes>
#include <cstdio>
#include <vector>

#include "batch.cu"

// stand-ins for the library's status helpers (defined with its handles)
namespace gbrng {
int set_error(int status) { return status; }
int cuda_status(cudaError_t e) { return e == cudaSuccess ? 0 : RNG_ERR_CUDA; }
int one_cta_smem(const void *, int) { return 0; }
}  // namespace gbrng
extern "C" int rng_last_error(void) { return 0; }

int main()
{
    using namespace gbrng;
    int threads = 0;
    size_t n_items = 0;
    if (std::scanf("%d %zu", &threads, &n_items) != 2)
        return 2;
    // stand-in device addresses: never dereferenced by the builder
    uint32_t *const base = reinterpret_cast<uint32_t *>(uintptr_t{1} << 40);
    std::vector<Gen> gens(n_items);
    std::vector<rng_batch_item> items(n_items);
    for (size_t i = 0; i < n_items; ++i) {
        int kind = 0, fmt = 0;
        uint64_t n = 0, s_begin = 0, s_end = 0, ld = 0, out_words = 0, steps = 0;
        if (std::scanf("%d %d %" SCNu64 " %" SCNu64 " %" SCNu64 " %" SCNu64 " %" SCNu64
                       " %" SCNu64,
                       &kind, &fmt, &n, &s_begin, &s_end, &ld, &out_words, &steps) != 8)
            return 2;
        gens[i].kind = kind;
        gens[i].n = n;
        gens[i].d_state = reinterpret_cast<uint32_t *>((uintptr_t)(i + 1) << 32);
        gens[i].d_a = reinterpret_cast<uint32_t *>(((uintptr_t)(i + 1) << 32) + 16);
        items[i] = rng_batch_item{reinterpret_cast<rng_handle>(&gens[i]), steps,
                                  base + out_words, fmt, s_begin, s_end, ld};
    }
    const uint64_t count = fill_units(items.data(), items.size(), threads, nullptr, 0);
    std::vector<Unit> units(count);
    fill_units(items.data(), items.size(), threads, units.data(), count);
    order_units(units.data(), count);
    std::printf("%" PRIu64 "\n", count);
    for (const Unit &u : units) {
        const uint64_t item = ((uintptr_t)u.state >> 32) - 1;
        std::printf("%" PRIu64 " %u %u %u %u %td %" PRIu64 "\n", item, u.code >> 3, u.s0,
                    u.count, u.tail, u.out - base, (uint64_t)u.steps);
    }
    return 0;
}
