// Launch policy of the generation kernels (shapes, splitting) and the
// dispatch of a call to its kind's launcher (gen_kernels.cuh): the three
// target kinds are instantiated here, the paper's own generators in
// generate_paper.cu.
#include <mutex>
#include <vector>

#include "gen_kernels.cuh"
#include "rng_tune.h"

namespace gbrng {
namespace {

// Launch shape per (kind, fmt): groups of four streams per thread V, CTA
// size, store hint, and one = one CTA per SM (a shared-memory reservation
// keeps a second CTA off the SM).  Defaults are the best measured on GB300;
// gbrng_set_launch / gbrng_set_launch_class change the first three (the
// autotuner does), gbrng_set_launch_ctas the last.
struct Shape {
    int v;
    int block;
    int hint;
    int one;
};
// MWC uint32 writes its rows through TMA bulk copies (hint 2): 6 % faster
// per launch on GB300 than 16-byte stores from two CTAs per SM, level with
// them from one.  xor128 uint32 was 1.4 % faster through TMA until 16-byte
// stores from one CTA per SM overtook it (below); the FP32 forms measured
// the same, and KISS and XORSHIFT8, whose steps cost more, ran 4-40 %
// slower that way.  Per-warp bulk copies of 512 B (each warp
// staging its own rows, no block barrier) were slower than both.
//
// Two size classes: calls of fewer than kSmallStreams streams (class 0) and
// the rest (class 1).  At 2^20 streams x 1024 the kernels fill the GPU
// differently (medians of three sweeps of every shape on one GB300): xor128
// FP32 ran 1345 GS/s with its 2^22 shape (1, 128) and 1615 with (2, 128);
// KISS FP32 1580 with (2, 512), 1619 with (1, 256) and 1706 with (1, 128);
// xor128 uint32 1691 through TMA and 1728 with (1, 128) and plain stores.
//
// One CTA of 512 threads per SM, against the best shapes without it (two
// rounds on one GB300, GS/s): at 2^22 x 1024, MWC f32 1807 -> 1821, xor128
// u32 1790-1800 (TMA) -> 1804, xor128 f32 1771 -> 1805, KISS u32 1757 ->
// 1797, KISS f32 1716 -> 1813 (with plain stores; 1765 streaming); MWC u32
// stays with TMA (1823 against 1818).  At 2^20 x 1024 only xor128 f32 gains
// (1609-1614 -> 1717 with V = 2).  As for the barrier-synced kernels, fewer
// warps writing at once keep each SM's write stream denser.
Shape g_shape[2][kKinds][2] = {
    {
        {{1, 256, 2, 0}, {2, 512, 1, 0}},  // MWC u32, f32
        {{1, 128, 0, 0}, {2, 512, 1, 1}},  // xor128
        {{2, 512, 1, 0}, {1, 128, 1, 0}},  // KISS
        {{2, 256, 1, 0}, {2, 256, 1, 0}},  // MWC16X2
        {{1, 256, 1, 0}, {1, 256, 1, 0}},  // XORSHIFT8 (eight state words per stream)
        {{2, 256, 1, 0}, {2, 256, 1, 0}},  // KISS_XOR
    },
    {
        {{1, 256, 2, 0}, {1, 512, 1, 1}},  // MWC u32, f32
        {{1, 512, 1, 1}, {1, 512, 1, 1}},  // xor128
        {{1, 512, 1, 1}, {1, 512, 0, 1}},  // KISS
        {{2, 256, 1, 0}, {2, 256, 1, 0}},  // MWC16X2
        {{1, 256, 1, 0}, {1, 256, 1, 0}},  // XORSHIFT8 (eight state words per stream)
        {{2, 256, 1, 0}, {2, 256, 1, 0}},  // KISS_XOR
    },
};
constexpr uint64_t kSmallStreams = (uint64_t)1 << 21;

// CTAs per SM of the barrier-synced kernels, [kind][fmt][realigned]: 1 =
// one CTA of 512 threads per SM, 0 = as many as fit (two at their register
// counts).  Measured on GB300 at (2^22 - 4) x 1024 (16-byte rows) and
// (2^22 - 2) x 1024 (realigned), GS/s with two CTAs -> with one:
//   MWC u32 1760 -> 1766 / 1686 -> 1756;  MWC f32 1717 -> 1783 / 1694 -> 1772
//   xor128 u32 1663 -> 1746 / 1689 -> 1753;  xor128 f32 1670 -> 1695 / 1710 -> 1685
//   KISS u32 1713 -> 1797 / 1683 -> 1744;  KISS f32 1720 -> 1617 / 1690 -> 1441
// Where the step is cheap, fewer warps writing at once keep the write
// stream denser; the FP32 forms of xor128 and KISS need the second CTA's
// warps to cover their arithmetic.  The paper's kinds keep 0 (not measured).
int g_row_ctas[kKinds][2][2] = {
    {{1, 1}, {1, 1}},  // MWC u32 (16-byte rows, realigned), f32
    {{1, 1}, {1, 0}},  // xor128
    {{1, 1}, {0, 0}},  // KISS
    {{0, 0}, {0, 0}},  // MWC16X2
    {{0, 0}, {0, 0}},  // XORSHIFT8
    {{0, 0}, {0, 0}},  // KISS_XOR
};

// Fewest rows of a split segment, as log2, per kind (0: never split).  The
// jump that starts a segment costs about as much as this many rows: MWC32 a
// tabulated Montgomery product, KISS that plus 32-column GF(2) products,
// xor128 128-column products, the base-2^16 MWC parts a 32-bit Montgomery
// powering each; XORSHIFT8's 256-column products cost more than splitting
// gains.
int g_split_log2[kKinds] = {6, 8, 7, 8, 0, 8};
// Calls of fewer threads than half of this are "few-stream" calls, which
// split when their rows allow.
constexpr uint64_t kFewStreamThreads = (uint64_t)kSMs * 1024;
// Threads a split generate call aims for: 2048 per SM, the most that can be
// resident.  Against 1024 per SM this was measured on GB300 at
// 76,632 x 16,384: MWC32 1584 -> 1740 GS/s, KISS 1575 -> 1680, xor128
// 1575 -> 1670; at 76,636 x 16,384, MWC16X2 1449 -> 1500 and KISS_XOR
// 1541 -> 1680.  Consumer (reduce) calls, one stream per thread, keep 1024.
constexpr uint64_t kSplitFillThreads = (uint64_t)kSMs * 2048;

}  // namespace

LaunchShape launch_shape(int kind, int fmt, uint64_t streams)
{
    const Shape s = g_shape[streams < kSmallStreams ? 0 : 1][kind][fmt];
    return LaunchShape{s.v, s.block, s.hint, s.one};
}

int row_ctas(int kind, int fmt, bool realigned)
{
    return g_row_ctas[kind][fmt][realigned ? 1 : 0];
}

namespace {

// The smallest multiple of 1 KB of dynamic shared memory above half an SM's
// share (less the per-CTA reservation), if the kernel then fits one CTA.
int find_one_cta_smem(const void *kernel, int threads, int dev)
{
    int per_sm = 0, reserved = 0, optin = 0, fit = 0;
    if (cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess)
        return 0;
    // two CTAs would need 2 * (smem + reserved) > per_sm
    const int smem = ((per_sm / 2 - reserved + 1 + 1023) / 1024) * 1024;
    if (smem <= 0 || smem > optin ||
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, kernel, threads, smem) !=
            cudaSuccess ||
        fit != 1) {
        cudaGetLastError();  // leave no sticky error from the probe behind
        return 0;
    }
    return smem;
}

}  // namespace

int one_cta_smem(const void *kernel, int threads)
{
    // answers per (kernel, threads, device), found once each
    struct Known {
        const void *kernel;
        int threads, dev, smem;
    };
    static std::mutex mu;
    static std::vector<Known> known;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return 0;
    std::lock_guard<std::mutex> lock(mu);
    for (const Known &k : known)
        if (k.kernel == kernel && k.threads == threads && k.dev == dev)
            return k.smem;
    const int smem = find_one_cta_smem(kernel, threads, dev);
    known.push_back(Known{kernel, threads, dev, smem});
    return smem;
}

uint64_t split_fill(bool reduce)
{
    return reduce ? kFewStreamThreads : kSplitFillThreads;
}

uint32_t split_max_segments(uint64_t n)
{
    const uint64_t threads = (n + 3) / 4;
    const uint64_t fill = std::max(split_fill(false), split_fill(true));
    return (uint32_t)std::min<uint64_t>(fill / std::max<uint64_t>(threads, 1), 65535);
}

bool split_plan(int kind, uint64_t streams, uint64_t steps, uint64_t streams_per_thread,
                uint64_t max_segments, uint64_t fill_threads, uint64_t *rows,
                uint64_t *segments)
{
    const int l0 = g_split_log2[kind];
    if (l0 == 0 || streams == 0 || streams > kSplitMaxStreams || steps > (1ull << 31))
        return false;
    const uint64_t threads = (streams + streams_per_thread - 1) / streams_per_thread;
    if (2 * threads > kFewStreamThreads)
        return false;  // enough streams to fill the device already
    const uint64_t want = std::min<uint64_t>(std::min<uint64_t>(fill_threads / threads, 65535),
                                             max_segments);
    uint64_t L = 1ull << l0;
    while (L < steps && (steps + L - 1) / L > want)
        L <<= 1;
    const uint64_t S = (steps + L - 1) / L;
    if (S < 2)
        return false;
    *rows = L;
    *segments = S;
    return true;
}

int launch_generate(int kind, int fmt, const GenLaunch &p, cudaStream_t st)
{
    switch (kind) {
    case RNG_MWC32: return launch_kind<RNG_MWC32>(fmt, p, st);
    case RNG_XOR128: return launch_kind<RNG_XOR128>(fmt, p, st);
    case RNG_KISS: return launch_kind<RNG_KISS>(fmt, p, st);
    default: return launch_generate_paper(kind, fmt, p, st);
    }
}

}  // namespace gbrng

extern "C" int gbrng_set_row_ctas(int kind, int fmt, int realigned, int ctas_per_sm)
{
    using namespace gbrng;
    if (kind < 0 || kind >= kKinds || fmt < 0 || fmt > 1 || realigned < 0 || realigned > 1 ||
        ctas_per_sm < 0 || ctas_per_sm > 1)
        return set_error(RNG_ERR_ARG);
    g_row_ctas[kind][fmt][realigned] = ctas_per_sm;
    return RNG_OK;
}

extern "C" int gbrng_get_row_ctas(int kind, int fmt, int realigned, int *ctas_per_sm)
{
    using namespace gbrng;
    if (kind < 0 || kind >= kKinds || fmt < 0 || fmt > 1 || realigned < 0 || realigned > 1 ||
        !ctas_per_sm)
        return set_error(RNG_ERR_ARG);
    *ctas_per_sm = g_row_ctas[kind][fmt][realigned];
    return RNG_OK;
}

extern "C" int gbrng_set_launch_class(int kind, int fmt, int size_class, int v, int block,
                                      int hint)
{
    using namespace gbrng;
    if (kind < 0 || kind >= kKinds || fmt < 0 || fmt > 1 || size_class < 0 || size_class > 1 ||
        (v != 1 && v != 2) || block < 32 || block > 512 || (block & (block - 1)) || hint < 0 ||
        hint > 2)
        return set_error(RNG_ERR_ARG);
    Shape &s = g_shape[size_class][kind][fmt];
    s.v = v;
    s.block = block;
    s.hint = hint;
    return RNG_OK;
}

extern "C" int gbrng_set_launch_ctas(int kind, int fmt, int size_class, int ctas_per_sm)
{
    using namespace gbrng;
    if (kind < 0 || kind >= kKinds || fmt < 0 || fmt > 1 || size_class < 0 || size_class > 1 ||
        ctas_per_sm < 0 || ctas_per_sm > 1)
        return set_error(RNG_ERR_ARG);
    g_shape[size_class][kind][fmt].one = ctas_per_sm;
    return RNG_OK;
}

extern "C" int gbrng_get_launch_ctas(int kind, int fmt, int size_class, int *ctas_per_sm)
{
    using namespace gbrng;
    if (kind < 0 || kind >= kKinds || fmt < 0 || fmt > 1 || size_class < 0 || size_class > 1 ||
        !ctas_per_sm)
        return set_error(RNG_ERR_ARG);
    *ctas_per_sm = g_shape[size_class][kind][fmt].one;
    return RNG_OK;
}

extern "C" int gbrng_get_launch_class(int kind, int fmt, int size_class, int *v, int *block,
                                      int *hint)
{
    using namespace gbrng;
    if (kind < 0 || kind >= kKinds || fmt < 0 || fmt > 1 || size_class < 0 || size_class > 1 ||
        !v || !block || !hint)
        return set_error(RNG_ERR_ARG);
    *v = g_shape[size_class][kind][fmt].v;
    *block = g_shape[size_class][kind][fmt].block;
    *hint = g_shape[size_class][kind][fmt].hint;
    return RNG_OK;
}

extern "C" int gbrng_set_launch(int kind, int fmt, int v, int block, int hint)
{
    return gbrng_set_launch_class(kind, fmt, 1, v, block, hint);
}

extern "C" int gbrng_set_split(int kind, int log2_rows)
{
    using namespace gbrng;
    if (kind < 0 || kind >= kKinds || log2_rows < 0 || log2_rows > 30)
        return set_error(RNG_ERR_ARG);
    g_split_log2[kind] = log2_rows;
    return RNG_OK;
}

extern "C" int gbrng_get_split(int kind, int *log2_rows)
{
    using namespace gbrng;
    if (kind < 0 || kind >= kKinds || !log2_rows)
        return set_error(RNG_ERR_ARG);
    *log2_rows = g_split_log2[kind];
    return RNG_OK;
}

extern "C" int gbrng_get_launch(int kind, int fmt, int *v, int *block, int *hint)
{
    return gbrng_get_launch_class(kind, fmt, 1, v, block, hint);
}
