// C-ABI of the generator library: handles, the hot-path call, host delivery
// and state checkpoints.  See include/rng.h for the contract of each call.
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "gbrng.cuh"

namespace gbrng {

namespace {
thread_local int t_last_error = RNG_OK;

// Makes the handle's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            ok = false;
            return;
        }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess)
            ok = false;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev)
            cudaSetDevice(prev);
    }
};

bool device_supported(int dev)
{
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
        return false;
    return prop.major == 10 && prop.minor == 3;
}

bool valid_kind(int k) { return k >= 0 && k < kKinds; }
bool valid_fmt(int f) { return f == RNG_U32 || f == RNG_F32; }

uint64_t max_streams(int kind)
{
    switch (kind) {
    case RNG_XOR128: return RNG_MAX_STREAMS_XOR;
    case RNG_MWC16X2:
    case RNG_KISS_XOR: return RNG_MAX_STREAMS_MWC16;
    case RNG_XORSHIFT8: return RNG_MAX_STREAMS_XS8;
    default: return RNG_MAX_STREAMS_MWC;
    }
}

void free_gen(Gen *g)
{
    if (!g)
        return;
    cudaFree(g->d_state);
    cudaFree(g->d_a);
    cudaFree(g->d_split);
    cudaFree(g->d_cnt);
    cudaFree(g->d_jmul);
    for (int i = 0; i < 2; ++i) {
        cudaFree(g->d_stage[i]);
        if (g->stage_ev[i])
            cudaEventDestroy(g->stage_ev[i]);
    }
    delete g;
}

}  // namespace

int set_error(int status)
{
    if (status != RNG_OK)
        t_last_error = status;
    return status;
}

int cuda_status(cudaError_t e)
{
    if (e == cudaSuccess)
        return RNG_OK;
    if (e == cudaErrorMemoryAllocation)
        return set_error(RNG_ERR_OOM);
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver ||
        e == cudaErrorNoKernelImageForDevice)
        return set_error(RNG_ERR_NODEV);
    return set_error(RNG_ERR_CUDA);
}

}  // namespace gbrng

using namespace gbrng;

namespace gbrng {
namespace {

// Streams s_begin .. s_begin + n_streams of the generator (kind, seed): the
// handle's stream s is global stream s_begin + s, with that stream's
// multiplier and splitmix64 started at seed + s_begin + s.
rng_handle create_range(int kind, uint64_t s_begin, uint64_t n_streams, uint64_t seed)
{
    if (!valid_kind(kind) || n_streams == 0 || s_begin > max_streams(kind) ||
        n_streams > max_streams(kind) - s_begin) {
        set_error(RNG_ERR_ARG);
        return nullptr;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || !device_supported(dev)) {
        set_error(RNG_ERR_NODEV);
        return nullptr;
    }
    Gen *g = new (std::nothrow) Gen();
    if (!g) {
        set_error(RNG_ERR_OOM);
        return nullptr;
    }
    g->kind = kind;
    g->device = dev;
    g->n = n_streams;
    g->seed = seed + s_begin;
    g->words = words_of(kind);
    int st = RNG_OK;
    if (cudaMalloc(&g->d_state, (size_t)g->words * n_streams * 4) != cudaSuccess) {
        st = set_error(RNG_ERR_OOM);
    } else if (has_mult(kind)) {
        // one multiplier per stream, or one packed pair for the base-2^16 kinds
        const uint32_t *table = nullptr;
        const uint64_t need = s_begin + n_streams;
        st = kind == RNG_MWC16X2 || kind == RNG_KISS_XOR ? mwc16_pair_table(need, &table)
                                                         : multiplier_table(need, &table);
        if (!st && cudaMalloc(&g->d_a, n_streams * 4) != cudaSuccess)
            st = set_error(RNG_ERR_OOM);
        if (!st)
            st = cuda_status(cudaMemcpy(g->d_a, table + s_begin, n_streams * 4,
                                        cudaMemcpyDeviceToDevice));
    }
    // buffers of split calls (few streams only): the final-state stash, the
    // arrival counters (zero) and the MWC jump multipliers
    if (!st && n_streams <= kSplitMaxStreams) {
        g->jmul_segs = split_max_segments(n_streams);
        if (cudaMalloc(&g->d_split, (size_t)g->words * n_streams * 4) != cudaSuccess ||
            cudaMalloc(&g->d_cnt, n_streams * 4) != cudaSuccess)
            st = set_error(RNG_ERR_OOM);
        else
            st = cuda_status(cudaMemset(g->d_cnt, 0, n_streams * 4));
    }
    // jump tables of the xorshift and LCG parts, built here so that no later
    // call (which may be captured in a CUDA graph) has to build them
    JumpTables tables;
    if (!st && needs_jump_tables(kind))
        st = jump_tables(&tables);
    if (!st)
        st = launch_seed(g, nullptr);
    if (!st)
        st = cuda_status(cudaStreamSynchronize(nullptr));
    if (st) {
        free_gen(g);
        return nullptr;
    }
    return reinterpret_cast<rng_handle>(g);
}

}  // namespace
}  // namespace gbrng

extern "C" rng_handle rng_create(int kind, uint64_t n_streams, uint64_t seed)
{
    return create_range(kind, 0, n_streams, seed);
}

extern "C" rng_handle rng_create_range(int kind, uint64_t s_begin, uint64_t n_streams,
                                       uint64_t seed)
{
    return create_range(kind, s_begin, n_streams, seed);
}

extern "C" void rng_destroy(rng_handle h)
{
    Gen *g = reinterpret_cast<Gen *>(h);
    if (!g)
        return;
    DeviceGuard dg(g->device);
    cudaStreamSynchronize(g->stream);
    free_gen(g);
}

extern "C" int rng_set_stream(rng_handle h, void *cuda_stream)
{
    Gen *g = reinterpret_cast<Gen *>(h);
    if (!g)
        return set_error(RNG_ERR_ARG);
    g->stream = static_cast<cudaStream_t>(cuda_stream);
    return RNG_OK;
}

extern "C" uint64_t rng_n_streams(rng_handle h)
{
    Gen *g = reinterpret_cast<Gen *>(h);
    return g ? g->n : 0;
}

extern "C" int rng_state_words(rng_handle h)
{
    Gen *g = reinterpret_cast<Gen *>(h);
    return g ? g->words : 0;
}

extern "C" int rng_generate(rng_handle h, uint64_t n_per_stream, void *out, int fmt)
{
    Gen *g = reinterpret_cast<Gen *>(h);
    if (!g || !valid_fmt(fmt))
        return set_error(RNG_ERR_ARG);
    if (n_per_stream == 0)
        return RNG_OK;
    if (!out || (uintptr_t)out % 4 != 0)
        return set_error(RNG_ERR_ARG);
    if (n_per_stream > UINT64_MAX / 4 / g->n)
        return set_error(RNG_ERR_ARG);
    DeviceGuard dg(g->device);
    if (!dg.ok)
        return set_error(RNG_ERR_CUDA);
    GenLaunch p{g->d_state, g->d_a, g->n, 0, g->n, n_per_stream, out, g->n, g};
    return launch_generate(g->kind, fmt, p, g->stream);
}

extern "C" int rng_generate_range(rng_handle h, uint64_t s_begin, uint64_t s_end,
                                  uint64_t n_per_stream, void *out, uint64_t ld, int fmt)
{
    Gen *g = reinterpret_cast<Gen *>(h);
    if (!g || !valid_fmt(fmt) || s_begin >= s_end || s_end > g->n)
        return set_error(RNG_ERR_ARG);
    if (n_per_stream == 0)
        return RNG_OK;
    const uint64_t count = s_end - s_begin;
    if (!out || (uintptr_t)out % 4 != 0 || ld < count ||
        (n_per_stream - 1) > (UINT64_MAX / 4 - count) / ld)
        return set_error(RNG_ERR_ARG);
    DeviceGuard dg(g->device);
    if (!dg.ok)
        return set_error(RNG_ERR_CUDA);
    GenLaunch p{g->d_state, g->d_a, g->n, s_begin, s_end, n_per_stream, out, ld, g};
    return launch_generate(g->kind, fmt, p, g->stream);
}

extern "C" int rng_generate_host(rng_handle h, uint64_t n_per_stream, void *host_out, int fmt)
{
    Gen *g = reinterpret_cast<Gen *>(h);
    if (!g || !valid_fmt(fmt))
        return set_error(RNG_ERR_ARG);
    if (n_per_stream == 0)
        return RNG_OK;
    if (!host_out || n_per_stream > UINT64_MAX / 4 / g->n)
        return set_error(RNG_ERR_ARG);
    DeviceGuard dg(g->device);
    if (!dg.ok)
        return set_error(RNG_ERR_CUDA);
    const size_t row_bytes = g->n * 4;
    const size_t target = (size_t)256 << 20;  // staging: two buffers of up to 256 MiB
    uint64_t rows = target / row_bytes;
    if (rows == 0)
        rows = 1;
    if (rows > n_per_stream)
        rows = n_per_stream;
    size_t need = rows * row_bytes;
    if (g->stage_bytes < need) {
        for (int i = 0; i < 2; ++i) {
            cudaFree(g->d_stage[i]);
            g->d_stage[i] = nullptr;
        }
        g->stage_bytes = 0;
        for (int i = 0; i < 2; ++i)
            if (cudaMalloc(&g->d_stage[i], need) != cudaSuccess)
                return set_error(RNG_ERR_OOM);
        g->stage_bytes = need;
        for (int i = 0; i < 2; ++i)
            if (!g->stage_ev[i] &&
                cudaEventCreateWithFlags(&g->stage_ev[i], cudaEventDisableTiming) != cudaSuccess)
                return set_error(RNG_ERR_CUDA);
    }
    cudaStream_t copy = nullptr;
    if (cudaStreamCreateWithFlags(&copy, cudaStreamNonBlocking) != cudaSuccess)
        return set_error(RNG_ERR_CUDA);
    cudaEvent_t gen_done[2] = {nullptr, nullptr};
    int st = RNG_OK;
    for (int i = 0; i < 2 && !st; ++i)
        if (cudaEventCreateWithFlags(&gen_done[i], cudaEventDisableTiming) != cudaSuccess)
            st = set_error(RNG_ERR_CUDA);
    char *dst = static_cast<char *>(host_out);
    uint64_t chunk = 0;
    for (uint64_t j0 = 0; j0 < n_per_stream && !st; j0 += rows, ++chunk) {
        int b = (int)(chunk & 1);
        uint64_t m = n_per_stream - j0 < rows ? n_per_stream - j0 : rows;
        // buffer b is free once its previous copy (chunk - 2) has finished
        if (chunk >= 2)
            st = cuda_status(cudaStreamWaitEvent(g->stream, g->stage_ev[b], 0));
        GenLaunch p{g->d_state, g->d_a, g->n, 0, g->n, m, g->d_stage[b], g->n, g};
        if (!st)
            st = launch_generate(g->kind, fmt, p, g->stream);
        if (!st)
            st = cuda_status(cudaEventRecord(gen_done[b], g->stream));
        if (!st)
            st = cuda_status(cudaStreamWaitEvent(copy, gen_done[b], 0));
        if (!st)
            st = cuda_status(cudaMemcpyAsync(dst + j0 * row_bytes, g->d_stage[b], m * row_bytes,
                                             cudaMemcpyDeviceToHost, copy));
        if (!st)
            st = cuda_status(cudaEventRecord(g->stage_ev[b], copy));
    }
    cudaError_t e1 = cudaStreamSynchronize(copy);
    cudaError_t e2 = cudaStreamSynchronize(g->stream);
    for (int i = 0; i < 2; ++i)
        if (gen_done[i])
            cudaEventDestroy(gen_done[i]);
    cudaStreamDestroy(copy);
    if (!st && e1 != cudaSuccess)
        st = cuda_status(e1);
    if (!st && e2 != cudaSuccess)
        st = cuda_status(e2);
    return st;
}

extern "C" int rng_jump(rng_handle h, uint64_t k)
{
    Gen *g = reinterpret_cast<Gen *>(h);
    if (!g)
        return set_error(RNG_ERR_ARG);
    DeviceGuard dg(g->device);
    if (!dg.ok)
        return set_error(RNG_ERR_CUDA);
    return launch_jump(g, k, g->stream);
}

extern "C" int rng_get_device_view(rng_handle h, rng_device_view *view)
{
    Gen *g = reinterpret_cast<Gen *>(h);
    if (!g || !view)
        return set_error(RNG_ERR_ARG);
    *view = rng_device_view{g->kind, g->device, g->words, g->n, g->d_state, g->d_a};
    return RNG_OK;
}

extern "C" int rng_get_state(rng_handle h, void *host_buf, size_t bytes)
{
    Gen *g = reinterpret_cast<Gen *>(h);
    if (!g || !host_buf || bytes != (size_t)g->words * g->n * 4)
        return set_error(RNG_ERR_ARG);
    DeviceGuard dg(g->device);
    int st = cuda_status(cudaStreamSynchronize(g->stream));
    if (!st)
        st = cuda_status(cudaMemcpy(host_buf, g->d_state, bytes, cudaMemcpyDeviceToHost));
    return st;
}

extern "C" int rng_set_state(rng_handle h, const void *host_buf, size_t bytes)
{
    Gen *g = reinterpret_cast<Gen *>(h);
    if (!g || !host_buf || bytes != (size_t)g->words * g->n * 4)
        return set_error(RNG_ERR_ARG);
    DeviceGuard dg(g->device);
    const uint32_t *w = static_cast<const uint32_t *>(host_buf);
    const uint64_t n = g->n;
    if (g->kind == RNG_XOR128 || g->kind == RNG_XORSHIFT8) {
        for (uint64_t s = 0; s < n; ++s) {
            uint32_t any = 0;
            for (int k = 0; k < g->words; ++k)
                any |= w[k * n + s];
            if (any == 0)
                return set_error(RNG_ERR_ARG);
        }
    } else if (g->kind == RNG_MWC16X2 || g->kind == RNG_KISS_XOR) {
        std::vector<uint32_t> a(n);
        int st = cuda_status(cudaMemcpy(a.data(), g->d_a, n * 4, cudaMemcpyDeviceToHost));
        if (st)
            return st;
        for (uint64_t s = 0; s < n; ++s) {
            for (int part = 0; part < 2; ++part) {
                const uint32_t ap = part ? a[s] >> 16 : a[s] & 0xFFFFu;
                const uint32_t z = w[part * n + s], x = z & 0xFFFFu, c = z >> 16;
                if (c >= ap || (x == 0 && c == 0) || (x == 0xFFFFu && c == ap - 1))
                    return set_error(RNG_ERR_ARG);
            }
            if (g->kind == RNG_KISS_XOR && w[2 * n + s] == 0)
                return set_error(RNG_ERR_ARG);
        }
    } else {
        std::vector<uint32_t> a(n);
        int st = cuda_status(cudaMemcpy(a.data(), g->d_a, n * 4, cudaMemcpyDeviceToHost));
        if (st)
            return st;
        for (uint64_t s = 0; s < n; ++s) {
            uint32_t x = w[s], c = w[n + s];
            if (c >= a[s] || (x == 0 && c == 0) || (x == 0xFFFFFFFFu && c == a[s] - 1))
                return set_error(RNG_ERR_ARG);
            if (g->kind == RNG_KISS && w[2 * n + s] == 0)
                return set_error(RNG_ERR_ARG);
        }
    }
    int st = cuda_status(cudaStreamSynchronize(g->stream));
    if (!st)
        st = cuda_status(cudaMemcpy(g->d_state, host_buf, bytes, cudaMemcpyHostToDevice));
    return st;
}

extern "C" int rng_last_error(void) { return t_last_error; }

extern "C" const char *rng_strerror(int status)
{
    switch (status) {
    case RNG_OK: return "ok";
    case RNG_ERR_ARG: return "invalid argument";
    case RNG_ERR_OOM: return "out of memory";
    case RNG_ERR_CUDA: return "CUDA error";
    case RNG_ERR_TIMEOUT: return "device-side wait timed out";
    case RNG_ERR_BUSY: return "over the admission budget";
    case RNG_ERR_NODEV: return "no supported CUDA device (sm_103)";
    default: return "unknown status";
    }
}
