// Batched generation: many generators of mixed kinds, stream counts, lengths
// and formats in ONE persistent kernel launch.  Every item's streams are cut
// into tiles; a CTA takes the next tile from a device work list through an
// atomic counter and runs the same per-thread body as the plain kernels
// (gen_body.cuh), so outputs and state are bit-identical to plain launches.
// Tiles are ordered by length, largest first, so that the longest tiles start
// first and the launch ends evenly.  Nothing waits on the device: a CTA only
// increments the counter and stops when the list is exhausted.
#include <algorithm>
#include <cstring>
#include <new>
#include <unordered_set>
#include <vector>

#include "gen_body.cuh"

namespace gbrng {
namespace {

struct Unit {
    uint32_t *state;     // generator state (SoA, stride n)
    const uint32_t *a;   // multipliers or nullptr
    uint32_t *out;       // item output, row stride n
    uint64_t n;          // generator streams
    uint64_t steps;      // outputs per stream
    uint32_t s0;         // first stream of the tile
    uint32_t count;      // streams in the tile
    uint32_t code;       // kind | fmt << 2 | vec << 3
    uint32_t pad;
};

template <int KIND, int FMT, int HINT>
__device__ __forceinline__ void run_unit(const Unit &u)
{
    const uint64_t end = (uint64_t)u.s0 + u.count;
    if (u.code & 8u) {
        body_vec<KIND, FMT, 1, HINT>(u.state, u.a, u.n, u.steps, u.out, u.n,
                                     u.s0 + 4 * (uint64_t)threadIdx.x, 0, end);
    } else {
        uint64_t s = u.s0 + (uint64_t)threadIdx.x;
        if (s < end)
            body_scalar<KIND, FMT, HINT>(u.state, u.a, u.n, u.steps, u.out, u.n, s);
    }
}

template <int HINT>
__global__ void __launch_bounds__(512)
batch_kernel(const Unit *__restrict__ units, uint64_t n_units, unsigned long long *next)
{
    __shared__ unsigned long long take;
    for (;;) {
        if (threadIdx.x == 0)
            take = atomicAdd(next, 1ull);
        __syncthreads();
        const unsigned long long u = take;
        __syncthreads();
        if (u >= n_units)
            return;
        const Unit U = units[u];
        switch (U.code & 7u) {
        case RNG_MWC32 | (RNG_U32 << 2): run_unit<RNG_MWC32, RNG_U32, HINT>(U); break;
        case RNG_MWC32 | (RNG_F32 << 2): run_unit<RNG_MWC32, RNG_F32, HINT>(U); break;
        case RNG_XOR128 | (RNG_U32 << 2): run_unit<RNG_XOR128, RNG_U32, HINT>(U); break;
        case RNG_XOR128 | (RNG_F32 << 2): run_unit<RNG_XOR128, RNG_F32, HINT>(U); break;
        case RNG_KISS | (RNG_U32 << 2): run_unit<RNG_KISS, RNG_U32, HINT>(U); break;
        case RNG_KISS | (RNG_F32 << 2): run_unit<RNG_KISS, RNG_F32, HINT>(U); break;
        default: break;
        }
    }
}

struct Plan {
    int device = 0;
    Unit *d_units = nullptr;
    uint64_t n_units = 0;
    unsigned long long *d_next = nullptr;
    int threads = 128;
    int grid = 0;
};

void free_plan(Plan *p)
{
    if (!p)
        return;
    cudaFree(p->d_units);
    cudaFree(p->d_next);
    delete p;
}

}  // namespace
}  // namespace gbrng

using namespace gbrng;

extern "C" rng_plan_handle rng_plan_create(const rng_batch_item *items, size_t n_items,
                                           int threads, int ctas_per_sm)
{
    if (!items || n_items == 0) {
        set_error(RNG_ERR_ARG);
        return nullptr;
    }
    if (threads == 0)
        threads = 128;
    if (threads < 32 || threads > 512 || (threads & (threads - 1)) || ctas_per_sm < 0 ||
        ctas_per_sm > 32) {
        set_error(RNG_ERR_ARG);
        return nullptr;
    }
    int device = -1;
    std::unordered_set<const void *> seen;
    std::vector<Unit> units;
    for (size_t i = 0; i < n_items; ++i) {
        const rng_batch_item &it = items[i];
        Gen *g = reinterpret_cast<Gen *>(it.h);
        if (!g || (it.fmt != RNG_U32 && it.fmt != RNG_F32)) {
            set_error(RNG_ERR_ARG);
            return nullptr;
        }
        if (device < 0)
            device = g->device;
        if (g->device != device || !seen.insert(g).second) {
            set_error(RNG_ERR_ARG);
            return nullptr;
        }
        if (it.n_per_stream == 0)
            continue;
        if (!it.out || (uintptr_t)it.out % 4 != 0 || it.n_per_stream > UINT64_MAX / 4 / g->n) {
            set_error(RNG_ERR_ARG);
            return nullptr;
        }
        bool vec = g->n % 4 == 0 && (uintptr_t)it.out % 16 == 0;
        uint64_t tile = vec ? 4ull * threads : (uint64_t)threads;
        uint32_t code = (uint32_t)g->kind | ((uint32_t)it.fmt << 2) | (vec ? 8u : 0u);
        for (uint64_t s0 = 0; s0 < g->n; s0 += tile) {
            Unit u{};
            u.state = g->d_state;
            u.a = g->d_a;
            u.out = static_cast<uint32_t *>(it.out);
            u.n = g->n;
            u.steps = it.n_per_stream;
            u.s0 = (uint32_t)s0;
            u.count = (uint32_t)std::min<uint64_t>(tile, g->n - s0);
            u.code = code;
            units.push_back(u);
        }
    }
    if (device < 0) {
        set_error(RNG_ERR_ARG);
        return nullptr;
    }
    std::stable_sort(units.begin(), units.end(),
                     [](const Unit &x, const Unit &y) { return x.steps > y.steps; });
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != device)
        cudaSetDevice(device);
    Plan *p = new (std::nothrow) Plan();
    int st = p ? RNG_OK : set_error(RNG_ERR_OOM);
    if (!st) {
        p->device = device;
        p->threads = threads;
        p->n_units = units.size();
        int sms = 0, fit = 0;
        st = cuda_status(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
        if (!st)
            st = cuda_status(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &fit, batch_kernel<0>, threads, 0));
        if (!st) {
            int per = ctas_per_sm ? std::min(ctas_per_sm, std::max(fit, 1)) : std::max(fit, 1);
            p->grid = sms * per;
        }
    }
    if (!st && p->n_units) {
        size_t bytes = p->n_units * sizeof(Unit);
        if (cudaMalloc(&p->d_units, bytes) != cudaSuccess)
            st = set_error(RNG_ERR_OOM);
        else
            st = cuda_status(cudaMemcpy(p->d_units, units.data(), bytes, cudaMemcpyHostToDevice));
    }
    if (!st && cudaMalloc(&p->d_next, sizeof(unsigned long long)) != cudaSuccess)
        st = set_error(RNG_ERR_OOM);
    if (prev >= 0 && prev != device)
        cudaSetDevice(prev);
    if (st) {
        free_plan(p);
        return nullptr;
    }
    return reinterpret_cast<rng_plan_handle>(p);
}

extern "C" int rng_plan_launch(rng_plan_handle h, void *cuda_stream)
{
    Plan *p = reinterpret_cast<Plan *>(h);
    if (!p)
        return set_error(RNG_ERR_ARG);
    if (p->n_units == 0)
        return RNG_OK;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != p->device)
        cudaSetDevice(p->device);
    int status = cuda_status(cudaMemsetAsync(p->d_next, 0, sizeof(unsigned long long), st));
    if (!status) {
        batch_kernel<0><<<p->grid, p->threads, 0, st>>>(p->d_units, p->n_units, p->d_next);
        status = cuda_status(cudaGetLastError());
    }
    if (prev >= 0 && prev != p->device)
        cudaSetDevice(prev);
    return status;
}

extern "C" uint64_t rng_plan_tiles(rng_plan_handle h)
{
    Plan *p = reinterpret_cast<Plan *>(h);
    return p ? p->n_units : 0;
}

extern "C" int rng_plan_shape(rng_plan_handle h, int *threads, int *grid)
{
    Plan *p = reinterpret_cast<Plan *>(h);
    if (!p || !threads || !grid)
        return set_error(RNG_ERR_ARG);
    *threads = p->threads;
    *grid = p->grid;
    return RNG_OK;
}

extern "C" void rng_plan_destroy(rng_plan_handle h)
{
    Plan *p = reinterpret_cast<Plan *>(h);
    if (!p)
        return;
    const int dev = p->device;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != dev)
        cudaSetDevice(dev);
    cudaDeviceSynchronize();
    free_plan(p);
    if (prev >= 0 && prev != dev)
        cudaSetDevice(prev);
}

extern "C" int rng_generate_batch(const rng_batch_item *items, size_t n_items, void *cuda_stream)
{
    rng_plan_handle p = rng_plan_create(items, n_items, 0, 0);
    if (!p)
        return rng_last_error();
    int st = rng_plan_launch(p, cuda_stream);
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream));
    rng_plan_destroy(p);
    if (!st && e != cudaSuccess)
        st = cuda_status(e);
    return st;
}

// ------------------------------------------------------------------------
// Allocation-free batched launch.  Same work list and the same persistent
// kernel as the plan path above, but the work list and the tile counter live
// in one fixed, file-scope device array instead of memory from cudaMalloc,
// and the host side builds the list in a fixed host array, so a call makes
// no device or host heap allocation.  Some callers cannot allocate device
// memory at the point where they need random numbers: an application whose
// pool allocator owns the whole device budget, or a latency-sensitive loop
// that must not pay for (or be synchronised by) a cudaMalloc/cudaFree pair.
// The paper has no counterpart of this entry point.
// ------------------------------------------------------------------------
#include <mutex>

namespace gbrng {
namespace {

constexpr uint64_t kNoAllocMaxTiles = 32768;  // work-list capacity, in tiles
constexpr size_t kNoAllocMaxItems = 4096;     // items per call
constexpr size_t kNoAllocHeader = 256;        // tile counter, then padding
constexpr size_t kNoAllocBytes = kNoAllocHeader + kNoAllocMaxTiles * sizeof(Unit);

// The scratch: bytes [0, 8) hold the tile counter, the work list starts at
// byte kNoAllocHeader.  Every GPU that loads the library holds it until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mutex;                      // guards the host arrays below
void *g_noalloc_dev_ptr[64] = {nullptr};         // device address of the scratch
Unit g_noalloc_host_units[kNoAllocMaxTiles];     // host copy of the work list
const void *g_noalloc_handles[kNoAllocMaxItems]; // duplicate check

}  // namespace
}  // namespace gbrng

extern "C" int rng_generate_batch_noalloc(const rng_batch_item *items, size_t n_items,
                                          void *cuda_stream)
{
    if (!items || n_items == 0 || n_items > kNoAllocMaxItems)
        return set_error(RNG_ERR_ARG);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    int device = -1;
    for (size_t i = 0; i < n_items; ++i) {
        Gen *g = reinterpret_cast<Gen *>(items[i].h);
        if (!g || (items[i].fmt != RNG_U32 && items[i].fmt != RNG_F32))
            return set_error(RNG_ERR_ARG);
        if (device < 0)
            device = g->device;
        if (g->device != device || device >= 64)
            return set_error(RNG_ERR_ARG);
        g_noalloc_handles[i] = g;
    }
    std::sort(g_noalloc_handles, g_noalloc_handles + n_items);
    for (size_t i = 1; i < n_items; ++i)
        if (g_noalloc_handles[i] == g_noalloc_handles[i - 1])
            return set_error(RNG_ERR_ARG);

    // Work list, as rng_plan_create with its default CTA size builds it.
    const int threads = 128;
    uint64_t n_units = 0;
    for (size_t i = 0; i < n_items; ++i) {
        const rng_batch_item &it = items[i];
        Gen *g = reinterpret_cast<Gen *>(it.h);
        if (it.n_per_stream == 0)
            continue;
        if (!it.out || (uintptr_t)it.out % 4 != 0 || it.n_per_stream > UINT64_MAX / 4 / g->n)
            return set_error(RNG_ERR_ARG);
        bool vec = g->n % 4 == 0 && (uintptr_t)it.out % 16 == 0;
        uint64_t tile = vec ? 4ull * threads : (uint64_t)threads;
        uint64_t tiles = (g->n + tile - 1) / tile;
        if (n_units + tiles > kNoAllocMaxTiles)
            return set_error(RNG_ERR_ARG);  // beyond the work-list capacity
        uint32_t code = (uint32_t)g->kind | ((uint32_t)it.fmt << 2) | (vec ? 8u : 0u);
        for (uint64_t s0 = 0; s0 < g->n; s0 += tile) {
            Unit &u = g_noalloc_host_units[n_units++];
            u = Unit{};
            u.state = g->d_state;
            u.a = g->d_a;
            u.out = static_cast<uint32_t *>(it.out);
            u.n = g->n;
            u.steps = it.n_per_stream;
            u.s0 = (uint32_t)s0;
            u.count = (uint32_t)std::min<uint64_t>(tile, g->n - s0);
            u.code = code;
        }
    }
    if (n_units == 0)
        return RNG_OK;
    // Longest tiles first; ties ordered by generator and first stream (an
    // in-place sort, no buffer; the order only affects scheduling).
    std::sort(g_noalloc_host_units, g_noalloc_host_units + n_units,
              [](const Unit &x, const Unit &y) {
                  if (x.steps != y.steps)
                      return x.steps > y.steps;
                  if (x.state != y.state)
                      return x.state < y.state;
                  return x.s0 < y.s0;
              });

    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess)
        return set_error(RNG_ERR_CUDA);
    if (prev != device && cudaSetDevice(device) != cudaSuccess)
        return set_error(RNG_ERR_CUDA);
    int st = RNG_OK;
    // Set-up, once per device with that device current: the device address
    // of the scratch array (its name in host code is only a host stand-in).
    if (!g_noalloc_dev_ptr[device]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr)
            st = cuda_status(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
        else
            g_noalloc_dev_ptr[device] = ptr;
    }
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    int sms = 0, fit = 0;
    if (!st)
        st = cuda_status(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    if (!st)
        st = cuda_status(
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, batch_kernel<0>, threads, 0));
    unsigned char *base = static_cast<unsigned char *>(g_noalloc_dev_ptr[device]);
    unsigned long long *next = reinterpret_cast<unsigned long long *>(base);
    Unit *units = reinterpret_cast<Unit *>(base + kNoAllocHeader);
    // The copy is from pageable memory: it is staged before the call returns,
    // so the host array may be reused by the next call.
    if (!st)
        st = cuda_status(cudaMemcpyAsync(units, g_noalloc_host_units, n_units * sizeof(Unit),
                                         cudaMemcpyHostToDevice, stream));
    if (!st)  // the counter keeps the last call's value: clear it
        st = cuda_status(cudaMemsetAsync(next, 0, sizeof(unsigned long long), stream));
    if (!st) {
        batch_kernel<0><<<sms * std::max(fit, 1), threads, 0, stream>>>(units, n_units, next);
        st = cuda_status(cudaGetLastError());
    }
    if (prev >= 0 && prev != device)
        cudaSetDevice(prev);
    return st;
}
