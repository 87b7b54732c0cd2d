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
