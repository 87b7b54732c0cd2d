// Batched generation: many generators of mixed kinds, stream counts, lengths
// and formats in ONE persistent kernel launch.  Every item's streams are cut
// into tiles; a CTA takes the next tile from a device work list through an
// atomic counter and runs the same per-thread bodies as the plain kernels
// (gen_body.cuh), so outputs and state are bit-identical to plain launches.
// Tiles are ordered by length, largest first, so that the longest tiles start
// first and the launch ends evenly.  Nothing waits on the device: a CTA only
// increments the counter and stops when the list is exhausted.
//
// Tiles of an item with n streams and output `out`:
//   aligned  (n % 4 == 0, out 16-byte aligned): 4*threads streams per tile,
//            with row barriers unless every row is 32-byte aligned;
//   shifted  (otherwise) the first n & ~3 streams, 4*(31*threads/32 + 1)
//            per tile, rows realigned by warp shuffles;
//   tail     the last n % 4 streams, one stream per thread: run by the last
//            warp of the item's last realigned tile when that warp holds no
//            group (most items), else as a tile of its own.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "gen_body.cuh"

namespace gbrng {
namespace {

enum TileMode : uint32_t { kTail = 0, kAligned = 1, kShifted = 2, kAlignedSync = 3 };

struct Unit {
    uint32_t *state;       // generator state (SoA, stride n)
    const uint32_t *a;     // multipliers or nullptr
    uint32_t *out;         // output element of stream s0 in row 0
    const uint32_t *fmap;  // mapped tiles: the output map (gen_body.cuh OutMap), else nullptr
    uint64_t ld;           // output row stride
    uint32_t n;            // generator streams (state stride; at most 2^30)
    uint32_t steps;        // outputs per stream
    uint32_t s0;           // first stream of the tile
    uint32_t count;        // streams in the tile
    uint32_t code;         // kind | fmt << 2 | mode << 3 (fmt unused in mixed tiles)
    uint32_t tail;         // shifted tiles: tail streams after the tile's (0-3)
};
static_assert(sizeof(Unit) == 64, "a tile is one 64-byte record");

// The scalar body with body_shift's barriers (one after the state loads,
// then one every SYNC_ROWS rows of the blocks of four), so that one warp of a
// realigned CTA can run the n % 4 tail streams beside the other warps'
// groups: the tail's words share DRAM sectors with the CTA's last chunk and
// reach L2 with it.  Threads that are not `live` step zero state and store
// nothing; every thread of the warp must call this.
template <int KIND, int FMT, int HINT>
__device__ __forceinline__ void body_scalar_sync(uint32_t *__restrict__ state,
                                                 const uint32_t *__restrict__ mult, uint64_t n,
                                                 uint32_t steps, uint32_t *__restrict__ p0,
                                                 uint64_t ld, uint64_t s, bool live,
                                                 const uint32_t *fmap = nullptr)
{
    constexpr int W = KindTraits<KIND>::W;
    uint32_t w[kMaxWords][4] = {};
    uint32_t a[4] = {0, 0, 0, 0};
    OutMap m;
    if constexpr (FMT == kFmtMixed)
        m.load(fmap);
    if (live) {
#pragma unroll
        for (int k = 0; k < W; ++k)
            w[k][0] = state[k * n + s];
        if constexpr (KindTraits<KIND>::MULT)
            a[0] = mult[s];
    }
    __syncthreads();  // body_shift's barrier after its state loads
    constexpr uint32_t every = KindTraits<KIND>::SYNC_ROWS / 4;
    const uint32_t blocks = steps / 4;
    uint32_t *p = p0;
    if constexpr (FMT == kFmtMixed) {  // rolled: the mapped kernels stay small
        for (uint32_t j = 0; j < steps; ++j) {
            if (j % (4 * every) == 0 && j < 4 * blocks)
                __syncthreads();
            const uint32_t o = step_enc<KIND, FMT>(w, a, 0);
            if (live)
                put4<FMT, HINT>(m, m.row(p), p, o);
            p += ld;
        }
    } else {
        for (uint32_t b = 0; b < blocks; ++b) {
            if (b % every == 0)
                __syncthreads();
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t o = step_enc<KIND, FMT>(w, a, 0);
                if (live)
                    store4<HINT>(p, o);
                p += ld;
            }
        }
        for (uint32_t j = 4 * blocks; j < steps; ++j) {
            const uint32_t o = step_enc<KIND, FMT>(w, a, 0);
            if (live)
                store4<HINT>(p, o);
            p += ld;
        }
    }
    if (live) {
#pragma unroll
        for (int k = 0; k < W; ++k)
            state[k * n + s] = w[k][0];
    }
}

template <int KIND, int FMT, int HINT>
__device__ __forceinline__ void run_unit(const Unit &u)
{
    const uint32_t mode = u.code >> 3;
    const uint32_t steps = u.steps;
    const uint64_t c_first = 4 * (uint64_t)threadIdx.x;
    if (mode == kAligned) {
        if (c_first < u.count)
            body_vec<KIND, FMT, 1, HINT>(u.state, u.a, u.n, steps, u.out + c_first, u.ld,
                                         u.s0 + c_first, 0, u.fmap);
    } else if (mode == kAlignedSync) {
        body_vec_sync<KIND, FMT, HINT>(u.state, u.a, u.n, steps, u.out + c_first, u.ld,
                                       u.s0 + c_first, c_first < u.count, u.fmap);
    } else if (mode == kShifted) {
        // tail streams u.s0 + count .. + tail: the last warp, which then
        // holds no group (fill_units checks), with the same barriers
        const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (u.tail && warp == (blockDim.x >> 5) - 1)
            body_scalar_sync<KIND, FMT, HINT>(u.state, u.a, u.n, steps,
                                              u.out + u.count + lane, u.ld,
                                              u.s0 + u.count + lane, lane < u.tail, u.fmap);
        else
            body_shift<KIND, FMT, HINT>(u.state, u.a, u.n, steps, u.out, u.ld, u.s0,
                                        u.count / 4, u.fmap);
    } else {
        const uint64_t c = threadIdx.x;
        if (c < u.count)
            body_scalar<KIND, FMT, HINT>(u.state, u.a, u.n, steps, u.out + c, u.ld, u.s0 + c,
                                         u.fmap);
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

// The persistent kernel of plans whose tiles carry output maps (the serving
// engine's): the same bodies, with the place and format of every output
// taken from its tile's map.  One kernel per kind (a plan of mapped tiles
// holds one kind), so that each stays small enough for the instruction
// cache and the plain batched kernel keeps its register count.
template <int KIND, int HINT>
__global__ void __launch_bounds__(512)
batch_kernel_mixed(const Unit *__restrict__ units, uint64_t n_units, unsigned long long *next)
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
        run_unit<KIND, kFmtMixed, HINT>(U);
    }
}

// Launches the mapped-tile kernel of `kind`; one_per_sm: reserve the shared
// memory that keeps the grid to one CTA per SM.
void launch_mixed(int kind, int grid, int threads, bool one_per_sm, cudaStream_t st,
                  const Unit *units, uint64_t n_units, unsigned long long *next)
{
    auto fn = kind == RNG_MWC32    ? batch_kernel_mixed<RNG_MWC32, 1>
              : kind == RNG_XOR128 ? batch_kernel_mixed<RNG_XOR128, 1>
                                   : batch_kernel_mixed<RNG_KISS, 1>;
    const int smem = one_per_sm ? one_cta_smem((const void *)fn, threads) : 0;
    fn<<<grid, threads, smem, st>>>(units, n_units, next);
}

// Plan shape when the caller passes 0 for both: CTAs of 512 threads, one per
// SM.  Measured on GB300 with the 10,000-instance workload (256-row pieces):
// 914 GSamples/s with 128 threads (as many CTAs as fit), about 1570 with 512
// (two per SM); then, on one box, 1605 with two CTAs of 512 per SM, 1641
// with one (1632 with the grid alone keeping to one, without the
// shared-memory reservation), 1504 with two of 256.  Serving, saturating:
// 1631 with two, 1664 with one.
constexpr int kDefaultThreads = 512;
constexpr int kDefaultCtas = 1;
constexpr int kHint = 1;  // streaming stores, as the plain kernels

// An item's stream range and row stride with the defaults filled in.
struct ItemRange {
    uint64_t s_begin, s_end, ld;
};

ItemRange range_of(const rng_batch_item &it, const Gen *g)
{
    ItemRange r{it.s_begin, it.s_end ? it.s_end : g->n, it.ld ? it.ld : g->n};
    return r;
}

// A handle and stream range, for the overlap check.
struct Claim {
    const void *h;
    uint64_t s_begin, s_end;
};

// Checks every item, and that items of the same handle cover disjoint
// stream ranges; `scratch` has room for n_items claims.  Sets *device to the
// items' device.
int validate_items(const rng_batch_item *items, size_t n_items, Claim *scratch, int *device)
{
    *device = -1;
    for (size_t i = 0; i < n_items; ++i) {
        const rng_batch_item &it = items[i];
        Gen *g = reinterpret_cast<Gen *>(it.h);
        if (!g || (it.fmt != RNG_U32 && it.fmt != RNG_F32) ||
            (g->kind != RNG_MWC32 && g->kind != RNG_XOR128 && g->kind != RNG_KISS))
            return set_error(RNG_ERR_ARG);
        if (*device < 0)
            *device = g->device;
        if (g->device != *device)
            return set_error(RNG_ERR_ARG);
        const ItemRange r = range_of(it, g);
        if (r.s_begin >= r.s_end || r.s_end > g->n || r.ld < r.s_end - r.s_begin)
            return set_error(RNG_ERR_ARG);
        if (it.n_per_stream) {
            const uint64_t count = r.s_end - r.s_begin;
            if (!it.out || (uintptr_t)it.out % 4 != 0 || it.n_per_stream >= (1ull << 32) ||
                (it.n_per_stream - 1) > (UINT64_MAX / 4 - count) / r.ld)
                return set_error(RNG_ERR_ARG);
        }
        scratch[i] = Claim{g, r.s_begin, r.s_end};
    }
    std::sort(scratch, scratch + n_items, [](const Claim &x, const Claim &y) {
        return x.h != y.h ? x.h < y.h : x.s_begin < y.s_begin;
    });
    for (size_t i = 1; i < n_items; ++i)
        if (scratch[i].h == scratch[i - 1].h && scratch[i].s_begin < scratch[i - 1].s_end)
            return set_error(RNG_ERR_ARG);
    return *device < 0 ? set_error(RNG_ERR_ARG) : RNG_OK;
}

// Writes the tiles of every item to out[0 .. cap) (out may be null) and
// returns how many there are.  maps (optional): item i's output format map
// (a device pointer), given to each of its tiles.
uint64_t fill_units(const rng_batch_item *items, size_t n_items, int threads, Unit *out,
                    uint64_t cap, const uint32_t *const *maps = nullptr)
{
    uint64_t count = 0;
    for (size_t i = 0; i < n_items; ++i) {
        const rng_batch_item &it = items[i];
        Gen *g = reinterpret_cast<Gen *>(it.h);
        if (it.n_per_stream == 0)
            continue;
        const ItemRange r = range_of(it, g);
        const uint64_t n_item = r.s_end - r.s_begin;
        uint32_t *base = static_cast<uint32_t *>(it.out);
        const bool aligned = n_item % 4 == 0 && r.ld % 4 == 0 && (uintptr_t)base % 16 == 0 &&
                             g->n % 4 == 0 && r.s_begin % 4 == 0;
        const bool sectors = aligned && r.ld % 8 == 0 && (uintptr_t)base % 32 == 0;
        const uint32_t amode = sectors ? kAligned : kAlignedSync;
        const uint64_t main = n_item & ~(uint64_t)3;
        // aligned tiles: 4 streams per thread; realigned tiles: 31K + 1
        // groups of four for K warps (one halo lane per warp but the last)
        const uint64_t tile = aligned ? 4ull * threads : 4ull * (31 * (threads / 32) + 1);
        auto put = [&](uint64_t c0, uint64_t c, uint32_t mode) {
            if (out && count < cap) {
                Unit &u = out[count];
                u = Unit{};
                u.state = g->d_state;
                u.a = g->d_a;
                u.out = base + c0;
                u.n = (uint32_t)g->n;
                u.ld = r.ld;
                u.steps = (uint32_t)it.n_per_stream;
                u.fmap = maps ? maps[i] : nullptr;
                u.s0 = (uint32_t)(r.s_begin + c0);
                u.count = (uint32_t)c;
                u.code = (uint32_t)g->kind | ((uint32_t)it.fmt << 2) | (mode << 3);
            }
            ++count;
        };
        for (uint64_t c0 = 0; c0 < main; c0 += tile)
            put(c0, std::min<uint64_t>(tile, main - c0), aligned ? amode : kShifted);
        // the tail joins the last realigned tile when that tile's last warp
        // holds no group (at most 31 (K - 1) groups: warp K - 2's halo lane
        // then holds no live group either)
        const uint64_t last = main % tile ? main % tile : tile;
        const bool join = !aligned && main > 0 && main < n_item &&
                          last / 4 <= 31ull * (threads / 32 - 1);
        if (join) {
            if (out && count - 1 < cap)
                out[count - 1].tail = (uint32_t)(n_item - main);
        } else if (main < n_item) {
            put(main, n_item - main, kTail);
        }
    }
    return count;
}

// Longest tiles first; ties by generator and first stream, so the order is
// deterministic (it only affects scheduling).
void order_units(Unit *u, uint64_t n)
{
    std::sort(u, u + n, [](const Unit &x, const Unit &y) {
        if (x.steps != y.steps)
            return x.steps > y.steps;
        if (x.state != y.state)
            return x.state < y.state;
        return x.s0 != y.s0 ? x.s0 < y.s0 : x.out < y.out;
    });
}

int grid_for(int device, int threads, int ctas_per_sm, int *grid, bool mixed = false)
{
    int sms = 0, fit = 0;
    int st = cuda_status(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    if (!st)
        st = cuda_status(mixed ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                     &fit, batch_kernel_mixed<RNG_KISS, kHint>, threads, 0)
                               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                     &fit, batch_kernel<kHint>, threads, 0));
    if (!st) {
        fit = std::max(fit, 1);
        *grid = sms * (ctas_per_sm ? std::min(ctas_per_sm, fit) : fit);
    }
    return st;
}

struct Plan {
    int device = 0;
    Unit *d_units = nullptr;
    uint64_t n_units = 0;
    uint64_t cap_units = 0;          // device work-list capacity
    unsigned long long *d_next = nullptr;
    int threads = kDefaultThreads;
    int grid = 0;
    std::vector<Claim> claims;       // refill overlap check
    // refill staging: two pinned host lists used in turn, so that the copy
    // to the device is a plain DMA and the call does not wait for it; a
    // refill reuses a list after the copy out of it (two refills earlier)
    // has finished (its event)
    Unit *pinned[2] = {nullptr, nullptr};
    uint64_t pinned_cap[2] = {0, 0};
    cudaEvent_t copied[2] = {nullptr, nullptr};
    int turn = 0;
    // output format maps of mixed tiles (plan_refill_mixed): device copy and
    // two pinned host lists used in turn with the tile lists
    bool mixed = false;  // the current tiles carry maps: batch_kernel_mixed runs them
    int mixed_kind = 0;  // their kind (one per mapped refill)
    int ctas_per_sm = 0;
    int grid_mixed = 0;
    uint32_t *d_maps = nullptr;
    uint64_t cap_maps = 0;  // words
    uint32_t *pinned_maps[2] = {nullptr, nullptr};
    uint64_t pinned_maps_cap[2] = {0, 0};
};

void free_plan(Plan *p)
{
    if (!p)
        return;
    for (int k = 0; k < 2; ++k) {
        if (p->copied[k]) {
            cudaEventSynchronize(p->copied[k]);
            cudaEventDestroy(p->copied[k]);
        }
        cudaFreeHost(p->pinned[k]);
        cudaFreeHost(p->pinned_maps[k]);
    }
    cudaFree(p->d_units);
    cudaFree(p->d_next);
    cudaFree(p->d_maps);
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
    if (threads == 0 && ctas_per_sm == 0)
        ctas_per_sm = kDefaultCtas;
    if (threads == 0)
        threads = kDefaultThreads;
    if (threads < 32 || threads > 512 || (threads & (threads - 1)) || ctas_per_sm < 0 ||
        ctas_per_sm > 32) {
        set_error(RNG_ERR_ARG);
        return nullptr;
    }
    int device = -1;
    std::vector<Claim> claims(n_items);
    if (validate_items(items, n_items, claims.data(), &device))
        return nullptr;
    std::vector<Unit> units(fill_units(items, n_items, threads, nullptr, 0));
    fill_units(items, n_items, threads, units.data(), units.size());
    order_units(units.data(), units.size());

    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != device)
        cudaSetDevice(device);
    Plan *p = new (std::nothrow) Plan();
    int st = p ? RNG_OK : set_error(RNG_ERR_OOM);
    if (!st) {
        p->device = device;
        p->threads = threads;
        p->ctas_per_sm = ctas_per_sm;
        p->n_units = units.size();
        st = grid_for(device, threads, ctas_per_sm, &p->grid);
    }
    if (!st && p->n_units) {
        size_t bytes = p->n_units * sizeof(Unit);
        if (cudaMalloc(&p->d_units, bytes) != cudaSuccess)
            st = set_error(RNG_ERR_OOM);
        else
            st = cuda_status(cudaMemcpy(p->d_units, units.data(), bytes, cudaMemcpyHostToDevice));
        p->cap_units = p->n_units;
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
        const bool one = p->ctas_per_sm == 1;
        if (p->mixed) {
            launch_mixed(p->mixed_kind, p->grid_mixed, p->threads, one, st, p->d_units,
                         p->n_units, p->d_next);
        } else {
            const int smem = one ? one_cta_smem((const void *)batch_kernel<kHint>, p->threads)
                                 : 0;
            batch_kernel<kHint><<<p->grid, p->threads, smem, st>>>(p->d_units, p->n_units,
                                                                  p->d_next);
        }
        status = cuda_status(cudaGetLastError());
    }
    if (prev >= 0 && prev != p->device)
        cudaSetDevice(prev);
    return status;
}

namespace gbrng {
namespace {

// Grows a pinned host list to at least `need` elements (keeps no contents).
template <class T>
int ensure_pinned(T **buf, uint64_t *cap, uint64_t need, uint64_t other_cap)
{
    if (need <= *cap)
        return RNG_OK;
    cudaFreeHost(*buf);
    *buf = nullptr;
    *cap = 0;
    const uint64_t want = std::max<uint64_t>(need, 2 * other_cap);
    if (cudaHostAlloc(reinterpret_cast<void **>(buf), want * sizeof(T), cudaHostAllocDefault) !=
        cudaSuccess)
        return set_error(RNG_ERR_OOM);
    *cap = want;
    return RNG_OK;
}

// Grows a device buffer to at least `need` elements (at least doubling, so
// that lists of varying length settle after a few ticks: the free below
// synchronises the device); waits first for work on `stream` that may
// still read the old one.
template <class T>
int ensure_device(T **buf, uint64_t *cap, uint64_t need, cudaStream_t stream)
{
    if (need <= *cap)
        return RNG_OK;
    const uint64_t want = std::max<uint64_t>(need, 2 * *cap);
    int st = cuda_status(cudaStreamSynchronize(stream));
    T *grown = nullptr;
    if (!st && cudaMalloc(&grown, want * sizeof(T)) != cudaSuccess)
        st = set_error(RNG_ERR_OOM);
    if (!st) {
        cudaFree(*buf);
        *buf = grown;
        *cap = want;
    }
    return st;
}

// The refill of rng_plan_refill and plan_refill_mixed: with `maps` (host
// words) every item i gets the map at word map_off[i] of them.
int refill(Plan *p, const rng_batch_item *items, size_t n_items, const uint64_t *map_off,
           const uint32_t *maps, uint64_t map_words, cudaStream_t stream)
{
    if (!p || !items || n_items == 0 || (maps && (!map_off || map_words == 0)))
        return set_error(RNG_ERR_ARG);
    int device = -1;
    p->claims.resize(n_items);
    int st = validate_items(items, n_items, p->claims.data(), &device);
    if (st)
        return st;
    if (device != p->device)
        return set_error(RNG_ERR_ARG);
    int kind = -1;  // a mapped refill holds one kind (its kernel carries one)
    if (maps)
        for (size_t i = 0; i < n_items; ++i) {
            const int k = reinterpret_cast<Gen *>(items[i].h)->kind;
            if (map_off[i] + 3 >= map_words || (kind >= 0 && k != kind))
                return set_error(RNG_ERR_ARG);
            kind = k;
        }
    const uint64_t n = fill_units(items, n_items, p->threads, nullptr, 0);
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != p->device)
        cudaSetDevice(p->device);
    const int k = p->turn;
    if (p->copied[k])  // the copies out of this turn's lists, two refills ago
        st = cuda_status(cudaEventSynchronize(p->copied[k]));
    else
        st = cuda_status(cudaEventCreateWithFlags(&p->copied[k], cudaEventDisableTiming));
    if (!st)
        st = ensure_pinned(&p->pinned[k], &p->pinned_cap[k], n, p->pinned_cap[k ^ 1]);
    if (!st)
        st = ensure_device(&p->d_units, &p->cap_units, n, stream);
    std::vector<const uint32_t *> dmaps;
    if (!st && maps) {
        st = ensure_pinned(&p->pinned_maps[k], &p->pinned_maps_cap[k], map_words,
                           p->pinned_maps_cap[k ^ 1]);
        if (!st)
            st = ensure_device(&p->d_maps, &p->cap_maps, map_words, stream);
        if (!st && !p->grid_mixed)
            st = grid_for(p->device, p->threads, p->ctas_per_sm, &p->grid_mixed, true);
        if (!st) {
            dmaps.resize(n_items);
            for (size_t i = 0; i < n_items; ++i)
                dmaps[i] = p->d_maps + map_off[i];
            std::memcpy(p->pinned_maps[k], maps, map_words * sizeof(uint32_t));
            st = cuda_status(cudaMemcpyAsync(p->d_maps, p->pinned_maps[k],
                                             map_words * sizeof(uint32_t),
                                             cudaMemcpyHostToDevice, stream));
        }
    }
    if (!st)
        fill_units(items, n_items, p->threads, p->pinned[k], n, maps ? dmaps.data() : nullptr);
    if (!st && n)
        st = cuda_status(cudaMemcpyAsync(p->d_units, p->pinned[k], n * sizeof(Unit),
                                         cudaMemcpyHostToDevice, stream));
    if (!st)
        st = cuda_status(cudaEventRecord(p->copied[k], stream));
    if (!st) {
        p->n_units = n;
        p->mixed = maps != nullptr;
        p->mixed_kind = kind;
        p->turn ^= 1;
    }
    if (prev >= 0 && prev != p->device)
        cudaSetDevice(prev);
    return st;
}

}  // namespace

int plan_refill_mixed(rng_plan_handle h, const rng_batch_item *items, size_t n_items,
                      const uint64_t *map_off, const uint32_t *maps, uint64_t map_words,
                      cudaStream_t stream)
{
    if (!maps)
        return set_error(RNG_ERR_ARG);
    return refill(reinterpret_cast<Plan *>(h), items, n_items, map_off, maps, map_words, stream);
}

}  // namespace gbrng

extern "C" int rng_plan_refill(rng_plan_handle h, const rng_batch_item *items, size_t n_items,
                               void *cuda_stream)
{
    return refill(reinterpret_cast<Plan *>(h), items, n_items, nullptr, nullptr, 0,
                  static_cast<cudaStream_t>(cuda_stream));
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
namespace gbrng {
namespace {

constexpr uint64_t kNoAllocMaxTiles = 32768;  // work-list capacity, in tiles
constexpr int kNoAllocThreads = 128;           // CTA size: tiles of 512 streams
constexpr size_t kNoAllocMaxItems = 4096;     // items per call
constexpr size_t kNoAllocHeader = 256;        // tile counter, then padding
constexpr size_t kNoAllocBytes = kNoAllocHeader + kNoAllocMaxTiles * sizeof(Unit);

// The scratch: bytes [0, 8) hold the tile counter, the work list starts at
// byte kNoAllocHeader.  Every GPU that loads the library holds it until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mutex;                      // guards the host arrays below
void *g_noalloc_dev_ptr[64] = {nullptr};         // device address of the scratch
Unit g_noalloc_host_units[kNoAllocMaxTiles];     // host copy of the work list
Claim g_noalloc_claims[kNoAllocMaxItems];       // overlap check

}  // namespace
}  // namespace gbrng

extern "C" int rng_generate_batch_noalloc(const rng_batch_item *items, size_t n_items,
                                          void *cuda_stream)
{
    if (!items || n_items == 0 || n_items > kNoAllocMaxItems)
        return set_error(RNG_ERR_ARG);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    int device = -1;
    int st = validate_items(items, n_items, g_noalloc_claims, &device);
    if (st)
        return st;
    if (device >= 64)
        return set_error(RNG_ERR_ARG);
    // Work list, as rng_plan_create builds it with CTAs of kNoAllocThreads.
    const int threads = kNoAllocThreads;
    const uint64_t n_units =
        fill_units(items, n_items, threads, g_noalloc_host_units, kNoAllocMaxTiles);
    if (n_units > kNoAllocMaxTiles)
        return set_error(RNG_ERR_ARG);  // beyond the work-list capacity
    if (n_units == 0)
        return RNG_OK;
    order_units(g_noalloc_host_units, n_units);

    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess)
        return set_error(RNG_ERR_CUDA);
    if (prev != device && cudaSetDevice(device) != cudaSuccess)
        return set_error(RNG_ERR_CUDA);
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
    int grid = 0;
    if (!st)
        st = grid_for(device, threads, 0, &grid);
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
        batch_kernel<kHint><<<grid, threads, 0, stream>>>(units, n_units, next);
        st = cuda_status(cudaGetLastError());
    }
    if (prev >= 0 && prev != device)
        cudaSetDevice(prev);
    return st;
}
