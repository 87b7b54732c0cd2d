// Device search for the MWC multipliers: a < 2^32, largest first, such that
// p = a*2^32 - 1 and q = (p - 1)/2 = a*2^31 - 1 are both prime (the
// safe-prime condition of the paper's MWC background section).  Stream s of
// an MWC32 or KISS generator uses entry s (parametrisation, Sec.
// "Parallelizing RNGs").
//
// One thread per candidate a.  A candidate must pass trial division by the
// primes below 1024 (for each prime l, l | q iff a = 2^-31 mod l and l | p iff
// a = 2^-32 mod l; both q and p exceed 1024, so a hit is a proof of
// compositeness) and then a deterministic Miller-Rabin test of q and p with
// the first twelve primes as bases (deterministic below 3.3e24; Sorenson and
// Webster 2017) in 64-bit Montgomery arithmetic.
//
// Candidates are scanned in batches of descending a.  Each CTA owns a tile of
// consecutive candidates and appends its hits, in descending order, to its
// own list in scratch memory; a second kernel scans the tile counts and
// concatenates the lists into the table.  The table is kept per device for
// the life of the process and only ever grows.
#include <mutex>
#include <vector>

#include "gbrng.cuh"
#include "modarith.cuh"

namespace gbrng {
namespace {

constexpr int kThreads = 256;
constexpr int kRounds = 64;                      // candidates per thread per tile
constexpr uint32_t kTile = kThreads * kRounds;   // 16384 candidates per CTA
constexpr uint32_t kTileCap = 1024;              // hits kept per tile
constexpr uint32_t kTilesPerBatch = 4096;        // 2^26 candidates per batch
constexpr int kMaxSmallPrimes = 180;

struct SmallPrimes {
    uint32_t l[kMaxSmallPrimes];
    uint32_t q_root[kMaxSmallPrimes];  // a mod l == q_root  <=>  l | a*2^31 - 1
    uint32_t p_root[kMaxSmallPrimes];  // a mod l == p_root  <=>  l | a*2^32 - 1
    int count;
};
__constant__ SmallPrimes c_primes;

__device__ bool miller_rabin_u64(uint64_t n)
{
    // n odd, n > 2^32 here.
    uint64_t inv = n;  // n*n = 1 mod 8: 3 correct bits, Newton doubles them
#pragma unroll
    for (int i = 0; i < 5; ++i)
        inv *= 2 - n * inv;
    uint64_t ninv = 0 - inv;
    uint64_t one = (0 - n) % n;  // R mod n
    uint64_t r2 = one;           // R^2 mod n by 64 modular doublings
    for (int i = 0; i < 64; ++i) {
        uint64_t d = r2 << 1;
        if ((r2 >> 63) || d >= n)
            d -= n;
        r2 = d;
    }
    uint64_t minus_one = n - one;
    uint64_t d = n - 1;
    int r = __ffsll((long long)d) - 1;
    d >>= r;
    const uint32_t bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    for (int i = 0; i < 12; ++i) {
        uint64_t b = mont_mul(bases[i], r2, n, ninv);
        uint64_t x = one;
        for (int bit = 63 - __clzll((long long)d); bit >= 0; --bit) {
            x = mont_mul(x, x, n, ninv);
            if ((d >> bit) & 1)
                x = mont_mul(x, b, n, ninv);
        }
        if (x == one || x == minus_one)
            continue;
        bool composite = true;
        for (int k = 1; k < r; ++k) {
            x = mont_mul(x, x, n, ninv);
            if (x == minus_one) {
                composite = false;
                break;
            }
        }
        if (composite)
            return false;
    }
    return true;
}

__device__ bool is_multiplier(uint32_t a)
{
    if (a < 2)
        return false;
    for (int i = 0; i < c_primes.count; ++i) {
        uint32_t r = a % c_primes.l[i];
        if (r == c_primes.q_root[i] || r == c_primes.p_root[i])
            return false;
    }
    uint64_t q = ((uint64_t)a << 31) - 1;
    uint64_t p = 2 * q + 1;
    return miller_rabin_u64(q) && miller_rabin_u64(p);
}

// Tile t of the batch covers a = a_hi - t*kTile - i, i in [0, kTile), a >= a_lo.
__global__ void __launch_bounds__(kThreads)
search_tiles(uint64_t a_hi, uint64_t a_lo, uint32_t *lists, uint32_t *counts,
             uint32_t *overflow)
{
    __shared__ uint32_t warp_hits[kThreads / 32];
    __shared__ uint32_t base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0)
        base = 0;
    __syncthreads();
    uint32_t *list = lists + (uint64_t)blockIdx.x * kTileCap;
    for (int round = 0; round < kRounds; ++round) {
        uint64_t off = (uint64_t)blockIdx.x * kTile + (uint64_t)round * kThreads + threadIdx.x;
        bool hit = false;
        uint32_t a = 0;
        if (off <= a_hi - a_lo) {
            a = (uint32_t)(a_hi - off);
            hit = is_multiplier(a);
        }
        uint32_t mask = __ballot_sync(0xffffffffu, hit);
        if (lane == 0)
            warp_hits[warp] = __popc(mask);
        __syncthreads();
        uint32_t before = base;
        for (int w = 0; w < warp; ++w)
            before += warp_hits[w];
        before += __popc(mask & ((1u << lane) - 1));
        if (hit) {
            if (before < kTileCap)
                list[before] = a;
            else
                atomicExch(overflow, 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t tot = 0;
            for (int w = 0; w < kThreads / 32; ++w)
                tot += warp_hits[w];
            base += tot;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        counts[blockIdx.x] = base < kTileCap ? base : kTileCap;
}

// One CTA: exclusive scan of the tile counts, then every tile's list is
// copied to table[done + prefix + i] while that index is below k.
__global__ void __launch_bounds__(1024)
gather_tiles(const uint32_t *lists, const uint32_t *counts, uint32_t n_tiles,
             uint32_t *table, uint64_t done, uint64_t k, unsigned long long *total)
{
    __shared__ uint32_t prefix[kTilesPerBatch + 1];
    __shared__ uint32_t warp_sum[32];
    // per-thread serial sums over kTilesPerBatch / 1024 tiles, then a block scan
    constexpr int per = kTilesPerBatch / 1024;
    uint32_t local[per];
    uint32_t s = 0;
    for (int i = 0; i < per; ++i) {
        uint32_t t = threadIdx.x * per + i;
        local[i] = t < n_tiles ? counts[t] : 0;
        s += local[i];
    }
    // inclusive warp scan of s
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t v = s;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o)
            v += y;
    }
    if (lane == 31)
        warp_sum[warp] = v;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = warp_sum[lane];
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o)
                w += y;
        }
        warp_sum[lane] = w;  // inclusive
    }
    __syncthreads();
    uint32_t excl = v - s + (warp > 0 ? warp_sum[warp - 1] : 0);
    for (int i = 0; i < per; ++i) {
        prefix[threadIdx.x * per + i] = excl;
        excl += local[i];
    }
    if (threadIdx.x == 1023)
        prefix[kTilesPerBatch] = excl;
    __syncthreads();
    // copy: one warp per tile
    for (uint32_t t = warp; t < n_tiles; t += 32) {
        uint32_t c = counts[t];
        for (uint32_t i = lane; i < c; i += 32) {
            uint64_t dst = done + prefix[t] + i;
            if (dst < k)
                table[dst] = lists[(uint64_t)t * kTileCap + i];
        }
    }
    if (threadIdx.x == 0)
        *total = prefix[kTilesPerBatch];
}

uint32_t pow_mod_u32(uint32_t b, uint32_t e, uint32_t m)
{
    uint64_t r = 1 % m, x = b % m;
    while (e) {
        if (e & 1)
            r = r * x % m;
        x = x * x % m;
        e >>= 1;
    }
    return (uint32_t)r;
}

struct DeviceTable {
    uint32_t *table = nullptr;
    uint64_t len = 0;         // entries found so far (all valid a >= next_hi+1)
    uint64_t cap = 0;
    uint64_t next_hi = 0xFFFFFFFFull;  // next candidate to scan
    bool primes_ready = false;
};

std::mutex g_mutex;
DeviceTable g_tables[64];

int upload_primes()
{
    SmallPrimes h{};
    std::vector<char> comp(1024, 0);
    int n = 0;
    for (uint32_t i = 3; i < 1024; i += 2) {
        if (comp[i])
            continue;
        for (uint32_t j = i * i; j < 1024; j += 2 * i)
            comp[j] = 1;
        uint32_t inv2 = (i + 1) / 2;
        h.l[n] = i;
        h.q_root[n] = pow_mod_u32(inv2, 31, i);
        h.p_root[n] = pow_mod_u32(inv2, 32, i);
        ++n;
    }
    h.count = n;
    return cuda_status(cudaMemcpyToSymbol(c_primes, &h, sizeof(h)));
}

// ------------------------------------------------ base-2^16 multipliers
// The paper's two-part MWC uses multipliers a < 2^16 with p = a 2^16 - 1 and
// q = a 2^15 - 1 both prime (392 of them).  p < 2^32, so Miller-Rabin with
// the bases 2, 7 and 61 is exact (no composite below 4,759,123,141 passes
// all three; Jaeschke 1993).  p, q >= 32767 > 61.
__device__ bool is_prime_u32(uint32_t n)
{
    if (n % 2 == 0)
        return n == 2;
    uint32_t d = n - 1;
    int r = 0;
    while ((d & 1) == 0) {
        d >>= 1;
        ++r;
    }
    const uint32_t bases[3] = {2, 7, 61};
    for (int i = 0; i < 3; ++i) {
        uint64_t x = 1, b = bases[i] % n;
        for (uint32_t e = d; e; e >>= 1) {
            if (e & 1)
                x = x * b % n;
            b = b * b % n;
        }
        if (x == 1 || x == n - 1)
            continue;
        bool composite = true;
        for (int k = 1; k < r; ++k) {
            x = x * x % n;
            if (x == n - 1) {
                composite = false;
                break;
            }
        }
        if (composite)
            return false;
    }
    return true;
}

// One CTA of 1024 threads: thread t tests a = 65535 - 64 t - i, i < 64
// (descending), and an exclusive scan of the hit counts in thread order puts
// the hits in descending order.
__global__ void __launch_bounds__(1024) mwc16_table_kernel(uint32_t *table, uint32_t *count)
{
    __shared__ uint32_t warp_sum[32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    uint64_t hits = 0;  // bit i: a = 65535 - 64 t - i passes
    for (int i = 0; i < 64; ++i) {
        const uint32_t a = 65535u - 64u * t - i;
        if (a >= 1 && is_prime_u32((a << 15) - 1) && is_prime_u32((a << 16) - 1))
            hits |= 1ull << i;
    }
    const uint32_t c = __popcll(hits);
    uint32_t incl = c;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o)
            incl += v;
    }
    if (lane == 31)
        warp_sum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = warp_sum[lane], wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o)
                wi += v;
        }
        warp_sum[lane] = wi - w;  // exclusive
        if (lane == 31)
            *count = wi;
    }
    __syncthreads();
    uint32_t pos = warp_sum[warp] + incl - c;
    for (int i = 0; i < 64; ++i)
        if ((hits >> i) & 1)
            table[pos++] = 65535u - 64u * t - i;
}

// Pair s (lexicographic, i < j) of the m-entry table, packed table[i] |
// table[j] << 16.
__global__ void mwc16_pairs_kernel(const uint32_t *table, uint32_t m, uint64_t k, uint32_t *out)
{
    const uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= k)
        return;
    uint64_t r = s;
    uint32_t i = 0;
    while (i + 1 < m && r >= m - 1 - i) {
        r -= m - 1 - i;
        ++i;
    }
    out[s] = table[i] | (table[i + 1 + r] << 16);
}

struct DevicePairs {
    uint32_t *pairs = nullptr;  // all 392 * 391 / 2 pairs
};
DevicePairs g_pairs[64];

}  // namespace

int multiplier_table(uint64_t k, const uint32_t **out)
{
    if (k == 0 || k > RNG_MAX_STREAMS_MWC)
        return set_error(RNG_ERR_ARG);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return set_error(RNG_ERR_NODEV);
    std::lock_guard<std::mutex> lock(g_mutex);
    DeviceTable &T = g_tables[dev];
    if (T.len >= k) {
        *out = T.table;
        return RNG_OK;
    }
    if (!T.primes_ready) {
        int st = upload_primes();
        if (st)
            return st;
        T.primes_ready = true;
    }
    // grow the table buffer
    if (T.cap < k) {
        uint64_t cap = T.cap ? T.cap : 4096;
        while (cap < k)
            cap *= 2;
        if (cap > RNG_MAX_STREAMS_MWC)
            cap = RNG_MAX_STREAMS_MWC;
        uint32_t *nt = nullptr;
        if (cudaMalloc(&nt, cap * sizeof(uint32_t)) != cudaSuccess)
            return set_error(RNG_ERR_OOM);
        if (T.len && cudaMemcpy(nt, T.table, T.len * 4, cudaMemcpyDeviceToDevice) != cudaSuccess) {
            cudaFree(nt);
            return set_error(RNG_ERR_CUDA);
        }
        cudaFree(T.table);
        T.table = nt;
        T.cap = cap;
    }
    // scratch: tile lists, tile counts, overflow flag, batch total
    uint32_t *lists = nullptr, *counts = nullptr, *flag = nullptr;
    unsigned long long *total = nullptr;
    size_t list_bytes = (size_t)kTilesPerBatch * kTileCap * 4;
    if (cudaMalloc(&lists, list_bytes) != cudaSuccess ||
        cudaMalloc(&counts, kTilesPerBatch * 4) != cudaSuccess ||
        cudaMalloc(&flag, 4) != cudaSuccess ||
        cudaMalloc(&total, 8) != cudaSuccess) {
        cudaFree(lists);
        cudaFree(counts);
        cudaFree(flag);
        return set_error(RNG_ERR_OOM);
    }
    int status = RNG_OK;
    cudaMemset(flag, 0, 4);
    while (T.len < k) {
        uint64_t a_hi = T.next_hi;
        if (a_hi < 2) {
            status = set_error(RNG_ERR_ARG);
            break;
        }
        uint64_t span = (uint64_t)kTilesPerBatch * kTile;
        uint64_t a_lo = a_hi + 1 > span ? a_hi + 1 - span : 1;
        uint32_t tiles = (uint32_t)((a_hi - a_lo + kTile) / kTile);
        search_tiles<<<tiles, kThreads>>>(a_hi, a_lo, lists, counts, flag);
        gather_tiles<<<1, 1024>>>(lists, counts, tiles, T.table, T.len, T.cap, total);
        unsigned long long found = 0;
        uint32_t over = 0;
        cudaError_t e = cudaMemcpy(&found, total, 8, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            e = cudaMemcpy(&over, flag, 4, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            status = cuda_status(e);
            break;
        }
        if (over) {  // a tile held more hits than its list: never seen; refuse
            status = set_error(RNG_ERR_CUDA);
            break;
        }
        if (T.len + found > T.cap) {
            // Hits past the buffer were dropped: keep what fits and resume
            // the next scan just below the last entry kept.
            T.len = T.cap;
            uint32_t last = 0;
            e = cudaMemcpy(&last, T.table + T.cap - 1, 4, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) {
                status = cuda_status(e);
                break;
            }
            T.next_hi = (uint64_t)last - 1;
            break;
        }
        T.len += found;
        T.next_hi = a_lo - 1;
    }
    cudaFree(lists);
    cudaFree(counts);
    cudaFree(flag);
    cudaFree(total);
    if (status)
        return status;
    if (T.len < k)
        return set_error(RNG_ERR_ARG);
    *out = T.table;
    return RNG_OK;
}

}  // namespace gbrng

namespace gbrng {

int mwc16_pair_table(uint64_t k, const uint32_t **out)
{
    if (k == 0 || k > RNG_MAX_STREAMS_MWC16)
        return set_error(RNG_ERR_ARG);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return set_error(RNG_ERR_NODEV);
    std::lock_guard<std::mutex> lock(g_mutex);
    DevicePairs &P = g_pairs[dev];
    if (!P.pairs) {
        uint32_t *table = nullptr, *count = nullptr, *pairs = nullptr;
        int st = RNG_OK;
        if (cudaMalloc(&table, 1024 * 4) != cudaSuccess || cudaMalloc(&count, 4) != cudaSuccess ||
            cudaMalloc(&pairs, RNG_MAX_STREAMS_MWC16 * 4) != cudaSuccess)
            st = set_error(RNG_ERR_OOM);
        uint32_t m = 0;
        if (!st) {
            mwc16_table_kernel<<<1, 1024>>>(table, count);
            st = cuda_status(cudaGetLastError());
        }
        if (!st)
            st = cuda_status(cudaMemcpy(&m, count, 4, cudaMemcpyDeviceToHost));
        if (!st && (uint64_t)m * (m - 1) / 2 != RNG_MAX_STREAMS_MWC16)
            st = set_error(RNG_ERR_CUDA);  // the search must find exactly 392
        if (!st) {
            const uint64_t total = RNG_MAX_STREAMS_MWC16;
            mwc16_pairs_kernel<<<(unsigned)((total + 255) / 256), 256>>>(table, m, total, pairs);
            st = cuda_status(cudaGetLastError());
        }
        if (!st)
            st = cuda_status(cudaDeviceSynchronize());
        cudaFree(table);
        cudaFree(count);
        if (st) {
            cudaFree(pairs);
            return st;
        }
        P.pairs = pairs;
    }
    *out = P.pairs;
    return RNG_OK;
}

}  // namespace gbrng

extern "C" int rng_mwc16_pairs(uint64_t k, uint32_t *dev_out)
{
    using namespace gbrng;
    if (!dev_out || k == 0 || k > RNG_MAX_STREAMS_MWC16)
        return set_error(RNG_ERR_ARG);
    const uint32_t *t = nullptr;
    int st = mwc16_pair_table(k, &t);
    if (st)
        return st;
    cudaError_t e = cudaMemcpy(dev_out, t, k * 4, cudaMemcpyDeviceToDevice);
    return e == cudaSuccess ? RNG_OK : cuda_status(e);
}

extern "C" int rng_multipliers(uint64_t k, uint32_t *dev_out)
{
    using namespace gbrng;
    if (!dev_out || k == 0 || k > RNG_MAX_STREAMS_MWC)
        return set_error(RNG_ERR_ARG);
    const uint32_t *t = nullptr;
    int st = multiplier_table(k, &t);
    if (st)
        return st;
    cudaError_t e = cudaMemcpy(dev_out, t, k * 4, cudaMemcpyDeviceToDevice);
    return e == cudaSuccess ? RNG_OK : cuda_status(e);
}
