// A small statistical battery on the device (rng_battery): counts of four
// tests of the DIEHARD / TestU01 families over stream-interleaved outputs,
// for the randomness checks the paper runs with those suites (Sec.
// "Performance evaluation").  The host forms the statistics from the counts.
//
//   monobit    one bits in all outputs
//   frequency  top 8 bits, 256 bins
//   serial     non-overlapping pairs (u_{2k}, u_{2k+1}) of a stream, top 4
//              bits of each, 16 x 16 cells
//   birthday   512 consecutive outputs of a stream, days = top 24 bits;
//              sorted, spacings (first day, then neighbour differences),
//              sorted; repeats = spacings equal to the one before; at most
//              RNG_BATTERY_BIRTHDAY_MAX samples
//
// count_kernel: a CTA takes 256 consecutive streams (coalesced row reads)
// and a tile of row pairs; histograms in shared memory, added to the global
// 64-bit counts once per CTA.  birthday_kernel: one CTA of 512 threads per
// sample, two bitonic sorts in shared memory.
#include <algorithm>

#include "gbrng.cuh"

namespace gbrng {
namespace {

constexpr int kCountThreads = 256;
constexpr uint64_t kPairsPerTile = 64;
constexpr int kDays = 512;

struct DeviceCounts {
    unsigned long long ones;
    unsigned long long bytes[256];
    unsigned long long serial[256];
    unsigned long long birthday[16];
};

__global__ void __launch_bounds__(kCountThreads)
count_kernel(const uint32_t *__restrict__ u, uint64_t n, uint64_t rows, uint64_t tile_pairs,
             DeviceCounts *out)
{
    __shared__ uint32_t bytes[256], serial[256];
    __shared__ unsigned long long ones_sum;
    const int t = threadIdx.x;
    bytes[t] = 0;
    serial[t] = 0;
    if (t == 0)
        ones_sum = 0;
    __syncthreads();
    const uint64_t s = (uint64_t)blockIdx.x * kCountThreads + t;
    const uint64_t r0 = (uint64_t)blockIdx.y * 2 * tile_pairs;
    uint64_t ones = 0;
    if (s < n) {
        const uint64_t r1 = min(rows, r0 + 2 * tile_pairs);
        uint64_t r = r0;
        for (; r + 1 < r1; r += 2) {
            const uint32_t a = __ldg(u + r * n + s), b = __ldg(u + (r + 1) * n + s);
            ones += __popc(a) + __popc(b);
            atomicAdd(&bytes[a >> 24], 1u);
            atomicAdd(&bytes[b >> 24], 1u);
            atomicAdd(&serial[(a >> 28) * 16 + (b >> 28)], 1u);
        }
        if (r < r1) {  // the last row of an odd count: no pair
            const uint32_t a = __ldg(u + r * n + s);
            ones += __popc(a);
            atomicAdd(&bytes[a >> 24], 1u);
        }
    }
    atomicAdd(&ones_sum, (unsigned long long)ones);
    __syncthreads();
    if (bytes[t])
        atomicAdd(&out->bytes[t], (unsigned long long)bytes[t]);
    if (serial[t])
        atomicAdd(&out->serial[t], (unsigned long long)serial[t]);
    if (t == 0)
        atomicAdd(&out->ones, ones_sum);
}

// Ascending bitonic sort of kDays values, one per thread.
__device__ __forceinline__ void bitonic512(uint32_t *v)
{
    const int i = threadIdx.x;
    for (int k = 2; k <= kDays; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            const int p = i ^ j;
            if (p > i) {
                const uint32_t a = v[i], b = v[p];
                const bool up = (i & k) == 0;
                if ((a > b) == up) {
                    v[i] = b;
                    v[p] = a;
                }
            }
            __syncthreads();
        }
    }
}

// Sample blockIdx.x = (stream s, block b): outputs rows 512 b .. 512 b + 511.
__global__ void __launch_bounds__(kDays)
birthday_kernel(const uint32_t *__restrict__ u, uint64_t n, uint64_t blocks_per_stream,
                DeviceCounts *out)
{
    __shared__ uint32_t day[kDays], gap[kDays];
    const int i = threadIdx.x;
    const uint64_t s = blockIdx.x % n;
    const uint64_t b = blockIdx.x / n;
    if (b >= blocks_per_stream)
        return;  // uniform across the CTA
    day[i] = __ldg(u + (b * kDays + i) * n + s) >> 8;
    __syncthreads();
    bitonic512(day);
    gap[i] = i == 0 ? day[0] : day[i] - day[i - 1];
    __syncthreads();
    bitonic512(gap);
    const int repeats = __syncthreads_count(i > 0 && gap[i] == gap[i - 1]);
    if (i == 0)
        atomicAdd(&out->birthday[repeats < 15 ? repeats : 15], 1ull);
}

}  // namespace
}  // namespace gbrng

using namespace gbrng;

extern "C" int rng_battery(const void *dev_u, uint64_t n_streams, uint64_t n_per_stream,
                           rng_battery_counts *host_counts, void *cuda_stream)
{
    if (!dev_u || !host_counts || n_streams == 0 || (uintptr_t)dev_u % 4 != 0 ||
        n_per_stream > UINT64_MAX / 4 / n_streams)
        return set_error(RNG_ERR_ARG);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const uint32_t *u = static_cast<const uint32_t *>(dev_u);
    DeviceCounts *d = nullptr;
    if (cudaMalloc(&d, sizeof(DeviceCounts)) != cudaSuccess)
        return set_error(RNG_ERR_OOM);
    int status = cuda_status(cudaMemsetAsync(d, 0, sizeof(DeviceCounts), st));
    const uint64_t gx = (n_streams + kCountThreads - 1) / kCountThreads;
    // row pairs per tile: at least kPairsPerTile, more when the grid's y
    // dimension (at most 65535) would not cover the rows
    const uint64_t pairs = (n_per_stream + 1) / 2;
    const uint64_t tile = std::max<uint64_t>(kPairsPerTile, (pairs + 65534) / 65535);
    const uint64_t gy = (pairs + tile - 1) / tile;
    if (!status && n_per_stream && gx > 0x7FFFFFFFull)
        status = set_error(RNG_ERR_ARG);
    if (!status && n_per_stream) {
        count_kernel<<<dim3((unsigned)gx, (unsigned)gy), kCountThreads, 0, st>>>(
            u, n_streams, n_per_stream, tile, d);
        status = cuda_status(cudaGetLastError());
    }
    const uint64_t blocks = n_per_stream / kDays;
    // sample i: block i / n_streams of stream i % n_streams, i < the cap
    const uint64_t samples = std::min<uint64_t>(blocks * n_streams, RNG_BATTERY_BIRTHDAY_MAX);
    if (!status && samples) {
        birthday_kernel<<<(unsigned)samples, kDays, 0, st>>>(u, n_streams, blocks, d);
        status = cuda_status(cudaGetLastError());
    }
    DeviceCounts h{};
    if (!status)
        status = cuda_status(cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, st));
    if (!status)
        status = cuda_status(cudaStreamSynchronize(st));
    cudaFree(d);
    if (status)
        return status;
    host_counts->n_outputs = n_streams * n_per_stream;
    host_counts->ones = h.ones;
    for (int k = 0; k < 256; ++k) {
        host_counts->bytes[k] = h.bytes[k];
        host_counts->serial[k] = h.serial[k];
    }
    host_counts->birthday_samples = samples;
    for (int k = 0; k < 16; ++k)
        host_counts->birthday[k] = h.birthday[k];
    return RNG_OK;
}
