// Jump-ahead tables and rng_jump (sequence splitting, Sec. "Parallelizing
// RNGs").  The tables hold, for m = 0..63, the GF(2) matrix of 2^m xor128
// steps (128 columns of 4 words), of 2^m XORSHIFT8 steps (256 columns of 8
// words), of 2^m xorshift32 steps (32 columns) and the affine map (A, C) of
// 2^m LCG steps.  One CTA builds them on the device by repeated squaring,
// once per device and process.
#include <mutex>

#include "jump.cuh"

namespace gbrng {
namespace {

constexpr int kLevels = 64;
constexpr int kMaxDevices = 64;

struct DeviceTables {
    void *mem = nullptr;
    JumpTables t{};
};
DeviceTables g_tables[kMaxDevices];
std::mutex g_mutex;

// Column j of level m is level m-1 applied to its own column j.
__global__ void __launch_bounds__(256)
build_tables(uint4 *t128, uint32_t *t32, uint2 *tl, uint4 *t8)
{
    __shared__ uint4 cur[128];
    __shared__ uint4 cur8[512];  // column j: cur8[2j] (words 0-3), cur8[2j+1] (4-7)
    __shared__ uint32_t cur32[32];
    const int j = threadIdx.x;
    {
        uint32_t v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int q = 0; q < 8; ++q)
            v[q] = (j >> 5) == q ? 1u << (j & 31) : 0u;
        xorshift8_step(v[0], v[1], v[2], v[3], v[4], v[5], v[6], v[7]);
        cur8[2 * j] = make_uint4(v[0], v[1], v[2], v[3]);
        cur8[2 * j + 1] = make_uint4(v[4], v[5], v[6], v[7]);
        t8[2 * j] = cur8[2 * j];
        t8[2 * j + 1] = cur8[2 * j + 1];
        if (j < 128) {
            uint32_t s[4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                s[q] = (j >> 5) == q ? 1u << (j & 31) : 0u;
            xor128_step(s[0], s[1], s[2], s[3]);
            cur[j] = make_uint4(s[0], s[1], s[2], s[3]);
            t128[j] = cur[j];
        }
        if (j < 32) {
            uint32_t y = 1u << j;
            xorshift32_step(y);
            cur32[j] = y;
            t32[j] = y;
        }
    }
    for (int m = 1; m < kLevels; ++m) {
        __syncthreads();
        // XORSHIFT8: every thread one column
        const uint4 lo = cur8[2 * j], hi = cur8[2 * j + 1];
        const uint32_t vw8[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
        uint4 r8lo = make_uint4(0, 0, 0, 0), r8hi = make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            for (int b = 0; b < 32; ++b) {
                if ((vw8[q] >> b) & 1u) {
                    const uint4 c0 = cur8[2 * (32 * q + b)], c1 = cur8[2 * (32 * q + b) + 1];
                    r8lo.x ^= c0.x;
                    r8lo.y ^= c0.y;
                    r8lo.z ^= c0.z;
                    r8lo.w ^= c0.w;
                    r8hi.x ^= c1.x;
                    r8hi.y ^= c1.y;
                    r8hi.z ^= c1.z;
                    r8hi.w ^= c1.w;
                }
            }
        }
        uint4 r = make_uint4(0, 0, 0, 0);
        if (j < 128) {
            const uint4 v = cur[j];
            const uint32_t vw[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                for (int b = 0; b < 32; ++b) {
                    if ((vw[q] >> b) & 1u) {
                        const uint4 c = cur[32 * q + b];
                        r.x ^= c.x;
                        r.y ^= c.y;
                        r.z ^= c.z;
                        r.w ^= c.w;
                    }
                }
            }
        }
        uint32_t r32 = 0;
        if (j < 32) {
            const uint32_t y = cur32[j];
            for (int b = 0; b < 32; ++b)
                if ((y >> b) & 1u)
                    r32 ^= cur32[b];
        }
        __syncthreads();
        cur8[2 * j] = r8lo;
        cur8[2 * j + 1] = r8hi;
        t8[m * 512 + 2 * j] = r8lo;
        t8[m * 512 + 2 * j + 1] = r8hi;
        if (j < 128) {
            cur[j] = r;
            t128[m * 128 + j] = r;
        }
        if (j < 32) {
            cur32[j] = r32;
            t32[m * 32 + j] = r32;
        }
    }
    if (j == 0) {
        uint32_t A = 69069u, C = 1234567u;  // one step of Eq. 7
        for (int m = 0; m < kLevels; ++m) {
            tl[m] = make_uint2(A, C);
            C = A * C + C;  // the map after itself
            A = A * A;
        }
    }
}

// Entry y*n + s: a_s^(y*rows) mod p_s in Montgomery form (0 for y = 0, the
// segment that needs no jump).
__global__ void __launch_bounds__(256)
mwc_table_kernel(const uint32_t *__restrict__ a, uint64_t n, uint64_t rows, uint32_t segs,
                 uint64_t *__restrict__ out)
{
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * segs)
        return;
    const uint64_t y = i / n, s = i - y * n;
    out[i] = y == 0 ? 0 : mwc_power(a[s], y * rows);
}

template <int KIND>
__global__ void __launch_bounds__(256) jump_kernel(rng_device_view v, uint64_t k, JumpTables T)
{
    const uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= v.n_streams)
        return;
    Engine<KIND> e;
    e.load(v, s);
    jump_engine<KIND>(e, k, T);
    e.store(v, s);
}

}  // namespace

int jump_tables(JumpTables *out)
{
    int dev = 0;
    int st = cuda_status(cudaGetDevice(&dev));
    if (st)
        return st;
    if (dev < 0 || dev >= kMaxDevices)
        return set_error(RNG_ERR_NODEV);
    std::lock_guard<std::mutex> lock(g_mutex);
    DeviceTables &d = g_tables[dev];
    if (!d.mem) {
        const size_t b128 = sizeof(uint4) * 128 * kLevels;
        const size_t b8 = sizeof(uint4) * 512 * kLevels;
        const size_t b32 = sizeof(uint32_t) * 32 * kLevels;
        const size_t bl = sizeof(uint2) * kLevels;
        void *mem = nullptr;
        if (cudaMalloc(&mem, b128 + b8 + b32 + bl) != cudaSuccess)
            return set_error(RNG_ERR_OOM);
        char *base = static_cast<char *>(mem);
        uint4 *t128 = reinterpret_cast<uint4 *>(base);
        uint4 *t8 = reinterpret_cast<uint4 *>(base + b128);
        uint32_t *t32 = reinterpret_cast<uint32_t *>(base + b128 + b8);
        uint2 *tl = reinterpret_cast<uint2 *>(base + b128 + b8 + b32);
        build_tables<<<1, 256>>>(t128, t32, tl, t8);
        st = cuda_status(cudaGetLastError());
        if (!st)
            st = cuda_status(cudaStreamSynchronize(0));
        if (st) {
            cudaFree(mem);
            return st;
        }
        d.mem = mem;
        d.t = JumpTables{t128, t32, tl, t8};
    }
    *out = d.t;
    return RNG_OK;
}

int mwc_jump_table(Gen *g, uint64_t rows, uint64_t segs, cudaStream_t st,
                   const uint64_t **table)
{
    if (!g->d_a || segs == 0 || segs > g->jmul_segs)
        return set_error(RNG_ERR_ARG);
    if (segs > g->jmul_cap) {
        // grow: the old table may still be read by earlier calls (on any
        // stream), so wait for the device before freeing it
        int e = cuda_status(cudaDeviceSynchronize());
        if (e)
            return e;
        cudaFree(g->d_jmul);
        g->d_jmul = nullptr;
        g->jmul_cap = 0;
        g->jmul_rows = 0;
        if (cudaMalloc(&g->d_jmul, (size_t)segs * g->n * 8) != cudaSuccess)
            return set_error(RNG_ERR_OOM);
        g->jmul_cap = (uint32_t)segs;
    }
    if (g->jmul_rows != rows) {
        const uint64_t total = g->n * g->jmul_cap;
        const uint64_t blocks = (total + 255) / 256;
        mwc_table_kernel<<<(unsigned)blocks, 256, 0, st>>>(g->d_a, g->n, rows, g->jmul_cap,
                                                           g->d_jmul);
        int e = cuda_status(cudaGetLastError());
        if (e)
            return e;
        g->jmul_rows = rows;
    }
    *table = g->d_jmul;
    return RNG_OK;
}

int launch_jump(Gen *g, uint64_t k, cudaStream_t stream)
{
    if (k == 0)
        return RNG_OK;
    JumpTables T{};
    if (needs_jump_tables(g->kind)) {
        int st = jump_tables(&T);
        if (st)
            return st;
    }
    rng_device_view v{g->kind, g->device, g->words, g->n, g->d_state, g->d_a};
    const uint64_t blocks = (g->n + 255) / 256;
    if (blocks > 0x7FFFFFFFull)
        return set_error(RNG_ERR_ARG);
    const unsigned b = (unsigned)blocks;
    switch (g->kind) {
    case RNG_MWC32: jump_kernel<RNG_MWC32><<<b, 256, 0, stream>>>(v, k, T); break;
    case RNG_XOR128: jump_kernel<RNG_XOR128><<<b, 256, 0, stream>>>(v, k, T); break;
    case RNG_KISS: jump_kernel<RNG_KISS><<<b, 256, 0, stream>>>(v, k, T); break;
    case RNG_MWC16X2: jump_kernel<RNG_MWC16X2><<<b, 256, 0, stream>>>(v, k, T); break;
    case RNG_XORSHIFT8: jump_kernel<RNG_XORSHIFT8><<<b, 256, 0, stream>>>(v, k, T); break;
    default: jump_kernel<RNG_KISS_XOR><<<b, 256, 0, stream>>>(v, k, T); break;
    }
    return cuda_status(cudaGetLastError());
}

}  // namespace gbrng
