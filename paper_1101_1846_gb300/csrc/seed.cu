// Per-stream seeding.  The paper gives every thread its own seeds (and, for
// MWC and KISS, its own multipliers) without fixing how the seeds are made;
// here stream s draws from splitmix64 (Steele, Lea and Flood, OOPSLA 2014)
// started at seed + s.  Mapping of draws to state words (include/rng.h):
//   MWC32  x = lo32(r), c = hi32(r) mod a; redraw while (x, c) is a fixed
//          point of the recurrence, (0, 0) or (2^32 - 1, a - 1)
//   xor128 (x, y, z, w) = lo/hi of two draws; redraw both while all zero
//   KISS   (x, c) as MWC32; then y = lo32, z = hi32 of the next draw; y
//          replaced by lo32 of further draws while zero
//   MWC16X2  from one draw r: part 1 x = bits 0-15, c = bits 16-31 mod a1,
//          part 2 x = bits 32-47, c = bits 48-63 mod a2, each kept as
//          x | c << 16; redraw while either part is a fixed point
//   XORSHIFT8  eight words = lo32, hi32 of four draws; redraw while all zero
//   KISS_XOR  the pair as MWC16X2, then y and the LCG word as KISS
#include "gbrng.cuh"

namespace gbrng {
namespace {

__device__ __forceinline__ uint64_t splitmix64_next(uint64_t &z)
{
    z += 0x9E3779B97F4A7C15ull;
    uint64_t r = z;
    r = (r ^ (r >> 30)) * 0xBF58476D1CE4E5B9ull;
    r = (r ^ (r >> 27)) * 0x94D049BB133111EBull;
    return r ^ (r >> 31);
}

__device__ __forceinline__ void draw_mwc(uint64_t &z, uint32_t a, uint32_t &x, uint32_t &c)
{
    // Each redraw is needed with probability below 2^-63; the loop ends.
    for (;;) {
        uint64_t r = splitmix64_next(z);
        x = (uint32_t)r;
        c = (uint32_t)(r >> 32) % a;
        bool fixed = (x == 0 && c == 0) || (x == 0xFFFFFFFFu && c == a - 1);
        if (!fixed)
            return;
    }
}

__device__ __forceinline__ void draw_mwc16x2(uint64_t &z, uint32_t a_pair, uint32_t &p1,
                                             uint32_t &p2)
{
    const uint32_t a1 = a_pair & 0xFFFFu, a2 = a_pair >> 16;
    for (;;) {
        const uint64_t r = splitmix64_next(z);
        const uint32_t x1 = (uint32_t)(r & 0xFFFFu), c1 = (uint32_t)((r >> 16) & 0xFFFFu) % a1;
        const uint32_t x2 = (uint32_t)((r >> 32) & 0xFFFFu), c2 = (uint32_t)(r >> 48) % a2;
        const bool bad1 = (x1 == 0 && c1 == 0) || (x1 == 0xFFFFu && c1 == a1 - 1);
        const bool bad2 = (x2 == 0 && c2 == 0) || (x2 == 0xFFFFu && c2 == a2 - 1);
        if (!bad1 && !bad2) {
            p1 = x1 | (c1 << 16);
            p2 = x2 | (c2 << 16);
            return;
        }
    }
}

__global__ void seed_kernel(int kind, uint64_t n, uint64_t seed, const uint32_t *a,
                            uint32_t *state)
{
    uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n)
        return;
    uint64_t z = seed + s;
    if (kind == RNG_MWC16X2 || kind == RNG_KISS_XOR) {
        uint32_t p1, p2;
        draw_mwc16x2(z, a[s], p1, p2);
        state[s] = p1;
        state[n + s] = p2;
        if (kind == RNG_KISS_XOR) {
            const uint64_t r = splitmix64_next(z);
            uint32_t y = (uint32_t)r;
            const uint32_t l = (uint32_t)(r >> 32);
            while (y == 0)
                y = (uint32_t)splitmix64_next(z);
            state[2 * n + s] = y;
            state[3 * n + s] = l;
        }
        return;
    }
    if (kind == RNG_XORSHIFT8) {
        uint32_t v[8];
        uint32_t any;
        do {
            any = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const uint64_t r = splitmix64_next(z);
                v[2 * i] = (uint32_t)r;
                v[2 * i + 1] = (uint32_t)(r >> 32);
                any |= v[2 * i] | v[2 * i + 1];
            }
        } while (any == 0);
#pragma unroll
        for (int k = 0; k < 8; ++k)
            state[k * n + s] = v[k];
        return;
    }
    if (kind == RNG_MWC32) {
        uint32_t x, c;
        draw_mwc(z, a[s], x, c);
        state[s] = x;
        state[n + s] = c;
    } else if (kind == RNG_XOR128) {
        uint32_t w0, w1, w2, w3;
        do {
            uint64_t r0 = splitmix64_next(z);
            uint64_t r1 = splitmix64_next(z);
            w0 = (uint32_t)r0;
            w1 = (uint32_t)(r0 >> 32);
            w2 = (uint32_t)r1;
            w3 = (uint32_t)(r1 >> 32);
        } while ((w0 | w1 | w2 | w3) == 0);
        state[s] = w0;
        state[n + s] = w1;
        state[2 * n + s] = w2;
        state[3 * n + s] = w3;
    } else {
        uint32_t x, c;
        draw_mwc(z, a[s], x, c);
        uint64_t r = splitmix64_next(z);
        uint32_t y = (uint32_t)r, w = (uint32_t)(r >> 32);
        while (y == 0)
            y = (uint32_t)splitmix64_next(z);
        state[s] = x;
        state[n + s] = c;
        state[2 * n + s] = y;
        state[3 * n + s] = w;
    }
}

}  // namespace

int launch_seed(Gen *g, cudaStream_t st)
{
    const int threads = 256;
    uint64_t blocks = (g->n + threads - 1) / threads;
    seed_kernel<<<(unsigned)blocks, threads, 0, st>>>(g->kind, g->n, g->seed, g->d_a,
                                                      g->d_state);
    return cuda_status(cudaGetLastError());
}

}  // namespace gbrng
