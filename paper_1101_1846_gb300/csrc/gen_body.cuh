// Per-thread generation bodies shared by the plain kernels (generate.cu) and
// the batched persistent kernel (batch.cu), so that both produce identical
// outputs and state by construction.
#pragma once

#include "gbrng.cuh"

namespace gbrng {

template <int KIND>
struct Words;
template <>
struct Words<RNG_MWC32> { static constexpr int W = 2; };
template <>
struct Words<RNG_XOR128> { static constexpr int W = 4; };
template <>
struct Words<RNG_KISS> { static constexpr int W = 4; };

template <int KIND>
__device__ __forceinline__ uint32_t step(uint32_t a, uint32_t *w)
{
    if constexpr (KIND == RNG_MWC32)
        return mwc_step(a, w[0], w[1]);
    else if constexpr (KIND == RNG_XOR128)
        return xor128_step(w[0], w[1], w[2], w[3]);
    else
        return kiss_step(a, w[0], w[1], w[2], w[3]);
}

template <int HINT>
__device__ __forceinline__ void store16(uint4 *p, uint4 v)
{
    if constexpr (HINT == 1)
        __stcs(p, v);  // streaming: evict-first
    else
        *p = v;
}

template <int HINT>
__device__ __forceinline__ void store4(uint32_t *p, uint32_t v)
{
    if constexpr (HINT == 1)
        __stcs(p, v);
    else
        *p = v;
}

template <int FMT>
__device__ __forceinline__ uint32_t encode(uint32_t u)
{
    if constexpr (FMT == RNG_F32)
        return __float_as_uint(unit_f32(u));
    else
        return u;
}

// Vector body: this thread owns V groups of four adjacent streams starting at
// s_first + v * v_stride (v < V); groups at or beyond s_end are idle.  n is
// the generator's stream count (state stride), ld the output row stride.
// Requires n % 4 == 0, 16-byte aligned state, multipliers and out, ld % 4 == 0.
template <int KIND, int FMT, int V, int HINT>
__device__ __forceinline__ void body_vec(uint32_t *__restrict__ state,
                                         const uint32_t *__restrict__ mult, uint64_t n,
                                         uint64_t steps, uint32_t *__restrict__ out,
                                         uint64_t ld, uint64_t s_first, uint64_t v_stride,
                                         uint64_t s_end)
{
    constexpr int W = Words<KIND>::W;
    constexpr bool HAS_A = KIND != RNG_XOR128;
    uint32_t st[V][4][W];
    uint32_t a[V][4];
    bool live[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        uint64_t s0 = s_first + v_stride * v;
        live[v] = s0 < s_end;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            a[v][i] = 0;
#pragma unroll
            for (int w = 0; w < W; ++w)
                st[v][i][w] = 0;
        }
        if (live[v]) {
#pragma unroll
            for (int w = 0; w < W; ++w) {
                uint4 q = *reinterpret_cast<const uint4 *>(state + w * n + s0);
                st[v][0][w] = q.x;
                st[v][1][w] = q.y;
                st[v][2][w] = q.z;
                st[v][3][w] = q.w;
            }
            if constexpr (HAS_A) {
                uint4 q = *reinterpret_cast<const uint4 *>(mult + s0);
                a[v][0] = q.x;
                a[v][1] = q.y;
                a[v][2] = q.z;
                a[v][3] = q.w;
            }
        }
    }

    uint32_t *row = out + s_first;
#pragma unroll 4
    for (uint64_t j = 0; j < steps; ++j) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
            uint4 o;
            o.x = encode<FMT>(step<KIND>(a[v][0], st[v][0]));
            o.y = encode<FMT>(step<KIND>(a[v][1], st[v][1]));
            o.z = encode<FMT>(step<KIND>(a[v][2], st[v][2]));
            o.w = encode<FMT>(step<KIND>(a[v][3], st[v][3]));
            if (live[v])
                store16<HINT>(reinterpret_cast<uint4 *>(row + v_stride * v), o);
        }
        row += ld;
    }

#pragma unroll
    for (int v = 0; v < V; ++v) {
        uint64_t s0 = s_first + v_stride * v;
        if (live[v]) {
#pragma unroll
            for (int w = 0; w < W; ++w) {
                uint4 q = make_uint4(st[v][0][w], st[v][1][w], st[v][2][w], st[v][3][w]);
                *reinterpret_cast<uint4 *>(state + w * n + s0) = q;
            }
        }
    }
}

// Scalar body: one stream s (< n), 4-byte stores; any n, 4-byte aligned out.
template <int KIND, int FMT, int HINT>
__device__ __forceinline__ void body_scalar(uint32_t *__restrict__ state,
                                            const uint32_t *__restrict__ mult, uint64_t n,
                                            uint64_t steps, uint32_t *__restrict__ out,
                                            uint64_t ld, uint64_t s)
{
    constexpr int W = Words<KIND>::W;
    uint32_t st[W];
#pragma unroll
    for (int w = 0; w < W; ++w)
        st[w] = state[w * n + s];
    uint32_t a = 0;
    if constexpr (KIND != RNG_XOR128)
        a = mult[s];
    uint32_t *p = out + s;
#pragma unroll 4
    for (uint64_t j = 0; j < steps; ++j) {
        store4<HINT>(p, encode<FMT>(step<KIND>(a, st)));
        p += ld;
    }
#pragma unroll
    for (int w = 0; w < W; ++w)
        state[w * n + s] = st[w];
}

}  // namespace gbrng
