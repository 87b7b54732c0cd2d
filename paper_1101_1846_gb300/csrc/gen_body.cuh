// Per-thread generation bodies shared by the plain kernels (generate.cu) and
// the batched persistent kernel (batch.cu), so that both produce identical
// outputs and state by construction.
//
// Three bodies:
//   body_vec    4 adjacent streams per group, V groups per thread, one
//               16-byte store per group per step; rows 32-byte aligned.
//   body_vec_sync  the same with one group per thread and a barrier every
//               SYNC_ROWS rows, for rows that are 16- but not 32-byte aligned.
//   body_shift  4 adjacent streams per thread for rows that are NOT 16-byte
//               aligned (any n, out 4-byte aligned): each row is written with
//               16-byte stores at the aligned positions, taking the words
//               that spill over from the lane on the left by a warp shuffle;
//               a halo lane per warp closes the warp boundaries, and only
//               the CTA's first and last words go out as 4-byte stores.
//   body_scalar one stream per thread, 4-byte stores (tails of < 4 streams).
#pragma once

#include "gbrng.cuh"

namespace gbrng {

// Per kind: state words per stream (W) and whether each stream has a
// multiplier word (MULT: a multiplier, or a packed pair of 16-bit ones).
template <int KIND>
struct KindTraits;
// W: state words per stream; MULT: a per-stream multiplier word; SYNC_ROWS:
// rows between block barriers in the barrier-synced bodies (a multiple of
// four).  Four keeps the warps closest; the two kinds whose steps cost most
// run faster with eight on GB300 (the two-word kinds and KISS slower).
template <>
struct KindTraits<RNG_MWC32> {
    static constexpr int W = 2, SYNC_ROWS = 4;
    static constexpr bool MULT = true;
};
template <>
struct KindTraits<RNG_XOR128> {
    static constexpr int W = 4, SYNC_ROWS = 4;
    static constexpr bool MULT = false;
};
template <>
struct KindTraits<RNG_KISS> {
    static constexpr int W = 4, SYNC_ROWS = 4;
    static constexpr bool MULT = true;
};
template <>
struct KindTraits<RNG_MWC16X2> {
    static constexpr int W = 2, SYNC_ROWS = 4;
    static constexpr bool MULT = true;
};
template <>
struct KindTraits<RNG_XORSHIFT8> {
    static constexpr int W = 8, SYNC_ROWS = 8;
    static constexpr bool MULT = false;
};
template <>
struct KindTraits<RNG_KISS_XOR> {
    static constexpr int W = 4, SYNC_ROWS = 8;
    static constexpr bool MULT = true;
};

// Register arrays hold up to kMaxWords words per stream; a kind touches only
// its first W, and the unused entries cost no registers.
constexpr int kMaxWords = 8;

// One step of stream i of a group of four: w[word][i], a[i].
template <int KIND, int FMT>
__device__ __forceinline__ uint32_t step_enc(uint32_t (&w)[kMaxWords][4],
                                             const uint32_t (&a)[4], int i)
{
    uint32_t u;
    if constexpr (KIND == RNG_MWC32)
        u = mwc_step(a[i], w[0][i], w[1][i]);
    else if constexpr (KIND == RNG_XOR128)
        u = xor128_step(w[0][i], w[1][i], w[2][i], w[3][i]);
    else if constexpr (KIND == RNG_KISS)
        u = kiss_step(a[i], w[0][i], w[1][i], w[2][i], w[3][i]);
    else if constexpr (KIND == RNG_MWC16X2)
        u = mwc16x2_step(a[i], w[0][i], w[1][i]);
    else if constexpr (KIND == RNG_XORSHIFT8)
        u = xorshift8_step(w[0][i], w[1][i], w[2][i], w[3][i], w[4][i], w[5][i], w[6][i],
                           w[7][i]);
    else
        u = kiss_xor_step(a[i], w[0][i], w[1][i], w[2][i], w[3][i]);
    if constexpr (FMT == RNG_F32)
        return __float_as_uint(unit_f32(u));
    else
        return u;  // uint32, or encoded at the store (kFmtMixed)
}

template <int HINT>
__device__ __forceinline__ void store16(uint32_t *p, uint32_t x, uint32_t y, uint32_t z,
                                        uint32_t w)
{
    uint4 v = make_uint4(x, y, z, w);
    if constexpr (HINT == 1)
        __stcs(reinterpret_cast<uint4 *>(p), v);  // streaming: evict-first
    else
        *reinterpret_cast<uint4 *>(p) = v;
}

template <int HINT>
__device__ __forceinline__ void store4(uint32_t *p, uint32_t v)
{
    if constexpr (HINT == 1)
        __stcs(p, v);
    else
        *p = v;
}

// Per-element output format and placement (the batched kernel's mapped
// tiles only).  A map describes a piece of a generator's output sequence
// laid out as one virtual window of consecutive elements (window index i =
// virtual element address - origin) that is stored in segments: segment k
// starts at window index b_k (b_0 = 0), has format f_k (RNG_U32 or
// RNG_F32), and its elements go d_k elements further than their virtual
// address (d_0 = 0; every d_k a multiple of 8, so that a stored chunk keeps
// its 32-byte alignment).  Device layout, 32-bit words:
//   [origin low, origin high, then per segment (b_k, f_k, d_k low, d_k high),
//    then (kFmtEnd, 0, 0, 0)], b_k increasing.
// Each thread keeps a cursor: seek(i) moves to the segment that holds i (i
// never decreases from call to call); seg_at(j) is the segment of element
// j >= the last seek point.  Stores are written as the bodies compute them
// for the virtual window and are placed and encoded here.
struct OutMap {
    uint32_t o = 0;               // low 32 bits of the origin's word address
    const uint32_t *e = nullptr;  // the current segment's entry
    uint32_t nb = kFmtEnd;        // start of the next segment
    int64_t df = 0;               // the current segment's shift, with its format
                                  // in bit 0 (shifts are multiples of 8)

    __device__ __forceinline__ static int64_t df_of(const uint32_t *entry)
    {
        return (int64_t)(((uint64_t)entry[3] << 32) | entry[2]) | (entry[1] & 1u);
    }
    __device__ __forceinline__ void load(const uint32_t *map)
    {
        o = map[0] >> 2 | map[1] << 30;
        e = map + 2;
        df = df_of(e);
        nb = e[4];
    }
    // window index of virtual address p (indices stay below 2^31)
    __device__ __forceinline__ uint32_t index(const uint32_t *p) const
    {
        return (uint32_t)((uintptr_t)p >> 2) - o;
    }
    __device__ __forceinline__ void seek(uint32_t i)
    {
        while (nb <= i && nb != kFmtEnd) {
            e += 4;
            df = df_of(e);
            nb = e[4];
        }
    }
    // Prepares the stores of a row starting at `row`, which fall within
    // window indices [i - 2, i + 4) (the realigned body stores from row - 2
    // to row + 3): true when they all lie in the current segment, so that
    // they can be stored with its shift and format without any lookup; else
    // moves the cursor to the segment of i - 3 for the careful path.
    __device__ __forceinline__ bool row(const uint32_t *row_ptr)
    {
        const uint32_t i = index(row_ptr);
        if (i + 4 < nb)
            return true;
        seek(i > 3 ? i - 3 : 0);
        return false;
    }
    // shift and format of element j >= the last seek point
    __device__ __forceinline__ int64_t seg_at(uint32_t j) const
    {
        int64_t r = df;
        if (j >= nb) {
            const uint32_t *q = e;
            uint32_t v = nb;
            while (v <= j && v != kFmtEnd) {
                q += 4;
                r = df_of(q);
                v = q[4];
            }
        }
        return r;
    }
    __device__ __forceinline__ static uint32_t *place(uint32_t *p, int64_t x)
    {
        return p + (x & ~(int64_t)1);
    }
};

__device__ __forceinline__ uint32_t f32_bits(uint32_t u) { return __float_as_uint(unit_f32(u)); }

// Stores of the bodies: with FMT = kFmtMixed the words arrive as uint32 for
// the virtual window and are placed and encoded here, each by its own
// segment; otherwise they are stored as they are (step_enc encoded them).
template <int FMT, int HINT>
__device__ __forceinline__ void put16(const OutMap &m, bool fast, uint32_t *p, uint32_t x,
                                      uint32_t y, uint32_t z, uint32_t w)
{
    if constexpr (FMT == kFmtMixed) {
        const uint32_t i = fast ? 0u : m.index(p);
        if (fast || i + 3 < m.nb) {  // one segment for all four (the common case)
            if (m.df & 1) {
                x = f32_bits(x);
                y = f32_bits(y);
                z = f32_bits(z);
                w = f32_bits(w);
            }
            store16<HINT>(OutMap::place(p, m.df), x, y, z, w);
        } else {  // a segment starts inside the chunk: word by word (rare;
                  // kept rolled, so that each store site stays small)
#pragma unroll 1
            for (int k = 0; k < 4; ++k) {
                const uint32_t v = k == 0 ? x : k == 1 ? y : k == 2 ? z : w;
                const int64_t dk = m.seg_at(i + k);
                store4<HINT>(OutMap::place(p + k, dk), (dk & 1) ? f32_bits(v) : v);
            }
        }
    } else {
        store16<HINT>(p, x, y, z, w);
    }
}

template <int FMT, int HINT>
__device__ __forceinline__ void put4(const OutMap &m, bool fast, uint32_t *p, uint32_t v)
{
    if constexpr (FMT == kFmtMixed) {
        const int64_t d = fast ? m.df : m.seg_at(m.index(p));
        store4<HINT>(OutMap::place(p, d), (d & 1) ? f32_bits(v) : v);
    } else {
        store4<HINT>(p, v);
    }
}

// 16-byte aligned group load/store of one state word of streams s0..s0+3.
__device__ __forceinline__ void load4(const uint32_t *p, uint32_t (&d)[4])
{
    uint4 q = *reinterpret_cast<const uint4 *>(p);
    d[0] = q.x;
    d[1] = q.y;
    d[2] = q.z;
    d[3] = q.w;
}

__device__ __forceinline__ void save4(uint32_t *p, const uint32_t (&d)[4])
{
    *reinterpret_cast<uint4 *>(p) = make_uint4(d[0], d[1], d[2], d[3]);
}

// Aligned vector body: V groups of four streams starting at s_first +
// v * v_stride (all of them live: the caller checks); row0 points at the
// output element of stream s_first in row 0 (16-byte aligned), and the
// group v outputs sit v * v_stride elements further along each row.
template <int KIND, int FMT, int V, int HINT>
__device__ __forceinline__ void body_vec(uint32_t *__restrict__ state,
                                         const uint32_t *__restrict__ mult, uint64_t n,
                                         uint32_t steps, uint32_t *__restrict__ row0,
                                         uint64_t ld, uint64_t s_first, uint64_t v_stride,
                                         const uint32_t *fmap = nullptr)
{
    constexpr int W = KindTraits<KIND>::W;
    uint32_t w[V][kMaxWords][4];
    uint32_t a[V][4];
    OutMap m;
    if constexpr (FMT == kFmtMixed)
        m.load(fmap);
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const uint64_t s0 = s_first + v_stride * v;
#pragma unroll
        for (int k = 0; k < W; ++k)
            load4(state + k * n + s0, w[v][k]);
        if constexpr (KindTraits<KIND>::MULT)
            load4(mult + s0, a[v]);
        else
            a[v][0] = a[v][1] = a[v][2] = a[v][3] = 0;
    }
    uint32_t *row = row0;
    if constexpr (FMT == kFmtMixed) {
        static_assert(V == 1, "mapped tiles take one group per thread");
        // stretches of rows inside one segment run the plain loop of that
        // segment's format at its shifted place; a row that meets a segment
        // start is stored word by word
        uint32_t j = 0;
        while (j < steps) {
            const uint32_t i = m.index(row);
            uint32_t run = 0;  // rows from j whose four words all lie before nb
            if (i + 3 < m.nb) {
                const uint64_t fit = (m.nb - i - 4) / ld + 1;
                run = fit < steps - j ? (uint32_t)fit : steps - j;
            }
            if (run) {
                uint32_t *q = OutMap::place(row, m.df);
                if (m.df & 1) {
#pragma unroll 4
                    for (uint32_t k = 0; k < run; ++k) {
                        uint32_t o0 = step_enc<KIND, RNG_F32>(w[0], a[0], 0);
                        uint32_t o1 = step_enc<KIND, RNG_F32>(w[0], a[0], 1);
                        uint32_t o2 = step_enc<KIND, RNG_F32>(w[0], a[0], 2);
                        uint32_t o3 = step_enc<KIND, RNG_F32>(w[0], a[0], 3);
                        store16<HINT>(q, o0, o1, o2, o3);
                        q += ld;
                    }
                } else {
#pragma unroll 4
                    for (uint32_t k = 0; k < run; ++k) {
                        uint32_t o0 = step_enc<KIND, RNG_U32>(w[0], a[0], 0);
                        uint32_t o1 = step_enc<KIND, RNG_U32>(w[0], a[0], 1);
                        uint32_t o2 = step_enc<KIND, RNG_U32>(w[0], a[0], 2);
                        uint32_t o3 = step_enc<KIND, RNG_U32>(w[0], a[0], 3);
                        store16<HINT>(q, o0, o1, o2, o3);
                        q += ld;
                    }
                }
                row += (uint64_t)run * ld;
                j += run;
            } else {
                m.seek(i > 3 ? i - 3 : 0);
                uint32_t o0 = step_enc<KIND, FMT>(w[0], a[0], 0);
                uint32_t o1 = step_enc<KIND, FMT>(w[0], a[0], 1);
                uint32_t o2 = step_enc<KIND, FMT>(w[0], a[0], 2);
                uint32_t o3 = step_enc<KIND, FMT>(w[0], a[0], 3);
                put16<FMT, HINT>(m, false, row, o0, o1, o2, o3);
                row += ld;
                ++j;
            }
        }
    } else {
#pragma unroll 4
        for (uint32_t j = 0; j < steps; ++j) {
#pragma unroll
            for (int v = 0; v < V; ++v) {
                uint32_t o0 = step_enc<KIND, FMT>(w[v], a[v], 0);
                uint32_t o1 = step_enc<KIND, FMT>(w[v], a[v], 1);
                uint32_t o2 = step_enc<KIND, FMT>(w[v], a[v], 2);
                uint32_t o3 = step_enc<KIND, FMT>(w[v], a[v], 3);
                store16<HINT>(row + v_stride * v, o0, o1, o2, o3);
            }
            row += ld;
        }
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const uint64_t s0 = s_first + v_stride * v;
#pragma unroll
        for (int k = 0; k < W; ++k)
            save4(state + k * n + s0, w[v][k]);
    }
}

// Aligned vector body for rows that are 16-byte but not 32-byte aligned
// (n % 8 != 0 or a 32-byte misaligned output): one group of four streams per
// thread, and a barrier every SYNC_ROWS rows.  A warp's 512-byte row window then
// begins or ends inside a 32-byte DRAM sector that its neighbour completes;
// keeping the CTA's warps within a few rows of each other lets the two
// halves meet in L2 instead of reaching DRAM as partial sectors (which cost a
// read-modify-write), and keeps the CTA's write stream on a few rows at a
// time (warps storing whole sectors but left to drift ran 16 % slower).  Every thread of the CTA must call this; threads whose
// group is not `live` compute on zero state and store nothing.
template <int KIND, int FMT, int HINT>
__device__ __forceinline__ void body_vec_sync(uint32_t *__restrict__ state,
                                              const uint32_t *__restrict__ mult, uint64_t n,
                                              uint32_t steps, uint32_t *__restrict__ row0,
                                              uint64_t ld, uint64_t s_first, bool live,
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
            load4(state + k * n + s_first, w[k]);
        if constexpr (KindTraits<KIND>::MULT)
            load4(mult + s_first, a);
    }
    uint32_t *row = row0;
    const uint32_t blocks = steps / 4;
    constexpr uint32_t every = KindTraits<KIND>::SYNC_ROWS / 4;  // blocks per barrier
    if constexpr (FMT == kFmtMixed) {  // rolled: the mapped kernels stay small
        for (uint32_t j = 0; j < steps; ++j) {
            if (j % (4 * every) == 0 && j < 4 * blocks)
                __syncthreads();
            uint32_t o0 = step_enc<KIND, FMT>(w, a, 0);
            uint32_t o1 = step_enc<KIND, FMT>(w, a, 1);
            uint32_t o2 = step_enc<KIND, FMT>(w, a, 2);
            uint32_t o3 = step_enc<KIND, FMT>(w, a, 3);
            if (live)
                put16<FMT, HINT>(m, m.row(row), row, o0, o1, o2, o3);
            row += ld;
        }
    } else {
        for (uint32_t b = 0; b < blocks; ++b) {
            if (b % every == 0)
                __syncthreads();
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint32_t o0 = step_enc<KIND, FMT>(w, a, 0);
                uint32_t o1 = step_enc<KIND, FMT>(w, a, 1);
                uint32_t o2 = step_enc<KIND, FMT>(w, a, 2);
                uint32_t o3 = step_enc<KIND, FMT>(w, a, 3);
                if (live)
                    store16<HINT>(row, o0, o1, o2, o3);
                row += ld;
            }
        }
        for (uint32_t j = 4 * blocks; j < steps; ++j) {
            uint32_t o0 = step_enc<KIND, FMT>(w, a, 0);
            uint32_t o1 = step_enc<KIND, FMT>(w, a, 1);
            uint32_t o2 = step_enc<KIND, FMT>(w, a, 2);
            uint32_t o3 = step_enc<KIND, FMT>(w, a, 3);
            if (live)
                store16<HINT>(row, o0, o1, o2, o3);
            row += ld;
        }
    }
    if (live) {
#pragma unroll
        for (int k = 0; k < W; ++k)
            save4(state + k * n + s_first, w[k]);
    }
}

// One row of the realigned body with the row's alignment R (the word
// address of the lane's own first element, mod 4) known at compile time.
// A lane's four words sit at positions R..3 of the aligned chunk C = row - R
// and 0..R-1 of the next chunk C + 4.
//   R = 1, 2: the lane stores chunk C, made of the last R words of lane l-1
//             (shuffled up) and its own first 4-R words ("prev" lanes:
//             l > 0 and live);
//   R = 3:    the lane stores chunk C + 4, made of its own last 3 words and
//             the first word of lane l+1 (shuffled down) ("next" lanes:
//             live, not a halo, and lane l+1 live).
// EDGE warps also store the stray words singly: the CTA's first lane its
// words 0 .. 3-R, the owner of its last group its words 4-R .. 3.
template <int KIND, int FMT, int HINT, int R, bool EDGE>
__device__ __forceinline__ void shift_row(uint32_t (&w)[kMaxWords][4], const uint32_t (&a)[4],
                                          uint32_t *row, bool owner, bool prev, bool next,
                                          bool lead, bool trail, OutMap &m)
{
    bool fast = true;
    if constexpr (FMT == kFmtMixed)
        fast = m.row(row);
    const uint32_t o0 = step_enc<KIND, FMT>(w, a, 0);
    const uint32_t o1 = step_enc<KIND, FMT>(w, a, 1);
    const uint32_t o2 = step_enc<KIND, FMT>(w, a, 2);
    const uint32_t o3 = step_enc<KIND, FMT>(w, a, 3);
    if constexpr (R == 0) {
        if (owner)
            put16<FMT, HINT>(m, fast, row, o0, o1, o2, o3);
    } else {
        if constexpr (R == 1) {
            const uint32_t p3 = __shfl_up_sync(0xffffffffu, o3, 1);
            if (prev)
                put16<FMT, HINT>(m, fast, row - 1, p3, o0, o1, o2);
        } else if constexpr (R == 2) {
            const uint32_t p2 = __shfl_up_sync(0xffffffffu, o2, 1);
            const uint32_t p3 = __shfl_up_sync(0xffffffffu, o3, 1);
            if (prev)
                put16<FMT, HINT>(m, fast, row - 2, p2, p3, o0, o1);
        } else {
            const uint32_t n0 = __shfl_down_sync(0xffffffffu, o0, 1);
            if (next)
                put16<FMT, HINT>(m, fast, row + 1, o1, o2, o3, n0);
        }
        if constexpr (EDGE) {
            if (lead) {
                put4<FMT, HINT>(m, fast, row, o0);
                if constexpr (R <= 2)
                    put4<FMT, HINT>(m, fast, row + 1, o1);
                if constexpr (R == 1)
                    put4<FMT, HINT>(m, fast, row + 2, o2);
            }
            if (trail) {
                if constexpr (R == 3)
                    put4<FMT, HINT>(m, fast, row + 1, o1);
                if constexpr (R >= 2)
                    put4<FMT, HINT>(m, fast, row + 2, o2);
                put4<FMT, HINT>(m, fast, row + 3, o3);
            }
        }
    }
}

// One row of the realigned body on a mapped tile, with the row's alignment
// R chosen at run time (uniform over the CTA): the four steps are written
// once and only the store pattern of shift_row differs by R, so that the
// mapped kernels stay small.
template <int KIND, int HINT>
__device__ __forceinline__ void shift_row_mixed(uint32_t (&w)[kMaxWords][4],
                                                const uint32_t (&a)[4], uint32_t *row, uint32_t r,
                                                bool owner, bool prev, bool next, bool lead,
                                                bool trail, OutMap &m)
{
    constexpr int F = kFmtMixed;
    const bool fast = m.row(row);
    const uint32_t o0 = step_enc<KIND, F>(w, a, 0);
    const uint32_t o1 = step_enc<KIND, F>(w, a, 1);
    const uint32_t o2 = step_enc<KIND, F>(w, a, 2);
    const uint32_t o3 = step_enc<KIND, F>(w, a, 3);
    if (r == 0) {
        if (owner)
            put16<F, HINT>(m, fast, row, o0, o1, o2, o3);
    } else if (r == 1) {
        const uint32_t p3 = __shfl_up_sync(0xffffffffu, o3, 1);
        if (prev)
            put16<F, HINT>(m, fast, row - 1, p3, o0, o1, o2);
        if (lead) {
            put4<F, HINT>(m, fast, row, o0);
            put4<F, HINT>(m, fast, row + 1, o1);
            put4<F, HINT>(m, fast, row + 2, o2);
        }
        if (trail)
            put4<F, HINT>(m, fast, row + 3, o3);
    } else if (r == 2) {
        const uint32_t p2 = __shfl_up_sync(0xffffffffu, o2, 1);
        const uint32_t p3 = __shfl_up_sync(0xffffffffu, o3, 1);
        if (prev)
            put16<F, HINT>(m, fast, row - 2, p2, p3, o0, o1);
        if (lead) {
            put4<F, HINT>(m, fast, row, o0);
            put4<F, HINT>(m, fast, row + 1, o1);
        }
        if (trail) {
            put4<F, HINT>(m, fast, row + 2, o2);
            put4<F, HINT>(m, fast, row + 3, o3);
        }
    } else {
        const uint32_t n0 = __shfl_down_sync(0xffffffffu, o0, 1);
        if (next)
            put16<F, HINT>(m, fast, row + 1, o1, o2, o3, n0);
        if (lead)
            put4<F, HINT>(m, fast, row, o0);
        if (trail) {
            put4<F, HINT>(m, fast, row + 1, o1);
            put4<F, HINT>(m, fast, row + 2, o2);
            put4<F, HINT>(m, fast, row + 3, o3);
        }
    }
}

// Rows in blocks of four: the alignment of row j + 4 equals that of row j,
// so within a block every row's alignment is a compile-time constant.
template <int KIND, int FMT, int HINT, int R0, int DR, bool EDGE>
__device__ __forceinline__ void shift_rows(uint32_t (&w)[kMaxWords][4], const uint32_t (&a)[4],
                                           uint32_t *&row, uint64_t ld, uint32_t blocks,
                                           bool owner, bool prev, bool next, bool lead,
                                           bool trail, OutMap &m)
{
    constexpr uint32_t every = KindTraits<KIND>::SYNC_ROWS / 4;  // blocks per barrier
    for (uint32_t b = 0; b < blocks; ++b) {
        if (b % every == 0)
            __syncthreads();  // keep the CTA's warps within a few rows of each other
        shift_row<KIND, FMT, HINT, R0, EDGE>(w, a, row, owner, prev, next, lead, trail, m);
        row += ld;
        shift_row<KIND, FMT, HINT, (R0 + DR) & 3, EDGE>(w, a, row, owner, prev, next, lead,
                                                        trail, m);
        row += ld;
        shift_row<KIND, FMT, HINT, (R0 + 2 * DR) & 3, EDGE>(w, a, row, owner, prev, next,
                                                            lead, trail, m);
        row += ld;
        shift_row<KIND, FMT, HINT, (R0 + 3 * DR) & 3, EDGE>(w, a, row, owner, prev, next,
                                                            lead, trail, m);
        row += ld;
    }
}

// One row with a run-time alignment (the at most three rows after the
// blocks of four).
template <int KIND, int FMT, int HINT>
__device__ __forceinline__ void shift_row_rt(uint32_t (&w)[kMaxWords][4], const uint32_t (&a)[4],
                                             uint32_t *row, uint32_t r, bool owner, bool prev,
                                             bool next, bool lead, bool trail, OutMap &m)
{
    switch (r) {
    case 0: shift_row<KIND, FMT, HINT, 0, true>(w, a, row, owner, prev, next, lead, trail, m); break;
    case 1: shift_row<KIND, FMT, HINT, 1, true>(w, a, row, owner, prev, next, lead, trail, m); break;
    case 2: shift_row<KIND, FMT, HINT, 2, true>(w, a, row, owner, prev, next, lead, trail, m); break;
    default: shift_row<KIND, FMT, HINT, 3, true>(w, a, row, owner, prev, next, lead, trail, m); break;
    }
}

template <int KIND, int FMT, int HINT, bool EDGE>
__device__ __forceinline__ void shift_rows_dispatch(uint32_t (&w)[kMaxWords][4], const uint32_t (&a)[4],
                                                    uint32_t *&row, uint64_t ld, uint32_t r0,
                                                    uint32_t blocks, bool owner, bool prev,
                                                    bool next, bool lead, bool trail, OutMap &m)
{
    const uint32_t dr = (uint32_t)(ld & 3);
    if constexpr (FMT == kFmtMixed) {
        // mapped tiles run row by row with the row phase chosen at run time
        // (a uniform branch): one small copy of the row per phase keeps the
        // mapped kernels within the instruction cache
        constexpr uint32_t every = KindTraits<KIND>::SYNC_ROWS / 4;
        uint32_t r = r0;
        for (uint32_t b = 0; b < blocks; ++b) {
            if (b % every == 0)
                __syncthreads();
#pragma unroll 1
            for (int q = 0; q < 4; ++q) {
                shift_row_mixed<KIND, HINT>(w, a, row, r, owner, prev, next, lead, trail, m);
                row += ld;
                r = (r + dr) & 3u;
            }
        }
        return;
    }
#define GBRNG_SHIFT_CASE(R0_, DR_)                                                            \
    case (R0_) * 4 + (DR_):                                                                   \
        shift_rows<KIND, FMT, HINT, R0_, DR_, EDGE>(w, a, row, ld, blocks, owner, prev, next, \
                                                    lead, trail, m);                          \
        break;
    switch (r0 * 4 + dr) {
        GBRNG_SHIFT_CASE(0, 0) GBRNG_SHIFT_CASE(0, 1) GBRNG_SHIFT_CASE(0, 2) GBRNG_SHIFT_CASE(0, 3)
        GBRNG_SHIFT_CASE(1, 0) GBRNG_SHIFT_CASE(1, 1) GBRNG_SHIFT_CASE(1, 2) GBRNG_SHIFT_CASE(1, 3)
        GBRNG_SHIFT_CASE(2, 0) GBRNG_SHIFT_CASE(2, 1) GBRNG_SHIFT_CASE(2, 2) GBRNG_SHIFT_CASE(2, 3)
        GBRNG_SHIFT_CASE(3, 0) GBRNG_SHIFT_CASE(3, 1) GBRNG_SHIFT_CASE(3, 2) GBRNG_SHIFT_CASE(3, 3)
    default: break;
    }
#undef GBRNG_SHIFT_CASE
}

// Realigned vector body, for rows that are not 16-byte aligned.  The CTA
// (K = blockDim.x / 32 warps, every thread must call this) covers up to
// 31K + 1 groups of four consecutive streams, starting at stream cta_s0
// whose output element in row 0 is cta_row0; `groups` of them are live.
// Lane l of warp k holds group g = 31k + l, so lane 31 of a warp other than
// the last holds the first group of the next warp as well: a halo, stepped
// from the same starting state but never written back.  Every warp's first
// element is 124 words after the previous warp's, so all warps see the same
// row alignment, and a warp's halo lane writes the chunk that straddles the
// warp boundary (shift_row); only the CTA's first lane and the owner of its
// last group store stray words singly.  The barrier after the state loads
// keeps every halo read ahead of the owner's write-back, and one every
// SYNC_ROWS rows keeps the warps together (see body_vec_sync): every warp runs the
// rows, idle lanes storing nothing.
template <int KIND, int FMT, int HINT>
__device__ __forceinline__ void body_shift(uint32_t *__restrict__ state,
                                           const uint32_t *__restrict__ mult, uint64_t n,
                                           uint32_t steps, uint32_t *__restrict__ cta_row0,
                                           uint64_t ld, uint64_t cta_s0, uint32_t groups,
                                           const uint32_t *fmap = nullptr)
{
    constexpr int W = KindTraits<KIND>::W;
    const int lane = threadIdx.x & 31;
    const int k = threadIdx.x >> 5;
    const int K = blockDim.x >> 5;
    const uint32_t g = 31u * k + lane;
    const bool live = g < groups;
    const bool owner = live && (lane < 31 || k == K - 1);
    const bool lead = (g == 0);                   // the CTA's first lane
    const bool trail = owner && g == groups - 1;  // owner of the CTA's last group
    const bool prev = live && lane > 0;                              // chunk C
    const bool next = owner && lane < 31 && g + 1 < groups;          // chunk C + 4
    const uint64_t s_first = cta_s0 + 4 * (uint64_t)g;
    uint32_t w[kMaxWords][4];
    uint32_t a[4];
    OutMap m;
    if constexpr (FMT == kFmtMixed)
        m.load(fmap);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        a[i] = 0;
#pragma unroll
        for (int q = 0; q < kMaxWords; ++q)
            w[q][i] = 0;
    }
    if (live) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
#pragma unroll
            for (int q = 0; q < W; ++q)
                w[q][i] = state[q * n + s_first + i];
            if constexpr (KindTraits<KIND>::MULT)
                a[i] = mult[s_first + i];
        }
    }
    __syncthreads();  // every halo state is read before any write-back
    const bool warp_edge = __any_sync(0xffffffffu, lead || trail);
    {  // every warp runs the rows (idle lanes store nothing): all reach every barrier
        uint32_t *row = cta_row0 + 4 * (uint64_t)g;
        const uint32_t r0 = (uint32_t)((uintptr_t)cta_row0 >> 2) & 3u;
        const uint32_t blocks = steps / 4;
        if (warp_edge)
            shift_rows_dispatch<KIND, FMT, HINT, true>(w, a, row, ld, r0, blocks, owner, prev,
                                                       next, lead, trail, m);
        else
            shift_rows_dispatch<KIND, FMT, HINT, false>(w, a, row, ld, r0, blocks, owner, prev,
                                                        next, lead, trail, m);
        uint32_t r = r0;  // rows 4*blocks.. keep the alignment of row 0 shifted by 4*dr == 0
        for (uint32_t j = 4 * blocks; j < steps; ++j) {
            if constexpr (FMT == kFmtMixed)
                shift_row_mixed<KIND, HINT>(w, a, row, r, owner, prev, next, lead, trail, m);
            else
                shift_row_rt<KIND, FMT, HINT>(w, a, row, r, owner, prev, next, lead, trail, m);
            row += ld;
            r = (r + (uint32_t)(ld & 3)) & 3u;
        }
    }
    if (owner) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int q = 0; q < W; ++q)
                state[q * n + s_first + i] = w[q][i];
    }
}

// Scalar body: one stream s (< n), 4-byte stores from p0 (its element in
// row 0); any n, 4-byte aligned output.
template <int KIND, int FMT, int HINT>
__device__ __forceinline__ void body_scalar(uint32_t *__restrict__ state,
                                            const uint32_t *__restrict__ mult, uint64_t n,
                                            uint32_t steps, uint32_t *__restrict__ p0,
                                            uint64_t ld, uint64_t s,
                                            const uint32_t *fmap = nullptr)
{
    constexpr int W = KindTraits<KIND>::W;
    uint32_t w[kMaxWords][4];
    uint32_t a[4] = {0, 0, 0, 0};
    OutMap m;
    if constexpr (FMT == kFmtMixed)
        m.load(fmap);
#pragma unroll
    for (int k = 0; k < kMaxWords; ++k)
        w[k][0] = k < W ? state[k * n + s] : 0;
    if constexpr (KindTraits<KIND>::MULT)
        a[0] = mult[s];
    uint32_t *p = p0;
    if constexpr (FMT == kFmtMixed) {  // rolled: the mapped kernels stay small
#pragma unroll 1
        for (uint32_t j = 0; j < steps; ++j) {
            const uint32_t o = step_enc<KIND, FMT>(w, a, 0);
            put4<FMT, HINT>(m, m.row(p), p, o);
            p += ld;
        }
    } else {
#pragma unroll 4
        for (uint32_t j = 0; j < steps; ++j) {
            store4<HINT>(p, step_enc<KIND, FMT>(w, a, 0));
            p += ld;
        }
    }
#pragma unroll
    for (int k = 0; k < W; ++k)
        state[k * n + s] = w[k][0];
}

}  // namespace gbrng
