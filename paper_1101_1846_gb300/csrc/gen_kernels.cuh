// The generation kernels, templated on the generator kind, and
// launch_kind<KIND>, which picks the kernel for a call.  Included by the
// translation units that instantiate them (generate.cu: the three target
// kinds; generate_paper.cu: the paper's own generators), so that each one
// compiles only its kinds.
//
// Every thread keeps the state of its streams in
// registers for the whole call, steps them n times and writes each step's
// outputs with one 16-byte store per group of four adjacent streams, so a
// warp writes 512 contiguous bytes of one output row per store instruction.
// The paper's kernels (Sec. "GPU implementations": MWC, XorShift in
// registers, KISS) keep one stream per thread with 4-byte stores; four
// streams per thread give the 16-byte stores and four independent
// dependency chains per thread.
//
// Layout: output j of stream s at out[j*ld + s] (ld = n_streams for a plain
// call); state word w of stream s at state[w*n + s].
//
// Paths (chosen per call by launch_kind):
//   aligned  n % 4 == 0 and out 16-byte aligned: gen_vec when every row is
//            32-byte aligned (a CTA of B threads covers 4*V*B consecutive
//            streams, thread t owns the groups starting at base + 4t + 4Bv,
//            v < V), else gen_vec_sync (one group per thread, barriers);
//   shifted  otherwise, for the first n & ~3 streams: gen_shift, rows written
//            with 16-byte stores after a warp-shuffle realignment;
//   tail     the last n % 4 streams, taken by one extra CTA of gen_shift with
//            4-byte stores.
#pragma once

#include <algorithm>

#include "gen_body.cuh"
#include "jump.cuh"

namespace gbrng {
namespace {

// Streams [s_begin, s_begin + count) of the generator; out points at the
// output element of stream s_begin in row 0.
template <int KIND, int FMT, int V, int HINT>
__global__ void __launch_bounds__(512)
gen_vec(uint32_t *__restrict__ state, const uint32_t *__restrict__ mult, uint64_t n,
        uint32_t steps, uint32_t *__restrict__ out, uint64_t ld, uint64_t s_begin,
        uint64_t count)
{
    const uint64_t B = blockDim.x;
    const uint64_t c_first = (uint64_t)blockIdx.x * (4 * V) * B + 4 * (uint64_t)threadIdx.x;
    if (V == 2 && c_first + 4 * B < count)
        body_vec<KIND, FMT, V, HINT>(state, mult, n, steps, out + c_first, ld,
                                     s_begin + c_first, 4 * B);
    else if (c_first < count)
        body_vec<KIND, FMT, 1, HINT>(state, mult, n, steps, out + c_first, ld,
                                     s_begin + c_first, 4 * B);
}

// Rows 16-byte but not 32-byte aligned: one group per thread, barriers every
// SYNC_ROWS rows; every thread runs the rows (idle groups store nothing).
template <int KIND, int FMT, int HINT>
__global__ void __launch_bounds__(512)
gen_vec_sync(uint32_t *__restrict__ state, const uint32_t *__restrict__ mult, uint64_t n,
             uint32_t steps, uint32_t *__restrict__ out, uint64_t ld, uint64_t s_begin,
             uint64_t count)
{
    const uint64_t c_first = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    body_vec_sync<KIND, FMT, HINT>(state, mult, n, steps, out + c_first, ld, s_begin + c_first,
                                   c_first < count);
}

// The first count & ~3 streams in realigned groups of four, 31K + 1 groups
// per CTA of K warps (see body_shift); the last CTA of the grid takes the
// count % 4 tail streams (one per thread), so that they run alongside the
// rest instead of after it.
template <int KIND, int FMT, int HINT>
__global__ void __launch_bounds__(512)
gen_shift(uint32_t *__restrict__ state, const uint32_t *__restrict__ mult, uint64_t n,
          uint32_t steps, uint32_t *__restrict__ out, uint64_t ld, uint64_t s_begin,
          uint64_t count)
{
    const uint64_t main = count & ~(uint64_t)3;
    if (main < count && blockIdx.x == gridDim.x - 1) {
        uint64_t c = main + threadIdx.x;
        if (c < count)
            body_scalar<KIND, FMT, HINT>(state, mult, n, steps, out + c, ld, s_begin + c);
        return;
    }
    const uint64_t per_cta = 31 * (blockDim.x / 32) + 1;
    const uint64_t g0 = (uint64_t)blockIdx.x * per_cta;
    const uint64_t left = main / 4 - g0;
    body_shift<KIND, FMT, HINT>(state, mult, n, steps, out + 4 * g0, ld, s_begin + 4 * g0,
                                (uint32_t)(left < per_cta ? left : per_cta));
}

// Sequence splitting (Sec. "Parallelizing RNGs") for calls with too few
// streams to fill the device: segment y of the grid produces rows
// [y*rows, min(steps, (y+1)*rows)) of every stream, starting from the state
// jumped ahead by y*rows steps (the MWC part by the handle's tabulated
// multiplier a^(y*rows), the xorshift and LCG parts by the device tables).
// One group of four streams per thread, rows 32-byte aligned (as gen_vec).
//
// Writing the final state back must wait until every segment has read the
// start state, and no segment may wait for another.  So each thread counts
// its arrival on the group's counter right after reading the start state;
// the last segment also stashes its final state and counts once more.  The
// arrival that brings the count to segments + 1 sees every read done and the
// final state ready: it writes the state (from registers or the stash) and
// clears the counter for the next call.
//
// SYNC: rows 16- but not 32-byte aligned.  As in body_vec_sync, a barrier
// every SYNC_ROWS rows keeps the CTA's warps together so that the two halves of
// a shared DRAM sector meet in L2; every thread of the CTA then runs the
// rows (a CTA shares its segment, hence its jump and its row count), and
// threads past the last group store nothing and count no arrival.
template <int KIND, int FMT, int HINT, bool SYNC>
__global__ void __launch_bounds__(256)
gen_split(uint32_t *__restrict__ state, const uint32_t *__restrict__ mult, uint64_t n,
          uint32_t steps, uint32_t rows, uint32_t *__restrict__ out, uint64_t ld,
          uint64_t s_begin, uint64_t count, uint32_t *__restrict__ stash,
          uint32_t *__restrict__ counters, const uint64_t *__restrict__ jmul, JumpTables T)
{
    uint64_t c_first = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    const bool live = c_first < count;
    if (!SYNC && !live)
        return;
    if (!live)
        c_first = 0;  // compute on stream 0's state, never store
    constexpr int W = KindTraits<KIND>::W;
    const uint64_t s0 = s_begin + c_first;
    const uint32_t segs = gridDim.y;
    const uint32_t y = blockIdx.y;
    const uint32_t first = y * rows;
    const uint32_t mine = min(rows, steps - first);
    uint32_t w[kMaxWords][4] = {};
    uint32_t a[4] = {};
#pragma unroll
    for (int k = 0; k < W; ++k)
        load4(state + k * n + s0, w[k]);
    if constexpr (KindTraits<KIND>::MULT)
        load4(mult + s0, a);
    __threadfence();  // the reads above are done before the arrival is counted
    uint32_t *cnt = counters + s0 / 4;
    const bool finish = live && atomicAdd(cnt, 1u) == segs;
    if (finish) {
        // every other arrival, the stash included, came first
        __threadfence();
#pragma unroll
        for (int k = 0; k < W; ++k) {
            const uint4 q = __ldcg(reinterpret_cast<const uint4 *>(stash + k * n + s0));
            *reinterpret_cast<uint4 *>(state + k * n + s0) = q;
        }
        *cnt = 0;
    }
    if (y > 0) {
        // MWC32 / KISS: the tabulated a^(y*rows) when the handle's table is
        // passed, else powering (calls captured in a CUDA graph)
        bool mwc_done = false;
        if constexpr (KIND == RNG_MWC32 || KIND == RNG_KISS) {
            if (jmul) {
                const uint4 lo =
                    __ldg(reinterpret_cast<const uint4 *>(jmul + (uint64_t)y * n + s0));
                const uint4 hi =
                    __ldg(reinterpret_cast<const uint4 *>(jmul + (uint64_t)y * n + s0 + 2));
                const uint64_t A[4] = {(uint64_t)lo.y << 32 | lo.x, (uint64_t)lo.w << 32 | lo.z,
                                       (uint64_t)hi.y << 32 | hi.x, (uint64_t)hi.w << 32 | hi.z};
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    mwc_apply(A[i], a[i], w[0][i], w[1][i]);
                mwc_done = true;
            }
        }
        if (mwc_done)
            jump_streams<KIND, 4, true>(w, a, first, T);
        else
            jump_streams<KIND, 4, false>(w, a, first, T);
    }
    uint32_t *row = out + (uint64_t)first * ld + c_first;
    if constexpr (SYNC) {
        for (uint32_t j = 0; j < mine; ++j) {
            if (j % KindTraits<KIND>::SYNC_ROWS == 0)
                __syncthreads();
            const uint32_t o0 = step_enc<KIND, FMT>(w, a, 0);
            const uint32_t o1 = step_enc<KIND, FMT>(w, a, 1);
            const uint32_t o2 = step_enc<KIND, FMT>(w, a, 2);
            const uint32_t o3 = step_enc<KIND, FMT>(w, a, 3);
            if (live)
                store16<HINT>(row, o0, o1, o2, o3);
            row += ld;
        }
        if (!live)
            return;  // after the last barrier
    } else {
#pragma unroll 4
        for (uint32_t j = 0; j < mine; ++j) {
            const uint32_t o0 = step_enc<KIND, FMT>(w, a, 0);
            const uint32_t o1 = step_enc<KIND, FMT>(w, a, 1);
            const uint32_t o2 = step_enc<KIND, FMT>(w, a, 2);
            const uint32_t o3 = step_enc<KIND, FMT>(w, a, 3);
            store16<HINT>(row, o0, o1, o2, o3);
            row += ld;
        }
    }
    if (y == segs - 1) {
#pragma unroll
        for (int k = 0; k < W; ++k)
            save4(stash + k * n + s0, w[k]);
        __threadfence();  // the stash is visible before its arrival is counted
        if (atomicAdd(cnt, 1u) == segs) {
#pragma unroll
            for (int k = 0; k < W; ++k)
                save4(state + k * n + s0, w[k]);
            *cnt = 0;
        }
    }
}

// Rows 32-byte aligned, outputs staged in shared memory and written by the
// TMA engine (bulk asynchronous copies, shared -> global): a CTA of
// kTmaThreads threads owns 4 * kTmaThreads consecutive streams (one group
// of four per thread), generates kTmaRows rows at a time into one of two
// shared buffers, and one thread writes each row's segment (4 KB for 1024
// streams) with one bulk copy.  A buffer is refilled only after its
// copies have finished reading it (wait_group.read), and the kernel waits
// for every copy before it ends.  Threads past the last stream run the rows
// with the others (the barriers are CTA-wide) and their words are not
// copied.
constexpr int kTmaThreads = 256;
constexpr int kTmaRows = 4;

__device__ __forceinline__ void tma_store_row(uint32_t *gdst, const uint32_t *ssrc,
                                              uint32_t bytes)
{
    const uint32_t saddr = static_cast<uint32_t>(__cvta_generic_to_shared(ssrc));
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;"
                 :
                 : "l"(gdst), "r"(saddr), "r"(bytes)
                 : "memory");
}

template <int KIND, int FMT>
__global__ void __launch_bounds__(kTmaThreads)
gen_tma(uint32_t *__restrict__ state, const uint32_t *__restrict__ mult, uint64_t n,
        uint32_t steps, uint32_t *__restrict__ out, uint64_t ld, uint64_t s_begin,
        uint64_t count)
{
    __shared__ __align__(128) uint32_t buf[2][kTmaRows][4 * kTmaThreads];
    constexpr int W = KindTraits<KIND>::W;
    const uint64_t c0 = (uint64_t)blockIdx.x * 4 * kTmaThreads;  // CTA's first stream
    const uint64_t c_first = c0 + 4 * (uint64_t)threadIdx.x;
    const bool live = c_first < count;
    const uint32_t bytes = (uint32_t)(4 * min((uint64_t)4 * kTmaThreads, count - c0));
    const uint64_t s0 = s_begin + c_first;
    uint32_t w[kMaxWords][4] = {};
    uint32_t a[4] = {};
    if (live) {
#pragma unroll
        for (int k = 0; k < W; ++k)
            load4(state + k * n + s0, w[k]);
        if constexpr (KindTraits<KIND>::MULT)
            load4(mult + s0, a);
    }
    const bool leader = threadIdx.x == 0;
    uint32_t row0 = 0;
    for (int b = 0; row0 < steps; b ^= 1, row0 += kTmaRows) {
        const uint32_t rows = min((uint32_t)kTmaRows, steps - row0);
        if (leader)  // the copies that read this buffer two blocks ago are done
            asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
        __syncthreads();
        for (uint32_t r = 0; r < rows; ++r) {
            const uint32_t o0 = step_enc<KIND, FMT>(w, a, 0);
            const uint32_t o1 = step_enc<KIND, FMT>(w, a, 1);
            const uint32_t o2 = step_enc<KIND, FMT>(w, a, 2);
            const uint32_t o3 = step_enc<KIND, FMT>(w, a, 3);
            *reinterpret_cast<uint4 *>(&buf[b][r][4 * threadIdx.x]) = make_uint4(o0, o1, o2, o3);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (leader) {
            for (uint32_t r = 0; r < rows; ++r)
                tma_store_row(out + (uint64_t)(row0 + r) * ld + c0, &buf[b][r][0], bytes);
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        }
    }
    if (leader)
        asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    if (live) {
#pragma unroll
        for (int k = 0; k < W; ++k)
            save4(state + k * n + s0, w[k]);
    }
}

constexpr int kSMs = 152;
// CTA size of the kernels with row barriers: large CTAs leave fewer CTA
// boundaries, where neighbouring CTAs that drift apart split sectors.
constexpr int kSyncBlock = 512;

// CTA size for `units` thread-sized pieces of work: shrink until the grid
// covers every SM (small problems), never below one warp.
inline int fit_threads(int threads, uint64_t units)
{
    while (threads > 32 && (units + threads - 1) / threads < kSMs)
        threads /= 2;
    return threads;
}

// V = 2 only for kinds of at most four state words: two groups of the
// eight-word XORSHIFT8 would not fit the registers of a 512-thread CTA.
template <int KIND, int FMT>
void pick_vec(int v, int hint,
              void (*&vec)(uint32_t *, const uint32_t *, uint64_t, uint32_t, uint32_t *,
                           uint64_t, uint64_t, uint64_t))
{
    if constexpr (KindTraits<KIND>::W <= 4) {
        if (v == 2) {
            vec = hint ? gen_vec<KIND, FMT, 2, 1> : gen_vec<KIND, FMT, 2, 0>;
            return;
        }
    }
    vec = hint ? gen_vec<KIND, FMT, 1, 1> : gen_vec<KIND, FMT, 1, 0>;
}

// One generate call of a KIND generator: picks the path from how the rows
// sit in memory (aligned / synced / realigned), or splits a few-stream call
// into jumped segments.
template <int KIND>
int launch_kind(int fmt, const GenLaunch &p, cudaStream_t st)
{
    using Fn = void (*)(uint32_t *, const uint32_t *, uint64_t, uint32_t, uint32_t *, uint64_t,
                        uint64_t, uint64_t);
    const uint64_t count = p.s_end - p.s_begin;
    if (p.steps == 0 || count == 0)
        return RNG_OK;
    const LaunchShape sh = launch_shape(KIND, fmt, count);
    Fn vec, shift, sync;
    if (fmt == RNG_F32) {
        pick_vec<KIND, RNG_F32>(sh.v, sh.hint, vec);
        shift = sh.hint ? gen_shift<KIND, RNG_F32, 1> : gen_shift<KIND, RNG_F32, 0>;
        sync = sh.hint ? gen_vec_sync<KIND, RNG_F32, 1> : gen_vec_sync<KIND, RNG_F32, 0>;
    } else {
        pick_vec<KIND, RNG_U32>(sh.v, sh.hint, vec);
        shift = sh.hint ? gen_shift<KIND, RNG_U32, 1> : gen_shift<KIND, RNG_U32, 0>;
        sync = sh.hint ? gen_vec_sync<KIND, RNG_U32, 1> : gen_vec_sync<KIND, RNG_U32, 0>;
    }
    // 16-byte rows and 16-byte state groups: every group of four streams
    // starts on a 16-byte boundary in the output and in the state words.
    const bool aligned = (count % 4 == 0) && (p.ld % 4 == 0) && ((uintptr_t)p.out % 16 == 0) &&
                         (p.n % 4 == 0) && (p.s_begin % 4 == 0) &&
                         ((uintptr_t)p.state % 16 == 0) &&
                         (p.a == nullptr || (uintptr_t)p.a % 16 == 0);
    // whole 32-byte sectors per warp and row: no barriers needed
    const bool sectors = aligned && (p.ld % 8 == 0) && ((uintptr_t)p.out % 32 == 0);
    const uint64_t main = count & ~(uint64_t)3;
    uint32_t *out = static_cast<uint32_t *>(p.out);
    uint64_t L = 0, S = 0;
    Gen *g = p.owner;
    if (g && g->d_split && aligned &&
        split_plan(KIND, count, p.steps, 4, g->jmul_segs, split_fill(false), &L, &S)) {
        JumpTables T{};
        const uint64_t *jmul = nullptr;
        int e = needs_jump_tables(KIND) ? jump_tables(&T) : RNG_OK;
        // Inside a CUDA graph capture the table is not (re)built: its kernel
        // would only run at replay while later direct calls took it as ready.
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        if (!e)
            e = cuda_status(cudaStreamIsCapturing(st, &cap));
        if (!e && mont_table(KIND) && cap == cudaStreamCaptureStatusNone)
            e = mwc_jump_table(g, L, S, st, &jmul);
        if (e)
            return e;
        using SplitFn = void (*)(uint32_t *, const uint32_t *, uint64_t, uint32_t, uint32_t,
                                 uint32_t *, uint64_t, uint64_t, uint64_t, uint32_t *,
                                 uint32_t *, const uint64_t *, JumpTables);
        SplitFn fn;
        if (sectors)
            fn = fmt == RNG_F32 ? (sh.hint ? gen_split<KIND, RNG_F32, 1, false>
                                           : gen_split<KIND, RNG_F32, 0, false>)
                                : (sh.hint ? gen_split<KIND, RNG_U32, 1, false>
                                           : gen_split<KIND, RNG_U32, 0, false>);
        else
            fn = fmt == RNG_F32 ? (sh.hint ? gen_split<KIND, RNG_F32, 1, true>
                                           : gen_split<KIND, RNG_F32, 0, true>)
                                : (sh.hint ? gen_split<KIND, RNG_U32, 1, true>
                                           : gen_split<KIND, RNG_U32, 0, true>);
        const dim3 grid((unsigned)((count / 4 + 255) / 256), (unsigned)S);
        fn<<<grid, 256, 0, st>>>(p.state, p.a, p.n, (uint32_t)p.steps, (uint32_t)L, out, p.ld,
                                 p.s_begin, count, g->d_split, g->d_cnt, jmul, T);
        return cuda_status(cudaGetLastError());
    }
    // Calls longer than 2^31 steps are cut into pieces (the kernels count
    // steps in 32 bits); the state carries from piece to piece.
    for (uint64_t done = 0; done < p.steps;) {
        const uint32_t steps = (uint32_t)std::min<uint64_t>(p.steps - done, 1u << 31);
        uint32_t *o = out + done * p.ld;
        if (aligned && !sectors) {
            int threads = fit_threads(kSyncBlock, count / 4);
            uint64_t blocks = (count / 4 + threads - 1) / threads;
            if (blocks > 0x7FFFFFFFull)
                return set_error(RNG_ERR_ARG);
            const int smem = row_ctas(KIND, fmt, false) && threads == kSyncBlock
                                 ? one_cta_smem((const void *)sync, threads)
                                 : 0;
            sync<<<(unsigned)blocks, threads, smem, st>>>(p.state, p.a, p.n, steps, o, p.ld,
                                                          p.s_begin, count);
        } else if (aligned && sh.hint == 2) {
            // outputs staged in shared memory, rows written by bulk copies
            const uint64_t blocks = (count + 4 * kTmaThreads - 1) / (4 * kTmaThreads);
            if (blocks > 0x7FFFFFFFull)
                return set_error(RNG_ERR_ARG);
            auto tma = fmt == RNG_F32 ? gen_tma<KIND, RNG_F32> : gen_tma<KIND, RNG_U32>;
            tma<<<(unsigned)blocks, kTmaThreads, 0, st>>>(p.state, p.a, p.n, steps, o, p.ld,
                                                          p.s_begin, count);
        } else if (aligned) {
            int threads = sh.block;
            uint64_t groups = count / 4;
            while (threads > 32 && (groups + (uint64_t)threads * sh.v - 1) /
                                           ((uint64_t)threads * sh.v) < kSMs)
                threads /= 2;
            uint64_t per_block = (uint64_t)threads * sh.v;
            uint64_t blocks = (groups + per_block - 1) / per_block;
            if (blocks > 0x7FFFFFFFull)
                return set_error(RNG_ERR_ARG);
            // one CTA per SM only for the shape's own CTA size (small calls
            // halve it above to fill the SMs)
            const int smem =
                sh.one && threads == sh.block ? one_cta_smem((const void *)vec, threads) : 0;
            vec<<<(unsigned)blocks, threads, smem, st>>>(p.state, p.a, p.n, steps, o, p.ld,
                                                         p.s_begin, count);
        } else {
            // realigned groups plus, when count % 4 != 0, one more CTA for the tail
            int threads = fit_threads(kSyncBlock, main / 4);
            const uint64_t per_cta = 31 * (threads / 32) + 1;
            uint64_t blocks = (main / 4 + per_cta - 1) / per_cta + (count > main ? 1 : 0);
            if (blocks > 0x7FFFFFFFull)
                return set_error(RNG_ERR_ARG);
            const int smem = row_ctas(KIND, fmt, true) && threads == kSyncBlock
                                 ? one_cta_smem((const void *)shift, threads)
                                 : 0;
            shift<<<(unsigned)blocks, threads, smem, st>>>(p.state, p.a, p.n, steps, o, p.ld,
                                                           p.s_begin, count);
        }
        int e = cuda_status(cudaGetLastError());
        if (e)
            return e;
        done += steps;
    }
    return RNG_OK;
}

}  // namespace
}  // namespace gbrng
