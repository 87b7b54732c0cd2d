// Inline consumers (rng_generate_reduce): every stream advances exactly as
// in rng_generate, each output is consumed in registers where it is made,
// and only one 64-bit result per stream and the final state are written.
// This is the paper's second regime, generation without writing the numbers
// back (Sec. "Performance evaluation"; Tables I-III), with the numbers
// actually used so that no step can be optimised away.  The kernels step
// the streams through Engine<KIND> of the public device header, the same
// path a user kernel takes.
//
// One stream per thread, loaded with coalesced 4-byte accesses across the
// warp.  Few streams with long sequences are split into segments of 2^l
// rows (split_plan; grid y = segment) that start from jumped states; their
// results are added into out with 64-bit atomics (exact, in any order), and
// the final state is written back by the last arrival, as in gen_split.
#include "jump.cuh"

namespace gbrng {
namespace {

constexpr int kThreads = 256;

// The sums run in chunks of up to 2^30 outputs with a 32-bit counter and an
// unroll of 32: loop bookkeeping then costs little beside the step (the MWC
// sum measured 11 % faster on GB300 than with a 64-bit counter and an
// unroll of 8; the other kinds were unchanged).
template <int OP, int KIND>
__device__ __forceinline__ uint64_t consume(Engine<KIND> &e, uint64_t m)
{
    uint64_t acc = 0;
    if constexpr (OP == RNG_SUM_U32 || OP == RNG_SUM_U24) {
        for (uint64_t done = 0; done < m;) {
            const uint32_t k = (uint32_t)(m - done < (1u << 30) ? m - done : (1u << 30));
#pragma unroll 32
            for (uint32_t j = 0; j < k; ++j) {
                if constexpr (OP == RNG_SUM_U32)
                    acc += e.next();
                else
                    acc += e.next() >> 8;
            }
            done += k;
        }
    } else {
        // pairs (u0, u1): inside when (u0>>8)^2 + (u1>>8)^2 < 2^48
#pragma unroll 4
        for (uint64_t j = 1; j < m; j += 2) {
            const uint64_t X = e.next() >> 8;
            const uint64_t Y = e.next() >> 8;
            acc += (X * X + Y * Y) >> 48 == 0 ? 1u : 0u;
        }
        if (m & 1)
            e.next();  // the unpaired last output is drawn and ignored
    }
    return acc;
}

// SPLIT = false: one segment (grid y = 1), the whole call per thread.
template <int KIND, int OP, bool SPLIT>
__global__ void __launch_bounds__(kThreads)
reduce_kernel(rng_device_view v, uint64_t steps, uint64_t rows, uint64_t *__restrict__ out,
              uint32_t *__restrict__ stash, uint32_t *__restrict__ counters,
              const uint64_t *__restrict__ jmul, JumpTables T)
{
    const uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= v.n_streams)
        return;
    Engine<KIND> e;
    e.load(v, s);
    if constexpr (!SPLIT) {
        out[s] = consume<OP>(e, steps);
        e.store(v, s);
        return;
    }
    // Split: the same arrival count as gen_split (one counter per stream).
    const uint32_t segs = gridDim.y;
    const uint64_t n = v.n_streams;
    uint32_t *state = static_cast<uint32_t *>(v.state);
    __threadfence();
    uint32_t *cnt = counters + s;
    if (atomicAdd(cnt, 1u) == segs) {
        __threadfence();
        for (int k = 0; k < v.state_words; ++k)
            state[k * n + s] = __ldcg(stash + k * n + s);
        *cnt = 0;
    }
    const uint64_t first = (uint64_t)blockIdx.y * rows;
    const uint64_t mine = steps - first < rows ? steps - first : rows;
    const uint64_t A = ((KIND == RNG_MWC32 || KIND == RNG_KISS) && blockIdx.y > 0 && jmul)
                           ? jmul[blockIdx.y * n + s]
                           : 0;
    jump_engine<KIND>(e, first, T, A);
    atomicAdd(reinterpret_cast<unsigned long long *>(out + s),
              (unsigned long long)consume<OP>(e, mine));
    if (blockIdx.y == segs - 1) {
        rng_device_view f = v;
        f.state = stash;
        e.store(f, s);
        __threadfence();
        if (atomicAdd(cnt, 1u) == segs) {
            e.store(v, s);
            *cnt = 0;
        }
    }
}

using ReduceFn = void (*)(rng_device_view, uint64_t, uint64_t, uint64_t *, uint32_t *,
                          uint32_t *, const uint64_t *, JumpTables);

template <int KIND, bool SPLIT>
ReduceFn pick(int op)
{
    if (op == RNG_SUM_U32)
        return reduce_kernel<KIND, RNG_SUM_U32, SPLIT>;
    if (op == RNG_SUM_U24)
        return reduce_kernel<KIND, RNG_SUM_U24, SPLIT>;
    return reduce_kernel<KIND, RNG_DISC, SPLIT>;
}

template <bool SPLIT>
ReduceFn pick_kind(int kind, int op)
{
    switch (kind) {
    case RNG_MWC32: return pick<RNG_MWC32, SPLIT>(op);
    case RNG_XOR128: return pick<RNG_XOR128, SPLIT>(op);
    case RNG_KISS: return pick<RNG_KISS, SPLIT>(op);
    case RNG_MWC16X2: return pick<RNG_MWC16X2, SPLIT>(op);
    case RNG_XORSHIFT8: return pick<RNG_XORSHIFT8, SPLIT>(op);
    default: return pick<RNG_KISS_XOR, SPLIT>(op);
    }
}

}  // namespace
}  // namespace gbrng

using namespace gbrng;

extern "C" int rng_generate_reduce(rng_handle h, uint64_t n_per_stream, int op, void *out)
{
    Gen *g = reinterpret_cast<Gen *>(h);
    if (!g || !out || (uintptr_t)out % 8 != 0 ||
        (op != RNG_SUM_U32 && op != RNG_SUM_U24 && op != RNG_DISC))
        return set_error(RNG_ERR_ARG);
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != g->device && cudaSetDevice(g->device) != cudaSuccess)
        return set_error(RNG_ERR_CUDA);
    cudaStream_t st = g->stream;
    uint64_t *o = static_cast<uint64_t *>(out);
    rng_device_view v{g->kind, g->device, g->words, g->n, g->d_state, g->d_a};
    uint64_t rows = n_per_stream, segs = 1;
    // pairs never straddle segments: split rows are powers of two >= 2
    const bool split = g->d_split &&
                       split_plan(g->kind, g->n, n_per_stream, 1, g->jmul_segs,
                                  split_fill(true), &rows, &segs);
    if (!split) {
        rows = n_per_stream;
        segs = 1;
    }
    ReduceFn fn = split ? pick_kind<true>(g->kind, op) : pick_kind<false>(g->kind, op);
    JumpTables T{};
    const uint64_t *jmul = nullptr;
    int status = RNG_OK;
    if (split && needs_jump_tables(g->kind))
        status = jump_tables(&T);
    // no table build inside a CUDA graph capture (see gen_kernels.cuh)
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (!status && split)
        status = cuda_status(cudaStreamIsCapturing(st, &cap));
    if (!status && split && mont_table(g->kind) && cap == cudaStreamCaptureStatusNone)
        status = mwc_jump_table(g, rows, segs, st, &jmul);
    if (!status && split)
        status = cuda_status(cudaMemsetAsync(o, 0, g->n * 8, st));
    if (!status) {
        const dim3 grid((unsigned)((g->n + kThreads - 1) / kThreads), (unsigned)segs);
        fn<<<grid, kThreads, 0, st>>>(v, n_per_stream, rows, o, g->d_split, g->d_cnt, jmul, T);
        status = cuda_status(cudaGetLastError());
    }
    if (prev >= 0 && prev != g->device)
        cudaSetDevice(prev);
    return status;
}
