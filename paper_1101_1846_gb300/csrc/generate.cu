// The generation kernels: every thread keeps the state of its streams in
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
// Vector kernel (n % 4 == 0, out 16-byte aligned): a CTA of B threads covers
// 4*V*B consecutive streams; thread t owns the groups of four starting at
// base + 4t + 4Bv, v < V, so each of its V stores per step is coalesced
// across the warp.  Scalar kernel (any n, any 4-byte aligned out): one
// stream per thread, 4-byte stores.
#include "gen_body.cuh"
#include "rng_tune.h"

namespace gbrng {
namespace {

template <int KIND, int FMT, int V, int HINT>
__global__ void __launch_bounds__(512)
gen_vec(uint32_t *__restrict__ state, const uint32_t *__restrict__ mult, uint64_t n,
        uint64_t steps, uint32_t *__restrict__ out, uint64_t ld)
{
    const uint64_t B = blockDim.x;
    const uint64_t s_first = (uint64_t)blockIdx.x * (4 * V) * B + 4 * (uint64_t)threadIdx.x;
    body_vec<KIND, FMT, V, HINT>(state, mult, n, steps, out, ld, s_first, 4 * B, n);
}

template <int KIND, int FMT, int HINT>
__global__ void __launch_bounds__(512)
gen_scalar(uint32_t *__restrict__ state, const uint32_t *__restrict__ mult, uint64_t n,
           uint64_t steps, uint32_t *__restrict__ out, uint64_t ld)
{
    uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n)
        body_scalar<KIND, FMT, HINT>(state, mult, n, steps, out, ld, s);
}

using KernelFn = void (*)(uint32_t *, const uint32_t *, uint64_t, uint64_t, uint32_t *,
                          uint64_t);

template <int KIND, int FMT>
KernelFn pick_vec(int v, int hint)
{
    if (v == 2)
        return hint ? gen_vec<KIND, FMT, 2, 1> : gen_vec<KIND, FMT, 2, 0>;
    return hint ? gen_vec<KIND, FMT, 1, 1> : gen_vec<KIND, FMT, 1, 0>;
}

template <int KIND>
KernelFn pick_vec_kind(int fmt, int v, int hint)
{
    return fmt == RNG_F32 ? pick_vec<KIND, RNG_F32>(v, hint) : pick_vec<KIND, RNG_U32>(v, hint);
}

template <int KIND>
KernelFn pick_scalar_kind(int fmt, int hint)
{
    if (fmt == RNG_F32)
        return hint ? gen_scalar<KIND, RNG_F32, 1> : gen_scalar<KIND, RNG_F32, 0>;
    return hint ? gen_scalar<KIND, RNG_U32, 1> : gen_scalar<KIND, RNG_U32, 0>;
}

// Launch shape per (kind, fmt): streams-per-thread groups V, CTA size, store
// hint.  Defaults are the measured best on GB300; gbrng_set_launch changes
// them (the autotuner does).
struct Shape {
    int v = 1;
    int block = 256;
    int hint = 0;
};
Shape g_shape[3][2];

}  // namespace

int launch_generate(int kind, int fmt, const GenLaunch &p, cudaStream_t st)
{
    if (p.steps == 0 || p.n == 0)
        return RNG_OK;
    const Shape sh = g_shape[kind][fmt];
    bool vec = (p.n % 4 == 0) && (p.ld % 4 == 0) &&
               ((uintptr_t)p.out % 16 == 0) && ((uintptr_t)p.state % 16 == 0) &&
               (p.a == nullptr || (uintptr_t)p.a % 16 == 0);
    KernelFn fn;
    uint64_t blocks;
    int threads = sh.block;
    if (vec) {
        fn = kind == RNG_MWC32    ? pick_vec_kind<RNG_MWC32>(fmt, sh.v, sh.hint)
             : kind == RNG_XOR128 ? pick_vec_kind<RNG_XOR128>(fmt, sh.v, sh.hint)
                                  : pick_vec_kind<RNG_KISS>(fmt, sh.v, sh.hint);
        uint64_t groups = p.n / 4;
        // small problems: shrink the CTA so that more SMs take part
        while (threads > 32 && (groups + threads * sh.v - 1) / (threads * sh.v) < 152)
            threads /= 2;
        uint64_t per_block = (uint64_t)threads * sh.v;
        blocks = (groups + per_block - 1) / per_block;
    } else {
        fn = kind == RNG_MWC32    ? pick_scalar_kind<RNG_MWC32>(fmt, sh.hint)
             : kind == RNG_XOR128 ? pick_scalar_kind<RNG_XOR128>(fmt, sh.hint)
                                  : pick_scalar_kind<RNG_KISS>(fmt, sh.hint);
        while (threads > 32 && (p.n + threads - 1) / threads < 152)
            threads /= 2;
        blocks = (p.n + threads - 1) / threads;
    }
    if (blocks > 0x7FFFFFFFull)
        return set_error(RNG_ERR_ARG);
    fn<<<(unsigned)blocks, threads, 0, st>>>(p.state, p.a, p.n, p.steps,
                                             static_cast<uint32_t *>(p.out), p.ld);
    return cuda_status(cudaGetLastError());
}

}  // namespace gbrng

extern "C" int gbrng_set_launch(int kind, int fmt, int v, int block, int hint)
{
    using namespace gbrng;
    if (kind < 0 || kind > 2 || fmt < 0 || fmt > 1 || (v != 1 && v != 2) || block < 32 ||
        block > 512 || (block & (block - 1)) || hint < 0 || hint > 1)
        return set_error(RNG_ERR_ARG);
    g_shape[kind][fmt] = Shape{v, block, hint};
    return RNG_OK;
}

extern "C" int gbrng_get_launch(int kind, int fmt, int *v, int *block, int *hint)
{
    using namespace gbrng;
    if (kind < 0 || kind > 2 || fmt < 0 || fmt > 1 || !v || !block || !hint)
        return set_error(RNG_ERR_ARG);
    *v = g_shape[kind][fmt].v;
    *block = g_shape[kind][fmt].block;
    *hint = g_shape[kind][fmt].hint;
    return RNG_OK;
}
