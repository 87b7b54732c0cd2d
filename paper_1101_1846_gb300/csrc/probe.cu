// Measurement kernels for the roofline denominators: a write-only bandwidth
// probe (the paper found its writes-only kernels capped well below the
// card's read+write bandwidth and measured a writes-only benchmark to
// confirm it; Sec. "Discussion") and integer-pipe throughput probes for the
// operations the generators are made of (the paper's usable operations per
// second, Eq. 9).
#include "gbrng.cuh"
#include "rng_tune.h"

namespace gbrng {
namespace {

template <int HINT>
__global__ void probe_write(uint4 *dst, uint64_t n16, int reps)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; ++r) {
        uint4 v = make_uint4(r, r + 1, r + 2, r + 3);
        for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) {
            if constexpr (HINT)
                __stcs(dst + i, v);
            else
                dst[i] = v;
        }
    }
}

// Integer-pipe probes: every thread runs 8 independent chains (latency
// hidden by ILP) of one operation.  Each operation is inline PTX marked
// volatile, so the compiler neither folds repeated applications (affine and
// GF(2) maps compose into one) nor drops them; the chains feed one word per
// thread written to `sink` so that nothing is dead.
//   op 0  32 x 32 + 32 -> 64 multiply-add as in an MWC step (mad.lo.cc +
//         madc.hi: 2 instructions)
//   op 1  32-bit multiply-add as in the LCG (mad.lo: 1 instruction)
//   op 2  shift and xor as in a xorshift step (shl + xor: 2 instructions)
//   op 3  32-bit add (1 instruction)
template <int OP>
__global__ void probe_int(uint32_t *sink, uint64_t iters)
{
    uint32_t x[8], c[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        x[k] = threadIdx.x * 2654435761u + k;
        c[k] = blockIdx.x + k;
    }
    const uint32_t a = 4294967118u;
    for (uint64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if constexpr (OP == 0) {
                uint32_t lo, hi;
                asm volatile("mad.lo.cc.u32 %0, %2, %3, %4;\n\t"
                             "madc.hi.u32 %1, %2, %3, 0;"
                             : "=&r"(lo), "=r"(hi)
                             : "r"(a), "r"(x[k]), "r"(c[k]));
                x[k] = lo;
                c[k] = hi;
            } else if constexpr (OP == 1) {
                asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x[k]) : "r"(69069u), "r"(c[k]));
            } else if constexpr (OP == 2) {
                asm volatile("{\n\t.reg .b32 t;\n\tshl.b32 t, %0, 13;\n\txor.b32 %0, %0, t;\n\t}"
                             : "+r"(x[k]));
            } else {
                asm volatile("add.u32 %0, %0, %1;" : "+r"(x[k]) : "r"(c[k]));
            }
        }
    }
    uint32_t r = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k)
        r ^= x[k] ^ c[k];
    sink[(uint64_t)blockIdx.x * blockDim.x + threadIdx.x] = r;
}

}  // namespace
}  // namespace gbrng

using namespace gbrng;

extern "C" int gbrng_probe_write(void *dst, uint64_t bytes, int blocks, int threads, int hint,
                                 int reps, void *cuda_stream)
{
    if (!dst || bytes % 16 || (uintptr_t)dst % 16 || blocks <= 0 || threads <= 0 ||
        threads > 1024 || reps <= 0)
        return set_error(RNG_ERR_ARG);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (hint)
        probe_write<1><<<blocks, threads, 0, st>>>(static_cast<uint4 *>(dst), bytes / 16, reps);
    else
        probe_write<0><<<blocks, threads, 0, st>>>(static_cast<uint4 *>(dst), bytes / 16, reps);
    return cuda_status(cudaGetLastError());
}

extern "C" int gbrng_probe_int(int op, uint32_t *sink, int blocks, int threads, uint64_t iters,
                               void *cuda_stream)
{
    if (!sink || blocks <= 0 || threads <= 0 || threads > 1024 || op < 0 || op > 3)
        return set_error(RNG_ERR_ARG);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    switch (op) {
    case 0: probe_int<0><<<blocks, threads, 0, st>>>(sink, iters); break;
    case 1: probe_int<1><<<blocks, threads, 0, st>>>(sink, iters); break;
    case 2: probe_int<2><<<blocks, threads, 0, st>>>(sink, iters); break;
    default: probe_int<3><<<blocks, threads, 0, st>>>(sink, iters); break;
    }
    return cuda_status(cudaGetLastError());
}
