// The generation kernels for the paper's own generators (the two-part
// base-2^16 MWC, the r = 8 XorShift of Eq. 5 and KISS in the xor form),
// compiled apart from the three target kinds so that neither translation
// unit carries the other's instantiations.
#include "gen_kernels.cuh"

namespace gbrng {

int launch_generate_paper(int kind, int fmt, const GenLaunch &p, cudaStream_t st)
{
    switch (kind) {
    case RNG_MWC16X2: return launch_kind<RNG_MWC16X2>(fmt, p, st);
    case RNG_XORSHIFT8: return launch_kind<RNG_XORSHIFT8>(fmt, p, st);
    case RNG_KISS_XOR: return launch_kind<RNG_KISS_XOR>(fmt, p, st);
    default: return set_error(RNG_ERR_ARG);
    }
}

}  // namespace gbrng
