// Instantiation of the hopping kernel for f32 spinors and links.
#include "dslash_kernel.cuh"

namespace qcd {

cudaError_t launch_dslash_f32(int recon, const DslashLaunch &a, cudaStream_t s)
{
    if (recon == 18) return launch_dslash_fmt<SpF32, GF32<18>>(a, s);
    if (recon == 12) return launch_dslash_fmt<SpF32, GF32<12>>(a, s);
    if (recon == 8) return launch_dslash_fmt<SpF32, GF32<8>>(a, s);
    return cudaErrorInvalidValue;
}

}  // namespace qcd
