// Instantiation of the hopping kernel for f16 spinors and links.
#include "dslash_kernel.cuh"

namespace qcd {

cudaError_t launch_dslash_f16(int recon, const DslashLaunch &a, cudaStream_t s)
{
    if (recon == 18) return launch_dslash_fmt<SpF16, G16<__half, 18>>(a, s);
    if (recon == 12) return launch_dslash_fmt<SpF16, G16<__half, 12>>(a, s);
    if (recon == 8) return launch_dslash_fmt<SpF16, G16<__half, 8>>(a, s);
    return cudaErrorInvalidValue;
}

}  // namespace qcd
