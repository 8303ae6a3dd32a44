// Instantiation of the hopping kernel for double-float (df64) spinors and
// links (reconstruct-18 only), dagger = 0.  The two dagger values live in
// separate translation units so that they compile in parallel.
#include "dslash_kernel.cuh"

namespace qcd {

cudaError_t launch_dslash_df64_d0(int recon, const DslashLaunch &a, cudaStream_t s)
{
    if (recon == 18) return launch_dslash_dag<SpDF64, GDF64<18>, 0>(a, s);
    return cudaErrorInvalidValue;
}

}  // namespace qcd
