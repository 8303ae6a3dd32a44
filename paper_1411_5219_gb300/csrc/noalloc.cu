// qcd_norm2_noalloc: the FP64 norm reduction with its scratch in a static
// device array, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a host framework that has reserved
// all device memory for its own caching allocator leaves nothing to
// allocate from, and on a latency-critical path cudaMalloc's implicit
// device-wide synchronisation is not acceptable.  This entry point takes
// the input and the output as device pointers and allocates nothing: the
// per-block partial sums and the ticket counter of its grid reduction live
// in g_norm2_scratch below, which every GPU that loads the library holds
// until the process exits.
#include <mutex>

#include "qcd_handles.h"

namespace qcd {
namespace {

constexpr int kNoallocThreads = 256;
constexpr int kNoallocPerThread = 8;
constexpr size_t kNoallocPerBlock = (size_t)kNoallocThreads * kNoallocPerThread;
// 8192 partial sums (64 KiB) and, after them, one 256-byte slot whose first
// word is the ticket counter.
constexpr int kNoallocMaxBlocks = 8192;
constexpr size_t kNoallocMaxElems = (size_t)kNoallocMaxBlocks * kNoallocPerBlock;  // 16,777,216 doubles

static __device__ __align__(256) double g_norm2_scratch[kNoallocMaxBlocks + 32];

// One partial per block (fixed tree inside the block); the last block to
// take a ticket adds the partials in block order, writes the result and
// resets the counter.
__global__ void __launch_bounds__(kNoallocThreads) norm2_noalloc_kernel(const double *x, size_t n, double *result,
                                                                        double *scratch)
{
    unsigned *counter = reinterpret_cast<unsigned *>(scratch + kNoallocMaxBlocks);
    const size_t base = (size_t)blockIdx.x * kNoallocPerBlock + threadIdx.x;
    double v[1] = {0.0};
#pragma unroll
    for (int k = 0; k < kNoallocPerThread; ++k) {
        const size_t i = base + (size_t)k * kNoallocThreads;
        if (i < n) {
            const double a = __ldg(x + i);
            v[0] = fma(a, a, v[0]);
        }
    }
    __shared__ double smem[32];
    __shared__ bool is_last;
    block_sum<1>(v, smem);
    if (threadIdx.x == 0) {
        scratch[blockIdx.x] = v[0];
        __threadfence();
        is_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double s[1] = {0.0};
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s[0] += __ldcg(scratch + b);
    block_sum<1>(s, smem);
    if (threadIdx.x == 0) {
        *result = s[0];
        *counter = 0u;
    }
}

// Device address of g_norm2_scratch, looked up once per device.
std::mutex g_setup_mu;
double *g_scratch_addr[64] = {};

qcd_status scratch_address(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return check_cuda(e, "norm2_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(QCD_ERR_INVALID_ARG, "norm2_noalloc: device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_norm2_scratch);
        if (e != cudaSuccess) return check_cuda(e, "norm2_noalloc: cudaGetSymbolAddress");
        g_scratch_addr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_addr[dev];
    return QCD_OK;
}

}  // namespace
}  // namespace qcd

using namespace qcd;

extern "C" qcd_status qcd_norm2_noalloc(const double *x_device, size_t n, double *result_device, void *stream)
{
    if (!result_device || (n > 0 && !x_device)) return fail(QCD_ERR_INVALID_ARG, "norm2_noalloc: NULL argument");
    if (n > kNoallocMaxElems)
        return fail(QCD_ERR_INVALID_ARG,
                    "norm2_noalloc: n = %zu exceeds the maximum of %zu doubles that its static scratch supports",
                    n, kNoallocMaxElems);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n == 0) return check_cuda(cudaMemsetAsync(result_device, 0, sizeof(double), s), "norm2_noalloc");
    double *scratch = nullptr;
    qcd_status st = scratch_address(&scratch);
    if (st != QCD_OK) return st;
    // the ticket counter must start at zero, whatever an earlier call left
    cudaError_t e = cudaMemsetAsync(scratch + kNoallocMaxBlocks, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return check_cuda(e, "norm2_noalloc: clear");
    const unsigned blocks = (unsigned)((n + kNoallocPerBlock - 1) / kNoallocPerBlock);
    norm2_noalloc_kernel<<<blocks, kNoallocThreads, 0, s>>>(x_device, n, result_device, scratch);
    note_launches();
    return check_cuda(cudaGetLastError(), "norm2_noalloc");
}
