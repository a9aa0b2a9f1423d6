// hs_selftest.cu -- exercises the bounded device waits without a GPU fault:
// one CTA waits on an mbarrier phase that no copy will ever complete, gives
// up after the given limit and reports HS_ERR_TIMEOUT through the caller's
// status word, exactly as the summing kernels do when a tile's copies do not
// arrive.  The context stays usable afterwards.
#include "hs_device.cuh"
#include "hs_internal.h"

namespace {

__global__ void wait_for_nothing(uint32_t *counters, unsigned long long limit_ns)
{
    __shared__ __align__(8) uint64_t bar_storage;
    const uint32_t bar = hs::smem_addr(&bar_storage);
    if (threadIdx.x == 0)
        hs::mbar_init(bar, 1); // one arrival expected; none will come
    __syncthreads();
    const bool ok = __syncthreads_or(!hs::mbar_wait_bounded(bar, 0, limit_ns)) == 0;
    if (!ok && threadIdx.x == 0)
        hs::set_status(counters, HS_ERR_TIMEOUT);
}

} // namespace

extern "C" hs_status hs_selftest_wait_timeout(uint32_t *counters, uint64_t limit_ns,
                                              hs_stream_t stream)
{
    if (!counters || limit_ns == 0 || limit_ns > 10000000000ull)
        return HS_ERR_INVALID;
    wait_for_nothing<<<1, 128, 0, reinterpret_cast<cudaStream_t>(stream)>>>(counters, limit_ns);
    return cudaGetLastError() == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}
