// Test hook for the bounded waits of the tensor-core kernels: the tcgen05 MMAs signal their
// completion on an mbarrier that every thread polls a bounded number of times (tc.cuh,
// mbar_wait_bounded); a wait that runs out raises a device flag and lets the kernel finish
// instead of hanging.  This entry point runs that same wait on a barrier that completes (one
// arrival) or that nothing completes, so a test can check both outcomes and that the device
// stays usable after a wait ran out.
#include <cuda_runtime.h>

#include "jetsci_internal.h"
#include "tc.cuh"

namespace jetsci {
namespace {

__global__ void __launch_bounds__(32) k_selftest_bounded_wait(uint32_t max_iter, int arrive, uint32_t *out) {
    __shared__ __align__(8) uint64_t mbar;
    if (threadIdx.x == 0) {
        tc::mbar_init(&mbar, 1);
        tc::fence_mbar_init();
    }
    __syncthreads();
    if (arrive && threadIdx.x == 0) tc::mbar_arrive(&mbar);
    __syncthreads();
    const bool ok = tc::mbar_wait_bounded(&mbar, 0, max_iter);
    if (threadIdx.x == 0) out[0] = ok ? 0u : 1u;
}

}  // namespace
}  // namespace jetsci

extern "C" jetsci_status jetsci_selftest_bounded_wait(uint32_t max_iter, int arrive, uint32_t *timed_out_host) {
    using namespace jetsci;
    if (!timed_out_host) return fail(JETSCI_ERR_ARG, "timed_out_host is NULL");
    if (max_iter < 1 || max_iter > (1u << 20)) return fail(JETSCI_ERR_ARG, "max_iter must be in 1 .. 2^20");
    uint32_t *d = nullptr;
    JETSCI_CUDA_TRY(cudaMalloc(&d, sizeof(uint32_t)));
    k_selftest_bounded_wait<<<1, 32>>>(max_iter, arrive, d);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(timed_out_host, d, sizeof(uint32_t), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "bounded-wait self-test");
    return JETSCI_OK;
}
