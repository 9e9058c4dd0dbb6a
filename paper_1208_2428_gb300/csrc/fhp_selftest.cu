// fhp_selftest.cu -- diagnostic: the bounded device-side waits give up.
//
// Every wait in the library's kernels (mbarrier phases of the shared-memory
// rings, completion counters of the multi-step kernels) is bounded: after
// kWaitLimitNs it returns false and the kernel records an error instead of
// spinning forever.  This kernel runs both wait helpers on conditions that
// never become true (a barrier nobody arrives on, a counter nobody bumps) and
// reports that each gave up, so that the timeout path itself is tested
// without faulting or hanging the GPU.
#include <cuda_runtime.h>

#include "../../include/fhp.h"
#include "fhp_debug.cuh"
#include "fhp_internal.h"
#include "fhp_quad.cuh"

namespace fhp {
namespace {

__global__ void wait_limits_kernel(const unsigned int* never_bumped, unsigned int* status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    unsigned int s = 0;
    if (!mbar_wait_bounded(&bar, 0u)) s |= 1u;                                // phase 0 never completes
    if (!wait_tiles(never_bumped, 0, 0, 0, false, 1u)) s |= 2u;               // counter stays 0
    *status = s;
}

// Debug builds: one index check that fails on purpose.  The check guards no
// access at all -- it only records its site in the error word -- so nothing
// outside any buffer is touched.
__global__ void debug_check_kernel(unsigned int* err) {
    if (threadIdx.x == 0 && blockIdx.x == 0) (void)dbg_ok(false, err, kSiteSelfTest);
}

}  // namespace
}  // namespace fhp

extern "C" int fhp_selftest_wait_limits(uint32_t* host_status) {
    if (!host_status) return FHP_EINVAL;
    unsigned int* d = nullptr;
    cudaError_t e = cudaMalloc((void**)&d, 2 * sizeof(unsigned int));
    if (e != cudaSuccess) return FHP_ENOMEM;
    e = cudaMemset(d, 0, 2 * sizeof(unsigned int));
    if (e == cudaSuccess) {
        fhp::wait_limits_kernel<<<1, 32>>>(d, d + 1);
        e = cudaGetLastError();
    }
    unsigned int s = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&s, d + 1, sizeof s, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return FHP_ECUDA;
    *host_status = s;
    return FHP_OK;
}

extern "C" int fhp_debug_selftest(uint32_t* host_word) {
    if (!host_word) return FHP_EINVAL;
    if (!fhp::kDebugBuild) return FHP_EINVAL;   // the release build has no index checks
    unsigned int* d = nullptr;
    cudaError_t e = cudaMalloc((void**)&d, sizeof(unsigned int));
    if (e != cudaSuccess) return FHP_ENOMEM;
    e = cudaMemset(d, 0, sizeof(unsigned int));
    if (e == cudaSuccess) {
        fhp::debug_check_kernel<<<1, 32>>>(d);
        e = cudaGetLastError();
    }
    unsigned int w = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&w, d, sizeof w, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return FHP_ECUDA;
    *host_word = w;
    return FHP_OK;
}
