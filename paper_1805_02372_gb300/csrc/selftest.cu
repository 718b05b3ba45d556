// Self-tests of the failure-detection path: each kernel waits on something that never
// happens, with the same bounded waits the hashing kernels use, and must return with
// PA_ERR_TIMEOUT in its status word (no trap, no fault; the context stays usable).
#include "common.cuh"

namespace pa {
namespace {

// A dependency counter that no item ever signals (the persistent kernel's wait).
__global__ void selftest_counter_wait(const uint32_t *counter, int *status) {
    __shared__ int flag;
    wait_count(counter, 1u, status, &flag);
}

// An mbarrier expecting bytes from a bulk copy that is never issued (the TMA wait).
__global__ void selftest_mbarrier_wait(int *status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_arrive_expect_tx(&bar, 16);
    mbar_wait_bounded(&bar, 0, status);
}

}  // namespace
}  // namespace pa

extern "C" int pa_selftest(int which, int *device_status) {
    using namespace pa;
    if (!device_status || (which != 1 && which != 2)) return PA_ERR_INVALID;
    int *mem = nullptr;
    PA_CUDA_TRY(cudaMalloc(&mem, 64));
    cudaError_t e = cudaMemset(mem, 0, 64);
    if (e == cudaSuccess) {
        if (which == 1)
            selftest_counter_wait<<<1, 32>>>(reinterpret_cast<const uint32_t *>(mem + 8), mem);
        else
            selftest_mbarrier_wait<<<1, 32>>>(mem);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int st = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&st, mem, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(mem);
    if (e != cudaSuccess) return cuda_fail(e);
    *device_status = st;
    return PA_OK;
}
