// Self-test of the bounded waits (failure detection without a fault): a kernel waits on
// a shared-memory mbarrier that nothing arrives on, through the same bounded wait the
// persistent work-queue kernels use, and must give up (about a second) and report
// CELESTE_ERR_TIMEOUT in a status word instead of hanging or trapping; the context stays
// usable afterwards.
#include "async_copy.cuh"
#include "internal.cuh"

namespace cel {

namespace {

__global__ void k_wait_nothing(int32_t* status) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_init_fence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // phase 0 never completes: no thread arrives and no copy is announced
        if (!mbar_wait_bounded(&bar, 0)) atomicExch(status, (int32_t)CELESTE_ERR_TIMEOUT);
    }
}

}  // namespace

}  // namespace cel

using namespace cel;

extern "C" celeste_status celeste_selftest_bounded_wait(void) {
    int32_t* d = nullptr;
    int32_t h = 0;
    cudaError_t e = cudaMalloc(&d, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(d, 0, sizeof(int32_t));
    if (e == cudaSuccess) {
        k_wait_nothing<<<1, 32>>>(d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (d) cudaFree(d);
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return CELESTE_ERR_CUDA;
    }
    if (h != 0) set_last_error("bounded wait gave up as expected");
    return h;
}
