// Self-test of the kernels' bounded mbarrier wait (the failure path of every table-copy and
// tensor-core GEMM wait): one CTA waits on a barrier that nothing completes until the bound
// runs out, records the failure bit and returns; the host reads the bit and the duration.
#include <cuda_runtime.h>

#include "apply_kernels.cuh"
#include "../../include/bras.h"

namespace bras {

__global__ void k_wait_selftest(int* status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);   // one arrival expected, none will come
        mbar_fence_init();
        mbar_wait_parity_bounded(&bar, 0u, status);
    }
    __syncthreads();
}

}  // namespace bras

extern "C" int bras_wait_selftest(int* bits, double* elapsed_ms) {
    using namespace bras;
    if (!bits || !elapsed_ms) return BRAS_ERR_INVALID;
    int* d = nullptr;
    if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return BRAS_ERR_OOM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = BRAS_OK;
    float ms = 0.f;
    if (cudaMemset(d, 0, sizeof(int)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        rc = BRAS_ERR_CUDA;
    } else {
        cudaEventRecord(e0, 0);
        k_wait_selftest<<<1, 32>>>(d);
        count_launch(1);
        cudaEventRecord(e1, 0);
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
            cudaMemcpy(bits, d, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = BRAS_ERR_CUDA;
    }
    *elapsed_ms = ms;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(d);
    return rc;
}
