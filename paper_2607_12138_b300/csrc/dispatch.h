// Per-(space kind, precision) launchers of the block kernels, one translation unit each.
#pragma once
#include <cuda_runtime.h>

#include "apply_kernels.cuh"

namespace bras {

// Kernels launched by this library since load (host counter, for launch accounting).
void count_launch(int k);
int64_t launches_so_far();

struct LaunchCommon {
    BlockArgs A;
    const void* dinv;   // T[n] 1/d for the combine pass
    int nblk;
    int64_t nsh;
    const int32_t *sh_ids, *sh_off, *sh_slots;
};

cudaError_t launch_h1_f64(const LaunchCommon& L, int nloc, int op, const double* x, double* y, double* part, int nrhs, cudaStream_t st);
cudaError_t launch_h1_f32(const LaunchCommon& L, int nloc, int op, const float* x, float* y, float* part, int nrhs, cudaStream_t st);
cudaError_t launch_pk_f64(const LaunchCommon& L, int nloc, int op, const double* x, double* y, double* part, int nrhs, cudaStream_t st);
cudaError_t launch_pk_f32(const LaunchCommon& L, int nloc, int op, const float* x, float* y, float* part, int nrhs, cudaStream_t st);
cudaError_t launch_pk_bf16(const LaunchCommon& L, int nloc, int op, const float* x, float* y, float* part, int nrhs, cudaStream_t st);

}  // namespace bras
