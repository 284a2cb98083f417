// Per-(space kind, precision) launchers of the block kernels, one translation unit each.
#pragma once
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "apply_kernels.cuh"

namespace bras {

// Kernels launched by this library since load (host counter, for launch accounting).
void count_launch(int k);
int64_t launches_so_far();
void count_graph_launch();

struct LaunchCommon {
    BlockArgs A;
    CombineArgs G;
    int nblk;
};

cudaError_t launch_h1_f64(const LaunchCommon& L, int nloc, int op, const double* x, double* y, double* part, int nrhs, cudaStream_t st);
cudaError_t launch_h1_f32(const LaunchCommon& L, int nloc, int op, const float* x, float* y, float* part, int nrhs, cudaStream_t st);
cudaError_t launch_pk_f64(const LaunchCommon& L, int nloc, int op, const double* x, double* y, double* part, int nrhs, cudaStream_t st);
cudaError_t launch_pk_f32(const LaunchCommon& L, int nloc, int op, const float* x, float* y, float* part, int nrhs, cudaStream_t st);
bool h1_tc_supported(int nloc);
uint32_t h1_tc_btile_bytes(int nloc);
size_t h1_tc_smem_bytes(int nloc, const BlockArgs& A, bool mr = false);
cudaError_t launch_h1_tc(const LaunchCommon& L, const unsigned char* btile, int nloc, int op, const float* x,
                         float* y, float* part, int nrhs, cudaStream_t st);
void h1_tc_build_btile(const double* ref, int nloc, std::vector<unsigned char>& out);
cudaError_t launch_h1_df(const LaunchCommon& L, int nloc, const double* x, double* y, double* part, int nrhs, cudaStream_t st);
cudaError_t launch_pk_bf16(const LaunchCommon& L, int nloc, int op, const float* x, float* y, float* part, int nrhs, cudaStream_t st);

}  // namespace bras
