// Device setup kernels (geometry, element matrices, local inverses).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace bras {

cudaError_t run_geometry(int dim, int space, int64_t E, const int32_t* perm, const double* coords,
                         const int32_t* cells, const double* rho_user, double* absdet, double* rho_int,
                         double* metric, double* ms64, double* bs64, float* ms32, float* bs32,
                         unsigned long long* bad, cudaStream_t st);

cudaError_t run_element_inverse(int n, int64_t E, int64_t Epad, const double* Rref, const double* metric,
                                double* Mpk64, float* Mpk32, double* Minv64, float* Minv32,
                                __nv_bfloat16* Minvbf, unsigned long long* bad, int* nfixed,
                                const int32_t* perm, cudaStream_t st);

// b[i] = (hi, lo) float pair of a[i] (hi = a rounded to FP32, lo = the rest rounded)
cudaError_t run_split_pairs(const double* a, float2* b, size_t n, cudaStream_t st);

// *out = max(*out, exponent bound of the largest row abs-sum of the packed cell matrices)
template <typename S>
cudaError_t run_row_bound(int n, int64_t E, int64_t Epad, const S* pk, int* out, cudaStream_t st);

}  // namespace bras
