// Matrix-free Schur complement of the mixed Poisson saddle point (Sec. 4, Sec. 5.1):
//   -S~ x = B M_bras^{-1} B^T x   (Eq. approx_positive_schur_general with C = 0)
// for the pairs RT_k / DG_{k-1} and BDM_k / DG_{k-1} (the pair of Sec. 5.1) on tetrahedra.  B's block of cell K is sign(det J_K) B^ with
// B^_ij = int_ref div phi_j chi_i (the contravariant Piola map makes div phi = div^ phi^ / det J),
// chi_i the mean-orthonormal polynomials of degree <= k - 1 on the reference tetrahedron.
//   1. copies w_(K,a) = s_(K,a) (B^T x_K)_a, written to their slots in dof-sorted order;
//   2. t_i = sum of the copies of dof i, in a fixed order (cell, then local index);
//   3. z = M_bras^{-1} t  (the BRAS apply);
//   4. y_K = B^ (s_K . z[l2g_K]).
// x and y hold n_q = k (k + 1) (k + 2) / 6 values per cell, cells in the caller's order.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace bras {
namespace {

// NLOC: local H(div) dofs (RT_k or BDM_k), NQ: local DG_{k-1} dofs
template <int NLOC, int NQ, typename T>
__global__ void __launch_bounds__(256) k_schur_bt(int64_t E, const T* __restrict__ Bd, const T* __restrict__ x,
                                                  const int8_t* __restrict__ sgn, const int32_t* __restrict__ pos,
                                                  T* __restrict__ wb) {
    __shared__ T Bs[NQ * NLOC];
    for (int i = threadIdx.x; i < NQ * NLOC; i += blockDim.x) Bs[i] = Bd[i];
    __syncthreads();
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < E; c += (int64_t)gridDim.x * blockDim.x) {
        T xq[NQ];
#pragma unroll
        for (int i = 0; i < NQ; ++i) xq[i] = x[c * NQ + i];
#pragma unroll
        for (int a = 0; a < NLOC; ++a) {
            T w = T(0);
#pragma unroll
            for (int i = 0; i < NQ; ++i) w = fma(Bs[i * NLOC + a], xq[i], w);
            const int64_t copy = c * NLOC + a;
            wb[pos[copy]] = sgn[copy] < 0 ? -w : w;
        }
    }
}

template <typename T>
__global__ void k_copy_sums(int64_t n, const int64_t* __restrict__ off, const T* __restrict__ wb, T* __restrict__ t) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T acc = T(0);
        for (int64_t s = off[i]; s < off[i + 1]; ++s) acc += wb[s];
        t[i] = acc;
    }
}

template <int NLOC, int NQ, typename T>
__global__ void __launch_bounds__(256) k_schur_b(int64_t E, const T* __restrict__ Bd, const T* __restrict__ z,
                                                 const int32_t* __restrict__ l2g, const int8_t* __restrict__ sgn,
                                                 T* __restrict__ y) {
    __shared__ T Bs[NQ * NLOC];
    for (int i = threadIdx.x; i < NQ * NLOC; i += blockDim.x) Bs[i] = Bd[i];
    __syncthreads();
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < E; c += (int64_t)gridDim.x * blockDim.x) {
        T acc[NQ];
#pragma unroll
        for (int i = 0; i < NQ; ++i) acc[i] = T(0);
#pragma unroll
        for (int a = 0; a < NLOC; ++a) {
            const int64_t copy = c * NLOC + a;
            const T v = z[l2g[copy]];
            const T sv = sgn[copy] < 0 ? -v : v;
#pragma unroll
            for (int i = 0; i < NQ; ++i) acc[i] = fma(Bs[i * NLOC + a], sv, acc[i]);
        }
#pragma unroll
        for (int i = 0; i < NQ; ++i) y[c * NQ + i] = acc[i];
    }
}

int grid_of(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 148 * 16)); }

template <int NLOC, int NQ, typename T>
int schur_typed(bras_ctx* c, int prec, const T* x, T* y, cudaStream_t st) {
    const size_t copies = (size_t)c->E * NLOC;
    const size_t need = 8 * (copies + 2 * (size_t)c->n);
    if (c->schur_ws_bytes < need) {
        if (c->schur_ws) dfree(c, c->schur_ws);
        c->schur_ws = dalloc_bytes(c, need);
        c->schur_ws_bytes = c->schur_ws ? need : 0;
        if (!c->schur_ws) return BRAS_ERR_OOM;
    }
    T* wb = static_cast<T*>(c->schur_ws);
    T* t = wb + copies;
    T* z = t + c->n;
    const T* Bd = sizeof(T) == 8 ? reinterpret_cast<const T*>(c->Bdiv64) : reinterpret_cast<const T*>(c->Bdiv32);
    k_schur_bt<NLOC, NQ, T><<<grid_of(c->E), 256, 0, st>>>(c->E, Bd, x, c->sgn_user, c->cpos, wb);
    k_copy_sums<T><<<grid_of(c->n), 256, 0, st>>>(c->n, c->coff, wb, t);
    count_launch(2);
    if (cudaGetLastError() != cudaSuccess) return BRAS_ERR_CUDA;
    int rc = run_op(c, prec, OP_BRAS, t, z, 1, st);
    if (rc != BRAS_OK) return rc;
    k_schur_b<NLOC, NQ, T><<<grid_of(c->E), 256, 0, st>>>(c->E, Bd, z, c->l2g_user, c->sgn_user, y);
    count_launch(1);
    return cudaGetLastError() == cudaSuccess ? BRAS_OK : BRAS_ERR_CUDA;
}

// n_loc names the family and order on tetrahedra: RT_k 4 / 15 / 36 / 70, BDM_k 12 / 30 / 60 / 105
template <typename T>
int schur_order(bras_ctx* c, int prec, const T* x, T* y, cudaStream_t st) {
    switch (c->nloc) {
        case 4: return schur_typed<4, 1, T>(c, prec, x, y, st);
        case 15: return schur_typed<15, 4, T>(c, prec, x, y, st);
        case 36: return schur_typed<36, 10, T>(c, prec, x, y, st);
        case 70: return schur_typed<70, 20, T>(c, prec, x, y, st);
        case 12: return schur_typed<12, 1, T>(c, prec, x, y, st);
        case 30: return schur_typed<30, 4, T>(c, prec, x, y, st);
        case 60: return schur_typed<60, 10, T>(c, prec, x, y, st);
        case 105: return schur_typed<105, 20, T>(c, prec, x, y, st);
        default: return BRAS_ERR_INVALID;
    }
}

}  // namespace

int schur_apply_impl(bras_ctx* c, int prec, const void* x, void* y, cudaStream_t st) {
    if (prec == BRAS_FP64) return schur_order<double>(c, prec, static_cast<const double*>(x), static_cast<double*>(y), st);
    return schur_order<float>(c, prec, static_cast<const float*>(x), static_cast<float*>(y), st);
}

}  // namespace bras
