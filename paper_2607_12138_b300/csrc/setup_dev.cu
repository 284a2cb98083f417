// Device part of bras_setup: geometry, Piola metrics, per-cell element matrices and their
// FP64 Cholesky inverses (Sec. 2.2: every M_K is SPD, so M_br^{-1} = diag M_K^{-1} exists).
#include <cuda_bf16.h>

#include <algorithm>

#include "packet.h"
#include "setup_dev.h"
#include "dispatch.h"

namespace bras {

// J_K = [x_1 - x_0, .., x_d - x_0]; |det J_K|; Piola metric G_K of Eq. piola_mass_pullbacks:
//   H(curl): |det J| J^{-1} J^{-T},   H(div): J^T J / |det J|,  stored as (00,11,22,01,02,12).
// H1: mscale = rho |det J| (M_K = mscale M_ref), bscale = 1 / mscale.
__global__ void k_geometry(int dim, int space, int64_t E, const int32_t* __restrict__ perm,
                           const double* __restrict__ coords, const int32_t* __restrict__ cells,
                           const double* __restrict__ rho_user, double* __restrict__ absdet,
                           double* __restrict__ rho_int, double* __restrict__ metric,
                           double* __restrict__ ms64, double* __restrict__ bs64, float* __restrict__ ms32,
                           float* __restrict__ bs32, unsigned long long* __restrict__ bad) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t K = perm[e];
        double J[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
        const int32_t* cv = cells + K * (dim + 1);
        const double* x0 = coords + (int64_t)cv[0] * dim;
        for (int j = 0; j < dim; ++j) {
            const double* xj = coords + (int64_t)cv[j + 1] * dim;
            for (int c = 0; c < dim; ++c) J[c][j] = xj[c] - x0[c];
        }
        double det;
        if (dim == 2) det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        else det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                   J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        const double ad = fabs(det);
        if (!(ad > 0.0)) atomicMin(bad, (unsigned long long)K);
        const double rw = rho_user ? rho_user[K] : 1.0;
        if (!(rw > 0.0)) atomicMin(bad, (unsigned long long)K);
        absdet[e] = ad;
        rho_int[e] = rw;
        if (space == 0) {
            const double m = rw * ad;
            if (ms64) { ms64[e] = m; bs64[e] = 1.0 / m; }
            if (ms32) { ms32[e] = (float)m; bs32[e] = (float)(1.0 / m); }
        } else {
            double G[3][3];
            if (space == 1) {
                // J^{-1} = adj(J)/det; G = |det| J^{-1} J^{-T} = adj adj^T / |det|
                double A[3][3];
                A[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
                A[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
                A[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
                A[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
                A[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
                A[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
                A[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
                A[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
                A[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) {
                        double s = 0;
                        for (int k = 0; k < 3; ++k) s += A[i][k] * A[j][k];
                        G[i][j] = s / ad;
                    }
            } else {
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) {
                        double s = 0;
                        for (int k = 0; k < 3; ++k) s += J[k][i] * J[k][j];
                        G[i][j] = s / ad;
                    }
            }
            metric[0 * E + e] = G[0][0] * rw;
            metric[1 * E + e] = G[1][1] * rw;
            metric[2 * E + e] = G[2][2] * rw;
            metric[3 * E + e] = G[0][1] * rw;
            metric[4 * E + e] = G[0][2] * rw;
            metric[5 * E + e] = G[1][2] * rw;
        }
    }
}

// One warp per cell.  A = M_K = sum_ab G_ab R_ab; packed copy written; Cholesky A = L L^T in
// place (FP64, fails on a pivot <= 0); W = L^{-1}; M_K^{-1} = W^T W written packed (FP64,
// FP32, and a bf16 copy that is re-checked for positive definiteness and, if rounding broke
// it, shifted by a small multiple of its mean diagonal until its Cholesky succeeds).
__device__ bool warp_cholesky(double* A, int n, int lane) {
    for (int k = 0; k < n; ++k) {
        __syncwarp();
        const double piv = A[k * n + k];
        if (!(piv > 0.0)) return false;
        const double d = sqrt(piv);
        __syncwarp();
        for (int i = k + 1 + lane; i < n; i += 32) A[i * n + k] /= d;
        __syncwarp();
        if (lane == 0) A[k * n + k] = d;
        for (int i = k + 1 + lane; i < n; i += 32) {
            const double lik = A[i * n + k];
            for (int j = k + 1; j <= i; ++j) A[i * n + j] -= lik * A[j * n + k];
        }
    }
    __syncwarp();
    return true;
}

__global__ void k_element_inverse(int n, int64_t E, int64_t Epad, const double* __restrict__ Rref,
                                  const double* __restrict__ metric, double* __restrict__ Mpk64,
                                  float* __restrict__ Mpk32, double* __restrict__ Minv64,
                                  float* __restrict__ Minv32, __nv_bfloat16* __restrict__ Minvbf,
                                  unsigned long long* __restrict__ bad, int* __restrict__ nfixed,
                                  const int32_t* __restrict__ perm) {
    extern __shared__ double sm[];
    const int warps = blockDim.x / 32, w = threadIdx.x / 32, lane = threadIdx.x % 32;
    double* A = sm + (size_t)w * 2 * n * n;
    double* W = A + n * n;
    const int nn = n * n;
    for (int64_t e = blockIdx.x * (int64_t)warps + w; e < E; e += (int64_t)gridDim.x * warps) {
        double g[6];
        for (int c = 0; c < 6; ++c) g[c] = metric[c * E + e];
        // M_K = sum_ab G_ab R_ab (R_ab = R_ba^T; symmetric G)
        const int ab[9][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}, {1, 0}, {2, 0}, {2, 1}};
        const int gi[9] = {0, 1, 2, 3, 4, 5, 3, 4, 5};
        for (int t = lane; t < nn; t += 32) {
            double s = 0;
            for (int m = 0; m < 9; ++m) s += g[gi[m]] * Rref[(size_t)(ab[m][0] * 3 + ab[m][1]) * nn + t];
            A[t] = s;
        }
        __syncwarp();
        for (int t = lane; t < nn; t += 32) {          // symmetrise (rounding of the sum)
            const int i = t / n, j = t % n;
            if (j < i) { const double v = 0.5 * (A[i * n + j] + A[j * n + i]); A[i * n + j] = v; }
        }
        __syncwarp();
        for (int i = 0; i < n; ++i)
            for (int j = lane; j <= i; j += 32) {
                const int idx = i * (i + 1) / 2 + j;
                if (Mpk64) Mpk64[pk_index(idx, e, n * (n + 1) / 2, 2)] = A[i * n + j];
                if (Mpk32) Mpk32[pk_index(idx, e, n * (n + 1) / 2, 4)] = (float)A[i * n + j];
            }
        __syncwarp();
        if (!warp_cholesky(A, n, lane)) {
            if (lane == 0) atomicMin(bad, (unsigned long long)perm[e]);
            continue;
        }
        // W = L^{-1}, column c by lane
        for (int c = lane; c < n; c += 32) {
            for (int i = 0; i < c; ++i) W[i * n + c] = 0.0;
            W[c * n + c] = 1.0 / A[c * n + c];
            for (int i = c + 1; i < n; ++i) {
                double s = 0;
                for (int k = c; k < i; ++k) s += A[i * n + k] * W[k * n + c];
                W[i * n + c] = -s / A[i * n + i];
            }
        }
        __syncwarp();
        // M^{-1} = W^T W  (lower, packed); keep it in A for the bf16 check
        for (int t = lane; t < nn; t += 32) {
            const int i = t / n, j = t % n;
            if (j > i) continue;
            double s = 0;
            for (int k = i; k < n; ++k) s += W[k * n + i] * W[k * n + j];
            const int idx = i * (i + 1) / 2 + j;
            if (Minv64) Minv64[pk_index(idx, e, n * (n + 1) / 2, 2)] = s;
            if (Minv32) Minv32[pk_index(idx, e, n * (n + 1) / 2, 4)] = (float)s;
            A[i * n + j] = s;
            A[j * n + i] = s;
        }
        __syncwarp();
        if (Minvbf) {
            double mean = 0;
            for (int i = 0; i < n; ++i) mean += A[i * n + i];
            mean /= n;
            double shift = 0.0;
            int attempt = 0;
            for (; attempt < 12; ++attempt) {
                for (int t = lane; t < nn; t += 32) {
                    const int i = t / n, j = t % n;
                    const double v = A[(j <= i) ? (i * n + j) : (j * n + i)] + (i == j ? shift : 0.0);
                    W[t] = (double)__bfloat162float(__float2bfloat16_rn((float)v));
                }
                __syncwarp();
                if (warp_cholesky(W, n, lane)) break;
                shift = (shift == 0.0) ? 1e-3 * mean : shift * 4.0;
            }
            if (attempt > 0 && lane == 0) atomicAdd(nfixed, 1);
            for (int i = 0; i < n; ++i)
                for (int j = lane; j <= i; j += 32) {
                    const double v = A[i * n + j] + (i == j ? shift : 0.0);
                    Minvbf[pk_index(i * (i + 1) / 2 + j, e, n * (n + 1) / 2, 8)] = __float2bfloat16_rn((float)v);
                }
        }
        __syncwarp();
    }
}

cudaError_t run_geometry(int dim, int space, int64_t E, const int32_t* perm, const double* coords,
                         const int32_t* cells, const double* rho_user, double* absdet, double* rho_int,
                         double* metric, double* ms64, double* bs64, float* ms32, float* bs32,
                         unsigned long long* bad, cudaStream_t st) {
    int nb = (int)std::min<int64_t>((E + 255) / 256, 148 * 32);
    k_geometry<<<nb, 256, 0, st>>>(dim, space, E, perm, coords, cells, rho_user, absdet, rho_int, metric,
                                   ms64, bs64, ms32, bs32, bad);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t run_element_inverse(int n, int64_t E, int64_t Epad, const double* Rref, const double* metric,
                                double* Mpk64, float* Mpk32, double* Minv64, float* Minv32,
                                __nv_bfloat16* Minvbf, unsigned long long* bad, int* nfixed,
                                const int32_t* perm, cudaStream_t st) {
    // one warp per cell, two n x n FP64 work arrays each: four warps a CTA while they fit the
    // opt-in shared memory (n_loc = 84 takes 113 KB a warp)
    int optin = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t per_warp = (size_t)2 * n * n * sizeof(double);
    const int warps = (int)std::max<size_t>(1, std::min<size_t>(4, (size_t)optin / per_warp));
    size_t smem = (size_t)warps * per_warp;
    if (smem > (size_t)optin) return cudaErrorInvalidValue;
    cudaError_t err = cudaFuncSetAttribute(k_element_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int nb = (int)std::min<int64_t>((E + warps - 1) / warps, 148 * 16);
    k_element_inverse<<<nb, warps * 32, smem, st>>>(n, E, Epad, Rref, metric, Mpk64, Mpk32, Minv64, Minv32, Minvbf,
                                                     bad, nfixed, perm);
    count_launch(1);
    return cudaGetLastError();
}

// Exponent bound of the largest row abs-sum of every packed symmetric cell matrix: one thread
// per cell; *out = max over cells of E with sum_q |A_aq| < 2^E (atomicMax, *out preset).
__device__ __forceinline__ double pk_abs(const double* pk, size_t i) { return fabs(pk[i]); }
__device__ __forceinline__ double pk_abs(const float* pk, size_t i) { return fabs((double)pk[i]); }
__device__ __forceinline__ double pk_abs(const __nv_bfloat16* pk, size_t i) { return fabs((double)__bfloat162float(pk[i])); }

template <typename S>
__global__ void k_row_bound(int n, int64_t E, int64_t Epad, const S* __restrict__ pk, int* out) {
    constexpr int G = 16 / (int)sizeof(S);
    int emax = -100000;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        double best = 0.0;
        for (int a = 0; a < n; ++a) {
            double sum = 0.0;
            for (int q = 0; q < n; ++q) {
                const int i = a >= q ? a * (a + 1) / 2 + q : q * (q + 1) / 2 + a;
                sum += pk_abs(pk, pk_index(i, e, n * (n + 1) / 2, G));
            }
            best = fmax(best, sum);
        }
        if (best > 0.0) {
            int ex;
            frexp(best, &ex);   // best < 2^ex
            emax = max(emax, ex);
        }
    }
    atomicMax(out, emax);
}

template <typename S>
cudaError_t run_row_bound(int n, int64_t E, int64_t Epad, const S* pk, int* out, cudaStream_t st) {
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((E + 255) / 256, 148 * 8));
    k_row_bound<S><<<nb, 256, 0, st>>>(n, E, Epad, pk, out);
    count_launch(1);
    return cudaGetLastError();
}
template cudaError_t run_row_bound<double>(int, int64_t, int64_t, const double*, int*, cudaStream_t);
template cudaError_t run_row_bound<float>(int, int64_t, int64_t, const float*, int*, cudaStream_t);
template cudaError_t run_row_bound<__nv_bfloat16>(int, int64_t, int64_t, const __nv_bfloat16*, int*, cudaStream_t);

// v -> (hi, lo) = ((float)v, (float)(v - hi)): a float pair within ~2^-48 of v
__global__ void k_split_pairs(const double* __restrict__ a, float2* __restrict__ b, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double v = a[i];
        const float h = (float)v;
        b[i] = make_float2(h, (float)(v - (double)h));
    }
}

cudaError_t run_split_pairs(const double* a, float2* b, size_t n, cudaStream_t st) {
    const int nb = (int)std::min<size_t>((n + 255) / 256, 148 * 8);
    k_split_pairs<<<nb, 256, 0, st>>>(a, b, n);
    count_launch(1);
    return cudaGetLastError();
}

}  // namespace bras
