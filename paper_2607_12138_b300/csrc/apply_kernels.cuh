// Block-fused element kernels: signed gather -> local dense multiply -> scatter.
//
// One CUDA thread block per cell block (up to 256 cells, one thread per cell):
//   1. stage the block's dofs in shared memory, x_s[u] = x[ids[u]] (times 1/d for BRAS:
//      the right factor D^{-1} of Eq. mhatinvbras_def);
//   2. each thread gathers its cell's local vector with the signs of P (the injection P_K of
//      Sec. 2.2) and multiplies by the local matrix in registers:
//        H1 (affine):   z_K = c_K * A_ref x_K, A_ref = M_ref (mass) or M_ref^{-1} (BRAS),
//                       c_K = rho_K |det J_K| or its reciprocal (Eq. piola_mass_pullbacks);
//        H(curl)/H(div): z_K = A_K x_K with A_K = M_K or M_K^{-1} streamed per cell as a
//                       packed symmetric matrix in a cell-interleaved layout (coalesced);
//   3. the signed local results go to shared memory, and every block-local dof sums its
//      copies in a fixed order (the P^T of Eq. M_PMbrP / mhatinvbras_def); dofs with all
//      copies in the block are final (times 1/d for BRAS, the left D^{-1}), the others
//      leave a partial sum that k_combine adds up in ascending block order.
// No floating-point atomics anywhere: results are bit-reproducible.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace bras {

void count_launch(int k);

enum { OP_MASS = 0, OP_BRAS = 1, OP_DIAG = 2 };
enum { KIND_H1 = 0, KIND_PACKED = 1 };

struct BlockArgs {
    const int32_t* blk_e0;
    const int32_t* blk_u0;
    const int32_t* blk_nint;
    const int32_t* blk_p0;
    const int32_t* ids;
    const uint16_t* incoff;
    const uint16_t* loc;
    const uint16_t* inc;
    const void* dinv;    // T[n]
    const void* refmat;  // T[nloc*nloc]   (H1)
    const void* scale;   // T[E]           (H1)
    const void* pk;      // S[npk][Epad]   (packed)
    int64_t Epad;
    int64_t npart;
    int max_u;
    int max_ne;
};

template <typename T> __device__ __forceinline__ T to_t(double v) { return (T)v; }
template <typename T> __device__ __forceinline__ T ld_mat(const double* p) { return (T)__ldg(p); }
template <typename T> __device__ __forceinline__ T ld_mat(const float* p) { return (T)__ldg(p); }
template <typename T> __device__ __forceinline__ T ld_mat(const __nv_bfloat16* p) {
    return (T)__bfloat162float(*p);
}

template <int NLOC, typename T, typename S, int KIND, int OP>
__global__ void __launch_bounds__(256, 1)
k_block(const BlockArgs A, const T* __restrict__ x, T* __restrict__ y, T* __restrict__ part, int nrhs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int b = blockIdx.x, r = blockIdx.y, tid = threadIdx.x;
    const int e0 = A.blk_e0[b], ne = A.blk_e0[b + 1] - e0;
    const int u0 = A.blk_u0[b], nu = A.blk_u0[b + 1] - u0;
    const int nint = A.blk_nint[b];
    T* xs = reinterpret_cast<T*>(smem_raw);
    T* zs = xs + ((A.max_u + 1) & ~1);
    T* Ms = zs + NLOC * A.max_ne;
    const T* __restrict__ dinv = static_cast<const T*>(A.dinv);

    if (KIND == KIND_H1) {
        const T* ref = static_cast<const T*>(A.refmat);
        for (int i = tid; i < NLOC * NLOC; i += blockDim.x) Ms[i] = ref[i];
    }
    if (OP != OP_DIAG) {
        for (int u = tid; u < nu; u += blockDim.x) {
            const int g = A.ids[u0 + u];
            T v = x[(size_t)g * nrhs + r];
            if (OP == OP_BRAS) v *= dinv[g];
            xs[u] = v;
        }
    }
    __syncthreads();

    const int e = tid;
    if (e < ne) {
        const uint16_t* __restrict__ L = A.loc + (size_t)e0 * NLOC + e;
        uint64_t neg = 0;
        T xl[NLOC];
#pragma unroll
        for (int a = 0; a < NLOC; ++a) {
            const uint16_t c = L[a * ne];
            const T v = (OP == OP_DIAG) ? T(0) : xs[c & 0x7fff];
            const bool s = (c & 0x8000) != 0;
            neg |= (uint64_t)s << a;
            xl[a] = s ? -v : v;
        }
        if (KIND == KIND_H1) {
            const T c = static_cast<const T*>(A.scale)[e0 + e];
#pragma unroll
            for (int a = 0; a < NLOC; ++a) {
                T acc = T(0);
                if (OP == OP_DIAG) {
                    acc = Ms[a * NLOC + a];
                } else {
#pragma unroll
                    for (int q = 0; q < NLOC; ++q) acc = fma(Ms[a * NLOC + q], xl[q], acc);
                }
                acc *= c;
                zs[a * ne + e] = ((neg >> a) & 1) && OP != OP_DIAG ? -acc : acc;
            }
        } else {
            const S* __restrict__ pk = static_cast<const S*>(A.pk) + e0 + e;
            T zl[NLOC];
#pragma unroll
            for (int a = 0; a < NLOC; ++a) zl[a] = T(0);
#pragma unroll
            for (int a = 0; a < NLOC; ++a) {
#pragma unroll
                for (int q = 0; q <= a; ++q) {
                    const int idx = a * (a + 1) / 2 + q;
                    if (OP == OP_DIAG) {
                        if (q == a) zl[a] = ld_mat<T>(pk + (size_t)idx * A.Epad);
                    } else {
                        const T m = ld_mat<T>(pk + (size_t)idx * A.Epad);
                        zl[a] = fma(m, xl[q], zl[a]);
                        if (q < a) zl[q] = fma(m, xl[a], zl[q]);
                    }
                }
            }
#pragma unroll
            for (int a = 0; a < NLOC; ++a)
                zs[a * ne + e] = ((neg >> a) & 1) && OP != OP_DIAG ? -zl[a] : zl[a];
        }
    }
    __syncthreads();

    const uint16_t* __restrict__ I = A.inc + (size_t)e0 * NLOC;
    const uint16_t* __restrict__ IO = A.incoff + u0 + b;
    for (int u = tid; u < nu; u += blockDim.x) {
        const int s0 = IO[u], s1 = IO[u + 1];
        T acc = T(0);
        for (int s = s0; s < s1; ++s) acc += zs[I[s]];
        if (u < nint) {
            const int g = A.ids[u0 + u];
            y[(size_t)g * nrhs + r] = (OP == OP_BRAS) ? acc * dinv[g] : acc;
        } else {
            part[(size_t)r * A.npart + A.blk_p0[b] + (u - nint)] = acc;
        }
    }
}

template <typename T, int OP>
__global__ void k_combine(int64_t nsh, const int32_t* __restrict__ sh_ids, const int32_t* __restrict__ sh_off,
                          const int32_t* __restrict__ sh_slots, const T* __restrict__ part, int64_t npart,
                          const T* __restrict__ dinv, T* __restrict__ y, int nrhs) {
    const int64_t total = nsh * nrhs;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = i / nrhs;
        const int r = (int)(i - j * nrhs);
        T acc = T(0);
        for (int s = sh_off[j]; s < sh_off[j + 1]; ++s) acc += part[(size_t)r * npart + sh_slots[s]];
        const int g = sh_ids[j];
        y[(size_t)g * nrhs + r] = (OP == OP_BRAS) ? acc * dinv[g] : acc;
    }
}

// Launch one block apply (block kernel + combine).  Returns a cudaError_t.
template <int NLOC, typename T, typename S, int KIND, int OP>
cudaError_t launch_block(const BlockArgs& A, int nblk, const T* x, T* y, T* part, int nrhs,
                         int64_t nsh, const int32_t* sh_ids, const int32_t* sh_off, const int32_t* sh_slots,
                         cudaStream_t st) {
    size_t smem = sizeof(T) * (((A.max_u + 1) & ~1) + (size_t)NLOC * A.max_ne + (KIND == KIND_H1 ? NLOC * NLOC : 0));
    auto kern = k_block<NLOC, T, S, KIND, OP>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    dim3 grid(nblk, nrhs);
    kern<<<grid, 256, smem, st>>>(A, x, y, part, nrhs);
    count_launch(1);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    if (nsh > 0) {
        int64_t total = nsh * nrhs;
        int nb = (int)std::min<int64_t>((total + 255) / 256, 148 * 16);
        k_combine<T, OP><<<nb, 256, 0, st>>>(nsh, sh_ids, sh_off, sh_slots, part, A.npart,
                                              static_cast<const T*>(A.dinv), y, nrhs);
        count_launch(1);
        err = cudaGetLastError();
    }
    return err;
}

}  // namespace bras
