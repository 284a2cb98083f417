// H1 mass apply with float-float local products (FP64 vectors, FP64 results): the residual
// b - M x of the FP64 refinement loop around the FP32 inner solve.
//
// Same block structure as k_block (apply_kernels.cuh): table packet staged by bulk async copies,
// x staged in shared memory, exact fixed-point in-block dof sums, partials of boundary dofs
// added up by the combine pass.
// All arithmetic runs on the FP32 units as float-float pairs (about 2^-48 relative, the
// accuracy of FP64 sums) -- B300 issues FP64, and conversions to and from it, at 1/64 of the
// FP32 rate:
//   * x is split once per block-local dof into (vh, vl) with vh + vl = x to 2^-48;
//   * each cell is split over TPC = ceil(n_loc / 8) threads, thread g owning the output rows
//     [g R, g R + R) of z_K = c_K M_ref x_K, R = ceil(n_loc / TPC) (35 = 5 x 7, 20 = 3 x 7;
//     Eq. piola_mass_pullbacks); each row is one
//     compensated chain (leading product exact by an FMA, cross terms into the low part,
//     running sum by a two-sum), and c_K multiplies it as a float pair;
//   * both halves of each product pair go into the dof's exact 64-bit fixed-point accumulator
//     (apply_kernels.cuh), converted to FP64 once per dof.
// Seven or eight independent rows per thread at 48 registers (two CTAs of up to 640 threads
// per SM) keep many warps in flight; lanes of a warp hold different cells of the same row
// group, so the rows of M_ref are broadcast reads.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "apply_kernels.cuh"

namespace bras {

constexpr int kDfRows = 8;   // at most this many output rows per thread

template <int NLOC> struct DfShape {
    static constexpr int TPC = (NLOC + kDfRows - 1) / kDfRows;   // threads per cell
    static constexpr int ROWS = (NLOC + TPC - 1) / TPC;          // rows per thread (35: 5 x 7)
};

template <int NLOC>
__global__ void __launch_bounds__(640, 2)
k_block_df(const BlockArgs A, const double* __restrict__ x, double* __restrict__ y, double* __restrict__ part,
           int nrhs) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
    unsigned char* tab = smem_raw + 128;
    int* fx = reinterpret_cast<int*>(smem_raw + 64);                                 // [0] ex, [1] ec
    float2* xs = reinterpret_cast<float2*>(tab + ((A.max_pkt + 127u) & ~127u));   // [u] (hi, lo)
    long long* ys = reinterpret_cast<long long*>(xs + ((A.max_u + 1) & ~1));       // [u] accumulators
    float2* Ms = reinterpret_cast<float2*>(ys + ((A.max_u + 1) & ~1));              // [NLOC][NLOC] (hi, lo)

    const int b = blockIdx.x / nrhs, r = blockIdx.x % nrhs, tid = threadIdx.x;
    const int cw = blockDim.x / DfShape<NLOC>::TPC;   // cells per row group
    const int g = tid / cw;                           // this thread: rows [8g, 8g + 8) of cells tid % cw + k cw
    const int e0 = A.blk_e0[b], ne = A.blk_e0[b + 1] - e0;
    const int u0 = A.blk_u0[b], nu = A.blk_u0[b + 1] - u0;
    const int nint = A.blk_nint[b];
    const int64_t p0 = (int64_t)r * A.npart + A.blk_p0[b];
    const uint32_t sa = pkt_size_a(nu, false), sb = pkt_size_b((uint32_t)(ne * NLOC), false);
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_fence_init();
        const unsigned char* src = A.pkt + A.blk_pkt[b];
        mbar_expect_tx(&bars[0], sa);
        bulk_copy_g2s(tab, src, sa, &bars[0]);
        mbar_expect_tx(&bars[1], sb);
        bulk_copy_g2s(tab + sa, src + sa, sb, &bars[1]);
        fx[0] = fx[1] = kExpZero;
    }
    const FxAcc acc{ys, (nu + 1) & ~1, A.fx_lo};
    acc.clear(acc.count);
    const double* ref = static_cast<const double*>(A.refmat);
    for (int i = tid; i < NLOC * NLOC; i += blockDim.x) {
        const double v = ref[i];
        const float hi = (float)v;
        Ms[i] = make_float2(hi, (float)(v - (double)hi));
    }
    __syncthreads();   // barriers and bounds initialised before anyone uses them
    for (int e = tid; e < ne; e += blockDim.x)
        atomicMax(&fx[1], exp_bound(static_cast<const double*>(A.scale)[e0 + e]));
    const int32_t* ids = reinterpret_cast<const int32_t*>(tab);
    const uint16_t* loc = reinterpret_cast<const uint16_t*>(tab + sa);

    const bool okA = cta_wait(&bars[0], 0, A.status, true);
    uint64_t amax = 0;   // largest |staged value| bits
    if (okA) {
        for (int u = tid; u < nu; u += 8 * blockDim.x) {
            double v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int uu = u + k * blockDim.x;
                v[k] = uu < nu ? x[(size_t)ids[uu] * nrhs + r] : 0.0;
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int uu = u + k * blockDim.x;
                if (uu < nu) {
                    const float hi = (float)v[k];
                    xs[uu] = make_float2(hi, (float)(v[k] - (double)hi));
                    amax = max(amax, abs_bits(v[k]));
                }
            }
        }
    }
    const int emax = exp_bound_bits(amax);
    if (emax > kExpZero) atomicMax(&fx[0], emax);
    if (!cta_wait(&bars[1], 0, A.status, okA)) {
        if (tid == 0) {
            mbar_wait_bounded(&bars[0], A.status);
            mbar_wait_bounded(&bars[1], A.status);
        }
        return;
    }

    // the block's fixed-point scale (2^k as a float: the products arrive as float pairs)
    bool bad;
    const int kx = fx_scale<float>(fx[0], fx[1], A.fx_er, A.fx_top, bad);
    const float sc = pow2<float>(kx);
    for (int e = tid % cw; e < ne; e += cw) {
        const double c = static_cast<const double*>(A.scale)[e0 + e];
        const float ch = (float)c, cl = (float)(c - (double)ch);
        constexpr int RW = DfShape<NLOC>::ROWS;
        const int a0 = g * RW;
        float sh[RW], sl[RW];
#pragma unroll
        for (int j = 0; j < RW; ++j) sh[j] = sl[j] = 0.f;
#pragma unroll 4
        for (int q = 0; q < NLOC; ++q) {
            const float2 v = xs[loc[q * ne + e]];
#pragma unroll
            for (int j = 0; j < RW; ++j) {
                const int a = a0 + j;
                if (a < NLOC) {
                    const float2 m = Ms[a * NLOC + q];
                    df_term(m.x, m.y, v.x, v.y, sh[j], sl[j]);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < RW; ++j) {
            const int a = a0 + j;
            if (a < NLOC) {
                float zh = 0.f, zl = 0.f;   // (sh + sl) (ch + cl)
                df_term(ch, cl, sh[j], sl[j], zh, zl);
                // both halves of the pair into the dof's fixed-point accumulator
                acc.add(loc[a * ne + e], fx_round(zh * sc) + fx_round(zl * sc));
            }
        }
    }
    __syncthreads();

    // totals in FP64: interior dofs to y, shared ones to their partial slots
    for (int u = tid; u < nu; u += blockDim.x) {
        const double v = bad ? __longlong_as_double(0x7ff8000000000000ll) : fx_value(acc.total(u), kx, 0.0);
        if (u < nint) y[(size_t)ids[u] * nrhs + r] = v;
        else part[p0 + (u - nint)] = v;
    }
}

template <int NLOC>
size_t df_smem_bytes(const BlockArgs& A, int threads) {
    return 128 + ((A.max_pkt + 127u) & ~127u) + 2 * 8 * (((size_t)A.max_u + 1) & ~(size_t)1) +
           sizeof(float2) * (size_t)NLOC * NLOC;
}

template <int NLOC>
cudaError_t launch_block_df(const BlockArgs& A, const CombineArgs& G, int nblk, const double* x, double* y,
                            double* part, int nrhs, cudaStream_t st) {
    // cells per row group: whole warps, at most 128 (640 threads at n_loc = 35, two CTAs per
    // SM at 48 registers; larger blocks loop over their cells)
    const int cw = std::min((A.max_ne + 31) / 32 * 32, 128);
    const int threads = cw * DfShape<NLOC>::TPC;
    const size_t smem = df_smem_bytes<NLOC>(A, threads);
    auto kern = k_block_df<NLOC>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (err != cudaSuccess) return err;
    kern<<<dim3(nblk * nrhs), threads, smem, st>>>(A, x, y, part, nrhs);
    count_launch(1);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    return launch_group_combine<double, OP_MASS>(G, part, A.npart, y, nrhs, false, st);
}

}  // namespace bras
