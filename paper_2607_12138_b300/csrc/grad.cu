// Element part of the adjoint gradient of the weighted mass solve, and weight updates.
//
// For M(rho) = sum_K rho_K P_K^T M_K^1 P_K with M_K^1 = |det J_K| M_ref (the weight enters the
// H1 pullback of Eq. piola_mass_pullbacks like det J does), dL/drho_K = -lambda_K^T M_K^1 x_K
// where lambda = M^{-1} dL/dx.  One thread per cell: signed gathers of x and lambda through
// the scatter tables and the quadratic form with M_ref from shared memory, fused.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"
#include "packet.h"

namespace bras {

template <int NLOC>
__global__ void k_grad_rho(int64_t E, int BE, const int32_t* __restrict__ blk_e0, const int32_t* __restrict__ blk_u0,
                           const int64_t* __restrict__ blk_pkt, const unsigned char* __restrict__ pkt,
                           const int32_t* __restrict__ perm, const double* __restrict__ absdet,
                           const double* __restrict__ Mref, const double* __restrict__ x,
                           const double* __restrict__ lam, double* __restrict__ rho_bar,
                           const double* __restrict__ rho_log) {
    __shared__ double Ms[NLOC * NLOC];
    for (int i = threadIdx.x; i < NLOC * NLOC; i += blockDim.x) Ms[i] = Mref[i];
    __syncthreads();
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(e / BE);
        const int e0 = blk_e0[b], ne = blk_e0[b + 1] - e0, el = (int)(e - e0);
        const uint32_t nu = (uint32_t)(blk_u0[b + 1] - blk_u0[b]);
        const unsigned char* P = pkt + blk_pkt[b];
        const int32_t* ids = reinterpret_cast<const int32_t*>(P);
        const uint16_t* L = reinterpret_cast<const uint16_t*>(P + pkt_size_a(nu, false)) + el;
        double xl[NLOC], ll[NLOC];
#pragma unroll
        for (int a = 0; a < NLOC; ++a) {
            const uint16_t c = L[a * ne];
            const int g = ids[c & 0x7fff];
            const double s = (c & 0x8000) ? -1.0 : 1.0;
            xl[a] = s * x[g];
            ll[a] = s * lam[g];
        }
        double acc = 0.0;
#pragma unroll
        for (int a = 0; a < NLOC; ++a) {
            double t = 0.0;
#pragma unroll
            for (int q = 0; q < NLOC; ++q) t = fma(Ms[a * NLOC + q], xl[q], t);
            acc = fma(ll[a], t, acc);
        }
        // rho_log: the log-density gradient zbar_K = rhobar_K * rho_K (rho = exp(z))
        rho_bar[perm[e]] = -absdet[e] * acc * (rho_log ? rho_log[e] : 1.0);
    }
}

cudaError_t grad_rho_launch(const bras_ctx* c, const double* x, const double* lam, double* rho_bar, bool wrt_log,
                            cudaStream_t st) {
    const double* rl = wrt_log ? c->rho : nullptr;
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((c->E + 127) / 128, 148 * 8));
#define GRAD_CASE(N)                                                                                              \
    case N:                                                                                                       \
        k_grad_rho<N><<<nb, 128, 0, st>>>(c->E, c->BE, c->blk_e0, c->blk_u0, c->blk_pkt, c->pkt, c->perm, c->absdet, \
                                          c->Mref64, x, lam, rho_bar, rl);                                        \
        count_launch(1);                                                                                          \
        break;
    switch (c->nloc) {
        GRAD_CASE(3)
        GRAD_CASE(4)
        GRAD_CASE(6)
        GRAD_CASE(10)
        GRAD_CASE(15)
        GRAD_CASE(20)
        GRAD_CASE(35)
        default: return cudaErrorInvalidValue;
    }
#undef GRAD_CASE
    return cudaGetLastError();
}

// from_log: the caller passes z with rho = exp(z)
__global__ void k_update_rho(int64_t E, const int32_t* __restrict__ perm, const double* __restrict__ rho_user,
                             const double* __restrict__ absdet, double* __restrict__ rho, double* __restrict__ ms64,
                             double* __restrict__ bs64, float* __restrict__ ms32, float* __restrict__ bs32, int from_log) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        const double rw = from_log ? exp(rho_user[perm[e]]) : rho_user[perm[e]];
        const double m = rw * absdet[e];
        rho[e] = rw;
        ms64[e] = m;
        bs64[e] = 1.0 / m;
        ms32[e] = (float)m;
        bs32[e] = (float)(1.0 / m);
    }
}

cudaError_t update_rho_launch(bras_ctx* c, const double* rho, bool from_log, cudaStream_t st) {
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((c->E + 255) / 256, 148 * 8));
    k_update_rho<<<nb, 256, 0, st>>>(c->E, c->perm, rho, c->absdet, c->rho, c->mscale64, c->bscale64, c->mscale32,
                                     c->bscale32, from_log ? 1 : 0);
    count_launch(1);
    return cudaGetLastError();
}

}  // namespace bras
