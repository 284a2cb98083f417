// Instantiations of the tensor-core H1 block kernels (FP32 vectors, 3xTF32 local GEMM).
#include <algorithm>

#include "dispatch.h"
#include "tc_kernels.cuh"

namespace bras {

// tensor cores pay off from n_loc = 20 (3D P3) on; smaller local matrices stay on the FP32 units
bool h1_tc_supported(int nloc) { return nloc == 20 || nloc == 35; }

uint32_t h1_tc_btile_bytes(int nloc) {
    switch (nloc) {
        case 10: return 2 * TcShape<10>::B_BYTES;
        case 15: return 2 * TcShape<15>::B_BYTES;
        case 20: return 2 * TcShape<20>::B_BYTES;
        case 35: return 2 * TcShape<35>::B_BYTES;
        default: return 0;
    }
}

size_t h1_tc_smem_bytes(int nloc, const BlockArgs& A, bool mr) {
    switch (nloc) {
        case 10: return tc_smem_bytes<10>(A, mr);
        case 15: return tc_smem_bytes<15>(A, mr);
        case 20: return tc_smem_bytes<20>(A, mr);
        case 35: return tc_smem_bytes<35>(A, mr);
        default: return 0;
    }
}

cudaError_t launch_h1_tc(const LaunchCommon& L, const unsigned char* btile, int nloc, int op, const float* x,
                         float* y, float* part, int nrhs, cudaStream_t st) {
    TcArgs TA;
    TA.A = L.A;
    TA.btile = btile;
#define BRAS_CASE(N, OPV)                                                                                   \
    if (nloc == N && op == OPV)                                                                             \
        return launch_block_tc<N, OPV>(TA, L.G, L.nblk, x, y, part, nrhs, st);
    BRAS_CASE(10, OP_MASS)
    BRAS_CASE(10, OP_BRAS)
    BRAS_CASE(15, OP_MASS)
    BRAS_CASE(15, OP_BRAS)
    BRAS_CASE(20, OP_MASS)
    BRAS_CASE(20, OP_BRAS)
    BRAS_CASE(35, OP_MASS)
    BRAS_CASE(35, OP_BRAS)
#undef BRAS_CASE
    return cudaErrorInvalidValue;
}

// Reference matrix (row-major n x n, FP64) -> [big | small] TF32 split in the no-swizzle
// K-major core-matrix layout of an N x K operand (zero padded), as raw bytes.
void h1_tc_build_btile(const double* ref, int nloc, std::vector<unsigned char>& out) {
    const int K = (nloc + 7) / 8 * 8, N = (nloc + 15) / 16 * 16;
    const size_t one = (size_t)N * K * 4;
    out.assign(2 * one, 0);
    for (int n = 0; n < nloc; ++n)
        for (int k = 0; k < nloc; ++k) {
            const float f = (float)ref[(size_t)n * nloc + k];
            uint32_t u;
            std::memcpy(&u, &f, 4);
            uint32_t big = u;
            if ((u & 0x7f800000u) != 0x7f800000u) big = (u + 0x1000u) & 0xFFFFE000u;   // round to nearest, ties away
            float fb;
            std::memcpy(&fb, &big, 4);
            const float fs = f - fb;
            const uint32_t off = umma_kmajor_offset(n, k, K);
            std::memcpy(out.data() + off, &fb, 4);
            std::memcpy(out.data() + one + off, &fs, 4);
        }
}

}  // namespace bras
