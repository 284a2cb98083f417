// Instantiations of the block kernels: launch_pk_f32.
#include <algorithm>

#include "dispatch.h"

namespace bras {

cudaError_t launch_pk_f32(const LaunchCommon& L, int nloc, int op, const float* x, float* y, float* part, int nrhs, cudaStream_t st) {
#define BRAS_CASE(N, OPV) \
    if (nloc == N && op == OPV) \
        return launch_block<N, float, float, KIND_PACKED, OPV>(L.A, L.G, L.nblk, x, y, part, nrhs, st);
    BRAS_CASE(3, OP_MASS)
    BRAS_CASE(3, OP_BRAS)
    BRAS_CASE(8, OP_MASS)
    BRAS_CASE(8, OP_BRAS)
    BRAS_CASE(4, OP_MASS)
    BRAS_CASE(4, OP_BRAS)
    BRAS_CASE(6, OP_MASS)
    BRAS_CASE(6, OP_BRAS)
    BRAS_CASE(15, OP_MASS)
    BRAS_CASE(15, OP_BRAS)
    BRAS_CASE(20, OP_MASS)
    BRAS_CASE(20, OP_BRAS)
    BRAS_CASE(36, OP_MASS)
    BRAS_CASE(36, OP_BRAS)
    BRAS_CASE(45, OP_MASS)
    BRAS_CASE(45, OP_BRAS)
    BRAS_CASE(24, OP_MASS)
    BRAS_CASE(24, OP_BRAS)
    BRAS_CASE(70, OP_MASS)
    BRAS_CASE(70, OP_BRAS)
    BRAS_CASE(84, OP_MASS)
    BRAS_CASE(84, OP_BRAS)
    BRAS_CASE(12, OP_MASS)
    BRAS_CASE(12, OP_BRAS)
    BRAS_CASE(30, OP_MASS)
    BRAS_CASE(30, OP_BRAS)
    BRAS_CASE(60, OP_MASS)
    BRAS_CASE(60, OP_BRAS)
    BRAS_CASE(105, OP_MASS)
    BRAS_CASE(105, OP_BRAS)
#undef BRAS_CASE
    return cudaErrorInvalidValue;
}

}  // namespace bras
