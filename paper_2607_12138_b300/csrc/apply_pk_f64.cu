// Instantiations of the block kernels: launch_pk_f64.
#include <algorithm>

#include "dispatch.h"

namespace bras {

cudaError_t launch_pk_f64(const LaunchCommon& L, int nloc, int op, const double* x, double* y, double* part, int nrhs, cudaStream_t st) {
#define BRAS_CASE(N, OPV) \
    if (nloc == N && op == OPV) \
        return launch_block<N, double, double, KIND_PACKED, OPV>(L.A, L.G, L.nblk, x, y, part, nrhs, st);
    BRAS_CASE(3, OP_MASS)
    BRAS_CASE(3, OP_BRAS)
    BRAS_CASE(3, OP_DIAG)
    BRAS_CASE(8, OP_MASS)
    BRAS_CASE(8, OP_BRAS)
    BRAS_CASE(8, OP_DIAG)
    BRAS_CASE(4, OP_MASS)
    BRAS_CASE(4, OP_BRAS)
    BRAS_CASE(4, OP_DIAG)
    BRAS_CASE(6, OP_MASS)
    BRAS_CASE(6, OP_BRAS)
    BRAS_CASE(6, OP_DIAG)
    BRAS_CASE(15, OP_MASS)
    BRAS_CASE(15, OP_BRAS)
    BRAS_CASE(15, OP_DIAG)
    BRAS_CASE(20, OP_MASS)
    BRAS_CASE(20, OP_BRAS)
    BRAS_CASE(20, OP_DIAG)
    BRAS_CASE(36, OP_MASS)
    BRAS_CASE(36, OP_BRAS)
    BRAS_CASE(36, OP_DIAG)
    BRAS_CASE(45, OP_MASS)
    BRAS_CASE(45, OP_BRAS)
    BRAS_CASE(45, OP_DIAG)
    BRAS_CASE(24, OP_MASS)
    BRAS_CASE(24, OP_BRAS)
    BRAS_CASE(24, OP_DIAG)
    BRAS_CASE(70, OP_MASS)
    BRAS_CASE(70, OP_BRAS)
    BRAS_CASE(70, OP_DIAG)
    BRAS_CASE(84, OP_MASS)
    BRAS_CASE(84, OP_BRAS)
    BRAS_CASE(84, OP_DIAG)
    BRAS_CASE(12, OP_MASS)
    BRAS_CASE(12, OP_BRAS)
    BRAS_CASE(12, OP_DIAG)
    BRAS_CASE(30, OP_MASS)
    BRAS_CASE(30, OP_BRAS)
    BRAS_CASE(30, OP_DIAG)
    BRAS_CASE(60, OP_MASS)
    BRAS_CASE(60, OP_BRAS)
    BRAS_CASE(60, OP_DIAG)
    BRAS_CASE(105, OP_MASS)
    BRAS_CASE(105, OP_BRAS)
    BRAS_CASE(105, OP_DIAG)
#undef BRAS_CASE
    return cudaErrorInvalidValue;
}

}  // namespace bras
