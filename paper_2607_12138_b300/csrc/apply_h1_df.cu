// Instantiations of the H1 mass apply with float-float local products (FP64 vectors and
// scatter sums), used for the refinement residual.
#include <algorithm>

#include "df_kernels.cuh"
#include "dispatch.h"

namespace bras {

cudaError_t launch_h1_df(const LaunchCommon& L, int nloc, const double* x, double* y, double* part, int nrhs,
                         cudaStream_t st) {
#define BRAS_CASE(N)                                                                                    \
    if (nloc == N)                                                                                      \
        return launch_block_df<N>(L.A, L.G, L.nblk, x, y, part, nrhs, st);
    BRAS_CASE(3)
    BRAS_CASE(4)
    BRAS_CASE(6)
    BRAS_CASE(10)
    BRAS_CASE(15)
    BRAS_CASE(20)
    BRAS_CASE(35)
#undef BRAS_CASE
    return cudaErrorInvalidValue;
}

}  // namespace bras
