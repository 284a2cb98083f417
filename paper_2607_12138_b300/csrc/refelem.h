// Reference-element mass blocks of the supported element families (host side).
#pragma once
#include <functional>
#include <vector>

namespace bras {

struct RefTables {
    int dim = 0, space = 0, order = 0, nloc = 0, ncomp = 0;
    // R[(a * ncomp + b) * nloc * nloc + i * nloc + j] = int_ref phi_i^a phi_j^b
    std::vector<double> R;
    // RT_k on tetrahedra only: Bdiv[i * nloc + j] = int_ref div phi_j chi_i, chi_i the
    // mean-orthonormal polynomials of degree <= k - 1 (nq of them; DG_{k-1})
    int nq = 0;
    std::vector<double> Bdiv;
};

// basis: H1 0 = Lagrange (equispaced nodes), 1 = Bernstein, 2 = Lagrange at GLL-based nodes;
// H(curl) / H(div) 0 = first kind (N1curl_k / RT_k), 1 = second kind (N2curl_k / BDM_k).
int n_local(int dim, int space, int order, int basis = 0);
int build_reference(int dim, int space, int order, RefTables* out, int basis = 0);

}  // namespace bras
