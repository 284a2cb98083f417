"""Schur complement of the mixed Poisson saddle point (Sec. 4 and Sec. 5.1): test infrastructure.

Mixed Poisson in H(div) x L^2: [[M, B^T], [B, 0]] with M the H(div) mass matrix and
B_ij = (div phi_j, chi_i) (Sec. 5.1).  Eliminating sigma gives the positive Schur complement
-S = B M^{-1} B^T (Eq. positive_schur_general with C = 0), and replacing M^{-1} by the BRAS
approximation gives -S~ = B M_bras^{-1} B^T (Eq. approx_positive_schur_general).

Pairs: BDM_k / DG_{k-1} (the pair of Sec. 5.1) and RT_k / DG_{k-1} on tetrahedra (div maps
both onto P_{k-1}).  Q basis: on the reference tetrahedron the polynomials of
degree <= k-1 orthonormal for the mean inner product (Gram-Schmidt of the monomials in the
order of ``monomials(3, .)``), mapped without a Piola transform (chi = chi^ o F^{-1}).  The
conforming H(div) space is the contravariant Piola one, phi = J phi^ / det J (the mass matrices
may use |det J| because a per-cell sign cancels in M_K), so div phi = div^ phi^ / det J and cell
K's block of B is sign(det J_K) B^ with B^_ij = int_ref div^ phi^_j chi^_i.  The spectrum of
S~^{-1} S does not depend on the Q basis (a change of basis is a congruence of both S and S~).
"""
from __future__ import annotations

import math

import mpmath
import numpy as np
import scipy.sparse as sp

from .assembly import jacobians
from .elements import _orthonormal_coeffs_tet, reference_element
from .polynomials import monomials, simplex_monomial_integral, to_mpf


def n_dg(order_rt: int) -> int:
    """Local dimension of DG_{k-1} on a tetrahedron."""
    k = order_rt
    return k * (k + 1) * (k + 2) // 6


def reference_divergence(k: int, space: str = "hdiv") -> np.ndarray:
    """B^ [n_dg, n_loc]: exact divergence of the RT_k ("hdiv") or BDM_k ("bdm") basis (monomial
    coefficients) against the orthonormal Q basis, integrated exactly."""
    ref = reference_element(space, 3, k)
    ms = monomials(3, k)
    idx = {m: i for i, m in enumerate(ms)}
    nm = len(ms)
    qs = monomials(3, k - 1)
    C = _orthonormal_coeffs_tet(k - 1)                        # chi_r = sum_i C[r, i] x^{q_i}
    B = np.zeros((len(qs), ref.n_loc))
    for j in range(ref.n_loc):
        div = {}                                              # monomial -> coefficient
        for c in range(3):
            for m, i in idx.items():
                cf = ref.phi_mp[c * nm + i, j]
                if cf != 0 and m[c] > 0:
                    dm = tuple(e - (1 if t == c else 0) for t, e in enumerate(m))
                    div[dm] = div.get(dm, 0) + cf * m[c]
        for r in range(len(qs)):
            acc = mpmath.mpf(0)
            for qi, q in enumerate(qs):
                if C[r, qi] == 0:
                    continue
                for dm, cf in div.items():
                    acc += C[r, qi] * cf * to_mpf(simplex_monomial_integral(tuple(a + b for a, b in zip(dm, q))))
            B[r, j] = float(acc)
    return B


def divergence_matrix(mesh, l2g, signs, n_dof: int, k: int, space: str = "hdiv") -> sp.csr_matrix:
    """Global B [n_cell * n_dg, n_dof]: cell K's DG dofs are rows K * n_dg .. K * n_dg + n_dg - 1."""
    Bh = reference_divergence(k, space)
    E, nloc = l2g.shape
    nq = Bh.shape[0]
    sdet = np.sign(np.linalg.det(jacobians(mesh.coords, mesh.cells)))
    s = (np.ones((E, nloc)) if signs is None else signs.astype(float)) * sdet[:, None]
    rows = (np.arange(E)[:, None, None] * nq + np.arange(nq)[None, :, None]).repeat(nloc, axis=2)
    cols = np.broadcast_to(l2g[:, None, :], (E, nq, nloc))
    vals = Bh[None, :, :] * s[:, None, :]
    return sp.csr_matrix((vals.ravel(), (rows.ravel(), cols.ravel())), shape=(E * nq, n_dof))


def schur_bras(B: sp.spmatrix, bras: sp.spmatrix) -> sp.csr_matrix:
    """-S~ = B M_bras^{-1} B^T (Eq. approx_positive_schur_general, C = 0)."""
    return (B @ bras @ B.T).tocsr()


def schur_exact_dense(B: sp.spmatrix, M: sp.spmatrix) -> np.ndarray:
    """-S = B M^{-1} B^T, dense (small meshes only)."""
    Bd = B.toarray()
    return Bd @ np.linalg.solve(M.toarray(), Bd.T)
