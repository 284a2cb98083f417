"""Element matrices, assembled M, multiplicity D and the explicit BRAS matrix (FP64).

Follows Sec. 2 of the paper:
  * M = P^T M_br P = sum_K P_K^T M_K P_K                         (Eq. M_PMbrP)
  * D = P^T P = diag(d_i), d_i = number of broken copies of dof i  (Sec. 2.2)
  * M_bras^{-1} = D^{-1} (sum_K P_K^T M_K^{-1} P_K) D^{-1}          (Eq. mhatinvbras_def,
                                                                    element-sum form)
  * M_diag^{-1} = diag(M)^{-1}                                       (Sec. 2.1)
  * element matrices by the Piola pullbacks (Eq. piola_mass_pullbacks): metric
    |det J| (H1), |det J| J^{-1} J^{-T} (H(curl)), J^T J / |det J| (H(div)).
The signed injection has (P)_{(K,a), l2g[K,a]} = signs[K,a]; D is still the copy count.
Each M_K^{-1} comes from an FP64 Cholesky factorisation of M_K.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .elements import reference_element


def jacobians(coords: np.ndarray, cells: np.ndarray) -> np.ndarray:
    """J_K = [x_1 - x_0, .., x_d - x_0] (columns), shape [E, d, d]."""
    X = coords[cells]                                   # [E, d+1, d]
    return np.transpose(X[:, 1:, :] - X[:, :1, :], (0, 2, 1))


def metrics(space: str, J: np.ndarray) -> np.ndarray:
    """Pulled-back mass coefficient G_K of Eq. piola_mass_pullbacks, with |det J|."""
    det = np.abs(np.linalg.det(J))
    if space in ("h1", "h1b", "h1g"):   # Lagrange (equispaced or GLL nodes) or Bernstein: scalar pullback
        return det[:, None, None]
    if space in ("hcurl", "n2curl"):
        Jinv = np.linalg.inv(J)
        return det[:, None, None] * Jinv @ np.transpose(Jinv, (0, 2, 1))
    if space in ("hdiv", "bdm"):
        return np.transpose(J, (0, 2, 1)) @ J / det[:, None, None]
    raise ValueError(space)


def element_matrices(coords, cells, space: str, order: int, rho=None) -> np.ndarray:
    """M_K for every cell, [E, n_loc, n_loc]; rho scales each M_K (density weight)."""
    dim = coords.shape[1]
    ref = reference_element(space, dim, order)
    R = ref.mass_blocks()                               # [c, c, n, n]
    G = metrics(space, jacobians(coords, cells))        # [E, c, c]
    Me = np.einsum("kab,abij->kij", G, R)
    if rho is not None:
        Me = Me * np.asarray(rho, dtype=np.float64)[:, None, None]
    return Me


def signed_values(l2g: np.ndarray, signs) -> np.ndarray:
    return np.ones(l2g.shape) if signs is None else np.asarray(signs, dtype=np.float64)


def injection(l2g: np.ndarray, signs, n_dof: int) -> sp.csr_matrix:
    """The conforming-to-broken map P, [n_br, n] (row (K,a) has sign at column l2g[K,a])."""
    E, n = l2g.shape
    rows = np.arange(E * n)
    return sp.csr_matrix((signed_values(l2g, signs).ravel(), (rows, l2g.ravel())), shape=(E * n, n_dof))


def multiplicity(l2g: np.ndarray, n_dof: int) -> np.ndarray:
    return np.bincount(l2g.ravel(), minlength=n_dof).astype(np.float64)


def _assemble_blocks(l2g, signs, blocks, n_dof) -> sp.csr_matrix:
    E, n = l2g.shape
    s = signed_values(l2g, signs)
    vals = blocks * s[:, :, None] * s[:, None, :]
    rows = np.repeat(l2g[:, :, None], n, axis=2)
    cols = np.repeat(l2g[:, None, :], n, axis=1)
    A = sp.coo_matrix((vals.ravel(), (rows.ravel(), cols.ravel())), shape=(n_dof, n_dof))
    return A.tocsr()


def assemble_mass(l2g, signs, Me, n_dof) -> sp.csr_matrix:
    """M = sum_K P_K^T M_K P_K."""
    return _assemble_blocks(l2g, signs, Me, n_dof)


def local_inverses(Me: np.ndarray) -> np.ndarray:
    """M_K^{-1} = L^{-T} L^{-1} from the FP64 Cholesky factor M_K = L L^T of each cell."""
    L = np.linalg.cholesky(Me)
    eye = np.broadcast_to(np.eye(Me.shape[1]), Me.shape)
    W = np.linalg.solve(L, eye)                       # L^{-1}, batched
    return np.transpose(W, (0, 2, 1)) @ W


def bras_inverse(l2g, signs, Me, n_dof, Minv=None) -> sp.csr_matrix:
    """Explicit M_bras^{-1} = D^{-1} (sum_K P_K^T M_K^{-1} P_K) D^{-1}."""
    if Minv is None:
        Minv = local_inverses(Me)
    S = _assemble_blocks(l2g, signs, Minv, n_dof)
    Dinv = sp.diags(1.0 / multiplicity(l2g, n_dof))
    return (Dinv @ S @ Dinv).tocsr()


def jacobi_diag(M: sp.spmatrix) -> np.ndarray:
    return np.asarray(M.diagonal()).copy()


class Problem:
    """Everything the oracle needs about one discretisation, assembled once."""

    def __init__(self, mesh, space: str, order: int, l2g, signs, n_dof: int, rho=None):
        self.space, self.order, self.n_dof = space, order, n_dof
        self.l2g, self.signs = l2g, signs
        self.Me = element_matrices(mesh.coords, mesh.cells, space, order, rho)
        self.M = assemble_mass(l2g, signs, self.Me, n_dof)
        self.Minv_loc = local_inverses(self.Me)
        self.B = bras_inverse(l2g, signs, self.Me, n_dof, self.Minv_loc)
        self.diag = jacobi_diag(self.M)
        self.d = multiplicity(l2g, n_dof)

    def mass_apply(self, x):
        return self.M @ x

    def bras_apply(self, x):
        return self.B @ x

    def jacobi_apply(self, x):
        x = np.asarray(x)
        return x / (self.diag if x.ndim == 1 else self.diag[:, None])
