"""Adjoint gradient of the density-weighted mass solve x = M(rho)^{-1} b.

M(rho) = sum_K rho_K P_K^T M_K^1 P_K, with M_K^1 the unit-density element matrix (the
weight enters the H1 pullback exactly like det J does, Eq. piola_mass_pullbacks).
For a loss L(x) with xbar = dL/dx:
    lambda = M^{-1} xbar            (M is symmetric),   bbar = lambda,
    rhobar_K = -lambda_K^T M_K^1 x_K,  lambda_K = P_K lambda, x_K = P_K x,
and for rho = exp(z), zbar = rhobar * rho.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .assembly import assemble_mass, element_matrices, signed_values


def rho_bar(Me_unit: np.ndarray, l2g, signs, x: np.ndarray, lam: np.ndarray) -> np.ndarray:
    s = signed_values(l2g, signs)
    xK = s * x[l2g]
    lK = s * lam[l2g]
    return -np.einsum("ka,kab,kb->k", lK, Me_unit, xK)


def loss_and_grad(mesh, space, order, l2g, signs, n_dof, z, b, x_star):
    """Exact (sparse direct) loss 0.5||x - x*||^2 and its gradients (bbar, zbar)."""
    Me1 = element_matrices(mesh.coords, mesh.cells, space, order)
    rho = np.exp(z)
    M = assemble_mass(l2g, signs, Me1 * rho[:, None, None], n_dof).tocsc()
    lu = spla.splu(M)
    x = lu.solve(b)
    xbar = x - x_star
    lam = lu.solve(xbar)
    rb = rho_bar(Me1, l2g, signs, x, lam)
    return 0.5 * float(xbar @ xbar), lam, rb * rho, x
