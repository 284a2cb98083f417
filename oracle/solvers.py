"""Textbook solvers and dense spectral tools (Sec. 3 of the paper).

* ``pcg``: Hestenes-Stiefel preconditioned CG, u_0 = 0, stopped when the recurrence
  residual satisfies ||r_k||_2 / ||r_0||_2 <= rtol, or after maxit iterations (Sec. 3:
  rtol 1e-10, 5000 iterations).  Several right-hand sides are independent solves.
* ``fixed_point``: damped u_{k+1} = u_k + omega Mt^{-1} (f - M u_k) (Sec. 3).
* ``kappa_hat``: spectral condition number lambda_max / lambda_min of the pencil
  (M, Mt) (Eq. spectral-kappa), from eigenvalues of L^T X L where M = L L^T and
  X = Mt^{-1} (similar to X M).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def pcg(A, b, precond=None, rtol: float = 1e-10, maxit: int = 5000, max_its: int | None = None):
    """Returns (x, iterations, history of ||r_k||/||r_0||).

    ``max_its`` (if given) runs exactly that many iterations with no stopping test.
    """
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    r = b.copy()
    z = precond(r) if precond is not None else r.copy()
    p = z.copy()
    rz = float(r @ z)
    r0 = float(np.sqrt(r @ r))
    hist = [1.0]
    its = 0
    limit = max_its if max_its is not None else maxit
    while its < limit:
        if max_its is None and hist[-1] <= rtol:
            break
        q = A(p)
        alpha = rz / float(p @ q)
        x += alpha * p
        r -= alpha * q
        its += 1
        hist.append(float(np.sqrt(r @ r)) / r0)
        if max_its is None and hist[-1] <= rtol:
            break
        z = precond(r) if precond is not None else r.copy()
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, its, np.array(hist)


def fixed_point(A, b, precond, omega: float, rtol: float = 1e-10, maxit: int = 5000):
    b = np.asarray(b, dtype=np.float64)
    u = np.zeros_like(b)
    r = b.copy()
    r0 = float(np.linalg.norm(r))
    its = 0
    while its < maxit and np.linalg.norm(r) / r0 > rtol:
        u = u + omega * precond(r)
        r = b - A(u)
        its += 1
    return u, its


def pencil_eigs(M_dense: np.ndarray, X_dense: np.ndarray) -> np.ndarray:
    """Eigenvalues of X M (X SPD approximation of M^{-1}), ascending."""
    L = np.linalg.cholesky(M_dense)
    return sla.eigvalsh(L.T @ X_dense @ L)


def kappa_hat(M_dense: np.ndarray, X_dense: np.ndarray) -> float:
    ev = pencil_eigs(M_dense, X_dense)
    return float(ev[-1] / ev[0])
