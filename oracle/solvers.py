"""Textbook solvers and dense spectral tools (Sec. 3 of the paper).

* ``pcg``: Hestenes-Stiefel preconditioned CG, u_0 = 0, stopped when the recurrence
  residual satisfies ||r_k||_2 / ||r_0||_2 <= rtol, or after maxit iterations (Sec. 3:
  rtol 1e-10, 5000 iterations).  Several right-hand sides are independent solves.
* ``fixed_point``: damped u_{k+1} = u_k + omega Mt^{-1} (f - M u_k) (Sec. 3).
* ``power_lambda_max``: the power iteration the paper uses for lambda_max(Mt^{-1} M) in
  the fixed-point weights omega_diag = 1 / lambda_max, omega_bras = 2 / (1 + lambda_max)
  (Sec. 3).
* ``chebyshev``: Chebyshev semi-iteration on a spectral interval [lmin, lmax] of
  Mt^{-1} M (Sec. 3: linear, no inner products in the update).
* ``cg_lanczos``: the extreme eigenvalues of the Lanczos tridiagonal matrix that preconditioned
  CG builds implicitly from its coefficients -- estimates of lambda_min, lambda_max of
  Mt^{-1} M and so of kappa_hat (Eq. spectral-kappa) on meshes too large for a dense solve.
* ``kappa_hat``: spectral condition number lambda_max / lambda_min of the pencil
  (M, Mt) (Eq. spectral-kappa), from eigenvalues of L^T X L where M = L L^T and
  X = Mt^{-1} (similar to X M).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def pcg(A, b, precond=None, rtol: float = 1e-10, maxit: int = 5000, max_its: int | None = None,
        coeffs: list | None = None):
    """Returns (x, iterations, history of ||r_k||/||r_0||).

    ``max_its`` (if given) runs exactly that many iterations with no stopping test.
    ``coeffs`` (if a list) receives (alpha_k, beta_k) per iteration, beta_k the coefficient of
    p_k = z_k + beta_k p_{k-1} (beta_0 = 0).
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
    beta = 0.0
    while its < limit:
        if max_its is None and hist[-1] <= rtol:
            break
        q = A(p)
        alpha = rz / float(p @ q)
        if coeffs is not None:
            coeffs.append((alpha, beta))
        x += alpha * p
        r -= alpha * q
        its += 1
        hist.append(float(np.sqrt(r @ r)) / r0)
        if max_its is None and hist[-1] <= rtol:
            break
        z = precond(r) if precond is not None else r.copy()
        rz_new = float(r @ z)
        beta = rz_new / rz
        p = z + beta * p
        rz = rz_new
    return x, its, np.array(hist)


def lanczos_tridiagonal(coeffs) -> np.ndarray:
    """T_k of the Lanczos process that CG on the preconditioned operator performs implicitly:
    T[j, j] = 1/alpha_j + beta_j/alpha_{j-1} (second term from j = 1), T[j, j+1] = T[j+1, j]
    = sqrt(beta_{j+1})/alpha_j."""
    k = len(coeffs)
    T = np.zeros((k, k))
    for j, (a, bta) in enumerate(coeffs):
        T[j, j] = 1.0 / a + (bta / coeffs[j - 1][0] if j > 0 else 0.0)
        if j + 1 < k:
            T[j, j + 1] = T[j + 1, j] = np.sqrt(coeffs[j + 1][1]) / a
    return T


def cg_lanczos(A, b, precond, steps: int):
    """(lambda_min, lambda_max, steps taken) of T_k after ``steps`` CG iterations (fewer if the
    residual vanishes); the Ritz values bracket-in towards the spectrum's ends."""
    coeffs: list = []
    pcg(A, b, precond, rtol=0.0, max_its=steps, coeffs=coeffs)
    ev = np.linalg.eigvalsh(lanczos_tridiagonal(coeffs))
    return float(ev[0]), float(ev[-1]), len(coeffs)


def fixed_point(A, b, precond, omega: float, rtol: float = 1e-10, maxit: int = 5000, max_its: int | None = None):
    """Damped preconditioned Richardson u_{k+1} = u_k + omega Mt^{-1}(f - M u_k), u_0 = 0
    (Sec. 3), stopped on ||f - M u_k|| / ||f|| <= rtol.  Returns (u, iterations).
    ``max_its`` runs exactly that many iterations with no stopping test."""
    b = np.asarray(b, dtype=np.float64)
    u = np.zeros_like(b)
    r = b.copy()
    r0 = float(np.linalg.norm(r))
    its = 0
    limit = max_its if max_its is not None else maxit
    while its < limit and (max_its is not None or np.linalg.norm(r) / r0 > rtol):
        u = u + omega * precond(r)
        r = b - A(u)
        its += 1
    return u, its


def power_lambda_max(A, precond, v0, iters: int):
    """lambda_max of T = Mt^{-1} M by the power iteration (Sec. 3, fixed-point weights).

    T is self-adjoint in the M inner product (u, v)_M = u^T M v, so its Rayleigh quotient
    there is (Mv)^T Mt^{-1} (Mv) / (v^T M v); each step replaces v by T v, rescaled to unit
    2-norm.  Returns the Rayleigh quotient of the last iterate before its update (a lower
    bound of lambda_max that converges to it)."""
    v = np.asarray(v0, dtype=np.float64).copy()
    lam = 0.0
    for _ in range(iters):
        w = A(v)
        z = precond(w)
        lam = float(w @ z) / float(w @ v)
        v = z / np.linalg.norm(z)
    return lam


def chebyshev_coefficients(lmin: float, lmax: float, count: int):
    """(c1[k], c2[k]) of the direction update d_k = c1[k] d_{k-1} + c2[k] Mt^{-1} r_k of the
    Chebyshev semi-iteration on [lmin, lmax]: with theta, delta the centre and half-width of
    the interval and sigma = theta / delta, rho_0 = 1 / sigma, rho_k = 1 / (2 sigma - rho_{k-1});
    c1[0] = 0, c2[0] = 1 / theta, and c1[k] = rho_k rho_{k-1}, c2[k] = 2 rho_k / delta."""
    theta, delta = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
    sigma = theta / delta
    c1, c2 = np.zeros(count), np.zeros(count)
    c2[0] = 1.0 / theta
    rho = 1.0 / sigma
    for k in range(1, count):
        rho_new = 1.0 / (2.0 * sigma - rho)
        c1[k] = rho_new * rho
        c2[k] = 2.0 * rho_new / delta
        rho = rho_new
    return c1, c2


def chebyshev(A, b, precond, lmin: float, lmax: float, rtol: float = 1e-10, maxit: int = 5000,
              max_its: int | None = None):
    """Preconditioned Chebyshev semi-iteration for M u = f on the interval [lmin, lmax] that
    contains the spectrum of Mt^{-1} M (Sec. 3): u_0 = 0, r_0 = f, and for k = 0, 1, ...
    d_k = c1[k] d_{k-1} + c2[k] Mt^{-1} r_k;  u_{k+1} = u_k + d_k;  r_{k+1} = r_k - M d_k,
    so that the error is e_k = T_k((theta - Mt^{-1}M) / delta) / T_k(theta / delta) e_0 with
    T_k the Chebyshev polynomial.  Stops on ||r_k|| / ||r_0|| <= rtol.  Returns (u, iterations)."""
    b = np.asarray(b, dtype=np.float64)
    limit = max_its if max_its is not None else maxit
    c1, c2 = chebyshev_coefficients(lmin, lmax, limit + 1)
    u = np.zeros_like(b)
    r = b.copy()
    d = np.zeros_like(b)
    r0 = float(np.linalg.norm(r))
    its = 0
    while its < limit and (max_its is not None or np.linalg.norm(r) / r0 > rtol):
        d = c1[its] * d + c2[its] * precond(r)
        u = u + d
        r = r - A(d)
        its += 1
    return u, its


def pencil_eigs(M_dense: np.ndarray, X_dense: np.ndarray) -> np.ndarray:
    """Eigenvalues of X M (X SPD approximation of M^{-1}), ascending."""
    L = np.linalg.cholesky(M_dense)
    return sla.eigvalsh(L.T @ X_dense @ L)


def kappa_hat(M_dense: np.ndarray, X_dense: np.ndarray) -> float:
    ev = pencil_eigs(M_dense, X_dense)
    return float(ev[-1] / ev[0])
