"""Dense monomial polynomials on the reference simplex, integrated exactly.

A scalar polynomial in d variables of degree <= D is a coefficient vector over
``monomials(d, D)``.  The reference simplex has vertices 0, e_1, .., e_d and the exact
integral of a monomial over it is ``prod(a_i!) / (|a| + d)!`` (Dirichlet integral).
"""
from __future__ import annotations

import functools
import itertools
import math

import numpy as np


@functools.lru_cache(maxsize=None)
def monomials(d: int, D: int) -> tuple[tuple[int, ...], ...]:
    """Exponent tuples of total degree <= D, ordered by degree, then descending lex."""
    out = []
    for deg in range(D + 1):
        out.extend(sorted((a for a in itertools.product(range(deg + 1), repeat=d) if sum(a) == deg),
                          reverse=True))
    return tuple(out)


def simplex_monomial_integral(a: tuple[int, ...]) -> float:
    d = len(a)
    return math.prod(math.factorial(x) for x in a) / math.factorial(sum(a) + d)


@functools.lru_cache(maxsize=None)
def gram(d: int, D: int) -> np.ndarray:
    """G[i, j] = integral over the reference simplex of m_i * m_j."""
    ms = monomials(d, D)
    G = np.empty((len(ms), len(ms)))
    for i, a in enumerate(ms):
        for j, b in enumerate(ms):
            G[i, j] = simplex_monomial_integral(tuple(x + y for x, y in zip(a, b)))
    return G


def eval_monomials(d: int, D: int, pts: np.ndarray) -> np.ndarray:
    """[n_pts, n_mono] values of the monomials at points [n_pts, d]."""
    ms = monomials(d, D)
    pts = np.atleast_2d(pts)
    out = np.ones((pts.shape[0], len(ms)))
    for j, a in enumerate(ms):
        for c in range(d):
            if a[c]:
                out[:, j] *= pts[:, c] ** a[c]
    return out


def _poly2_mul(p: np.ndarray, q: np.ndarray) -> np.ndarray:
    """Product of two polynomials in (s, t) stored as arrays P[i, j] -> s^i t^j."""
    out = np.zeros((p.shape[0] + q.shape[0] - 1, p.shape[1] + q.shape[1] - 1))
    for i in range(p.shape[0]):
        for j in range(p.shape[1]):
            if p[i, j] != 0.0:
                out[i:i + q.shape[0], j:j + q.shape[1]] += p[i, j] * q
    return out


def restrict_to_param(a: tuple[int, ...], origin: np.ndarray, tangents: list[np.ndarray]) -> np.ndarray:
    """Monomial x^a along x = origin + sum_r u_r tangents[r], as a 2-variable array.

    With one tangent the second axis has length 1 (a polynomial in u_1 only).
    """
    n_par = len(tangents)
    out = np.ones((1, 1))
    for c, e in enumerate(a):
        lin = np.zeros((2, 2)) if n_par == 2 else np.zeros((2, 1))
        lin[0, 0] = origin[c]
        lin[1, 0] = tangents[0][c]
        if n_par == 2:
            lin[0, 1] = tangents[1][c]
        for _ in range(e):
            out = _poly2_mul(out, lin)
    return out


def integrate_segment(P: np.ndarray) -> float:
    """Integral over u in [0, 1] of sum_i P[i, 0] u^i."""
    return float(sum(P[i, 0] / (i + 1) for i in range(P.shape[0])))


def integrate_triangle(P: np.ndarray) -> float:
    """Integral over the reference triangle {s, t >= 0, s + t <= 1} of sum P[i, j] s^i t^j."""
    tot = 0.0
    for i in range(P.shape[0]):
        for j in range(P.shape[1]):
            if P[i, j] != 0.0:
                tot += P[i, j] * math.factorial(i) * math.factorial(j) / math.factorial(i + j + 2)
    return tot


def shifted_legendre(j: int) -> np.ndarray:
    """Power-basis coefficients (ascending) of P_j(2u - 1) on [0, 1]."""
    leg = np.polynomial.Legendre.basis(j, domain=[0.0, 1.0]).convert(kind=np.polynomial.Polynomial)
    return np.asarray(leg.coef, dtype=np.float64)
