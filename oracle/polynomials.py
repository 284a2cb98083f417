"""Monomial polynomials on the reference simplex, integrated exactly.

A scalar polynomial in d variables of degree <= D is a coefficient vector over
``monomials(d, D)``.  The reference simplex has vertices 0, e_1, .., e_d and the exact
integral of a monomial over it is ``prod(a_i!) / (|a| + d)!`` (Dirichlet integral).
Integrals are exact rationals (``fractions.Fraction``); the element construction carries
them in 40-digit ``mpmath`` arithmetic and rounds to FP64 once, at the end.
"""
from __future__ import annotations

import functools
import itertools
import math
from fractions import Fraction

import mpmath
import numpy as np

mpmath.mp.dps = 40


@functools.lru_cache(maxsize=None)
def monomials(d: int, D: int) -> tuple[tuple[int, ...], ...]:
    """Exponent tuples of total degree <= D, ordered by degree, then descending lex."""
    out = []
    for deg in range(D + 1):
        out.extend(sorted((a for a in itertools.product(range(deg + 1), repeat=d) if sum(a) == deg),
                          reverse=True))
    return tuple(out)


def simplex_monomial_integral(a: tuple[int, ...]) -> Fraction:
    d = len(a)
    return Fraction(math.prod(math.factorial(x) for x in a), math.factorial(sum(a) + d))


@functools.lru_cache(maxsize=None)
def gram(d: int, D: int) -> mpmath.matrix:
    """G[i, j] = integral over the reference simplex of m_i * m_j (exact, as mpf)."""
    ms = monomials(d, D)
    G = mpmath.matrix(len(ms), len(ms))
    for i, a in enumerate(ms):
        for j, b in enumerate(ms):
            f = simplex_monomial_integral(tuple(x + y for x, y in zip(a, b)))
            G[i, j] = mpmath.mpf(f.numerator) / f.denominator
    return G


def eval_monomials(d: int, D: int, pts: np.ndarray) -> np.ndarray:
    """[n_pts, n_mono] FP64 values of the monomials at points [n_pts, d]."""
    ms = monomials(d, D)
    pts = np.atleast_2d(pts)
    out = np.ones((pts.shape[0], len(ms)))
    for j, a in enumerate(ms):
        for c in range(d):
            if a[c]:
                out[:, j] *= pts[:, c] ** a[c]
    return out


def _poly2_mul(p: dict, q: dict) -> dict:
    out: dict = {}
    for (i, j), a in p.items():
        for (k, l), b in q.items():
            out[(i + k, j + l)] = out.get((i + k, j + l), 0) + a * b
    return out


def restrict_to_param(a: tuple[int, ...], origin, tangents) -> dict:
    """Monomial x^a along x = origin + sum_r u_r tangents[r] as {(i, j): Fraction} in (u_1, u_2).

    origin / tangents have rational entries; with one tangent only j = 0 appears.
    """
    out = {(0, 0): Fraction(1)}
    for c, e in enumerate(a):
        lin = {(0, 0): Fraction(origin[c]), (1, 0): Fraction(tangents[0][c])}
        if len(tangents) == 2:
            lin[(0, 1)] = Fraction(tangents[1][c])
        for _ in range(e):
            out = _poly2_mul(out, lin)
    return out


def integrate_segment(P: dict) -> Fraction:
    """Integral over u in [0, 1] of sum P[(i, 0)] u^i."""
    return sum((c / (i + 1) for (i, j), c in P.items()), Fraction(0))


def integrate_triangle(P: dict) -> Fraction:
    """Integral over {s, t >= 0, s + t <= 1} of sum P[(i, j)] s^i t^j."""
    return sum((c * Fraction(math.factorial(i) * math.factorial(j), math.factorial(i + j + 2))
                for (i, j), c in P.items()), Fraction(0))


def shifted_legendre(j: int) -> list[Fraction]:
    """Power-basis coefficients (ascending) of P_j(2u - 1) on [0, 1] (Rodrigues form:
    P_j(2u - 1) = sum_i (-1)^(j+i) C(j, i) C(j+i, i) u^i)."""
    return [Fraction((-1) ** (j + i) * math.comb(j, i) * math.comb(j + i, i)) for i in range(j + 1)]


def to_mpf(f: Fraction) -> mpmath.mpf:
    return mpmath.mpf(f.numerator) / f.denominator
