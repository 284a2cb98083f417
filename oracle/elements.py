"""Reference elements (Sec. 3 element families) built by dualising a monomial span.

Construction, identical for every family:
  1. a spanning set of the polynomial space written in monomial coefficients;
  2. an orthonormal basis Q of its span (SVD; the rank must equal the known dimension);
  3. the dof functionals F as row vectors over the coefficients;
  4. nodal basis Phi = Q (F Q)^{-1}, so that F Phi = I.

Spaces (reference tetrahedron / triangle with vertices 0, e_1, .., e_d):
  * Lagrange P_p: all monomials of degree <= p; dofs = values at the equispaced nodes
    ``sum alpha_i v_i / p`` (multi-indices in ascending lexicographic order).
  * Nedelec first kind N1curl_k (3D): P_{k-1}^3 + x cross (homogeneous P_{k-1})^3.
  * Raviart-Thomas RT_k (3D): P_{k-1}^3 + x (homogeneous P_{k-1}).
Dof functionals (this project's convention; the paper names Firedrake's families only):
  * edge (a, b), x(u) = v_a + u (v_b - v_a):  int_0^1 phi(x(u)) . (v_b - v_a) L_j(u) du,
    L_j the shifted Legendre polynomial, j = 0..k-1;
  * N1curl face (a, b, c), x(s, t) = v_a + s t1 + t t2 with t1 = v_b - v_a, t2 = v_c - v_a:
    int_T phi . t_m q ds dt over the reference triangle T, q running over the orthonormal
    polynomials of degree <= k-2 on T (q outer, m = 1, 2 inner);
  * RT face: int_T phi . (t1 x t2) q ds dt, q orthonormal of degree <= k-1 on T;
  * interior: int_K phi_c q dx, q orthonormal of degree <= k-3 (N1curl) or <= k-2 (RT) on
    the reference tetrahedron, q outer, component c inner.
"Orthonormal" is for the mean inner product (1/|T|) int f g (so the constant is 1 and the
lowest-order dofs are plain circulations / fluxes): Gram-Schmidt of the monomials in the order of ``_face_test_monomials``
(triangle: degree ascending, then power of t ascending) or ``monomials(3, .)`` (tetrahedron)
with positive leading coefficients, i.e. the rows of L^{-1} for the monomial Gram matrix
G / |T| = L L^T.  Edge and face tuples are lexicographic in the local vertex numbers.
"""
from __future__ import annotations

import functools
import itertools
import math
from dataclasses import dataclass

import numpy as np

from .polynomials import (gram, integrate_segment, integrate_triangle, monomials,
                          eval_monomials, restrict_to_param, shifted_legendre,
                          simplex_monomial_integral)

EDGES_3D = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
FACES_3D = [(0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)]


@dataclass(frozen=True)
class RefElement:
    space: str          # "h1", "hcurl", "hdiv"
    dim: int
    order: int
    degree: int         # max polynomial degree of the basis
    phi: np.ndarray     # [n_comp * n_mono, n_loc] nodal basis coefficients
    n_comp: int

    @property
    def n_loc(self) -> int:
        return self.phi.shape[1]

    def component(self, c: int) -> np.ndarray:
        nm = len(monomials(self.dim, self.degree))
        return self.phi[c * nm:(c + 1) * nm, :]

    def mass_blocks(self) -> np.ndarray:
        """R[a, b] = int_ref phi^a phi^b^T  (shape [n_comp, n_comp, n_loc, n_loc])."""
        G = gram(self.dim, self.degree)
        R = np.empty((self.n_comp, self.n_comp, self.n_loc, self.n_loc))
        for a in range(self.n_comp):
            for b in range(self.n_comp):
                R[a, b] = self.component(a).T @ G @ self.component(b)
        return R

    def evaluate(self, pts: np.ndarray) -> np.ndarray:
        """Reference basis values [n_pts, n_loc, n_comp] at reference points."""
        V = eval_monomials(self.dim, self.degree, pts)
        return np.stack([V @ self.component(c) for c in range(self.n_comp)], axis=2)


def _ref_vertices(d: int) -> np.ndarray:
    return np.vstack([np.zeros(d), np.eye(d)])


def _dualise(span: np.ndarray, F: np.ndarray, dim_expected: int) -> np.ndarray:
    U, s, _ = np.linalg.svd(span, full_matrices=False)
    rank = int(np.sum(s > 1e-10 * s[0]))
    if rank != dim_expected:
        raise AssertionError(f"span rank {rank} != {dim_expected}")
    Q = U[:, :rank]
    A = F @ Q
    if A.shape != (rank, rank):
        raise AssertionError(f"{A.shape[0]} functionals for a space of dimension {rank}")
    return Q @ np.linalg.inv(A)


@functools.lru_cache(maxsize=None)
def lagrange(dim: int, p: int) -> RefElement:
    ms = monomials(dim, p)
    nodes = sorted(a for a in itertools.product(range(p + 1), repeat=dim + 1) if sum(a) == p)
    V = _ref_vertices(dim)
    pts = np.array([np.asarray(a, dtype=np.float64) @ V / p for a in nodes])
    F = eval_monomials(dim, p, pts)                      # point evaluations
    phi = _dualise(np.eye(len(ms)), F, len(ms))
    return RefElement("h1", dim, p, p, phi, 1)


def _vec(c: int, j: int, nm: int) -> np.ndarray:
    v = np.zeros(3 * nm)
    v[c * nm + j] = 1.0
    return v


def _edge_functionals(k: int, nm: int, ms) -> list[np.ndarray]:
    V = _ref_vertices(3)
    rows = []
    for a, b in EDGES_3D:
        tau = V[b] - V[a]
        for j in range(k):
            L = shifted_legendre(j)[:, None]
            row = np.zeros(3 * nm)
            for mi, m in enumerate(ms):
                P = restrict_to_param(m, V[a], [tau])
                val = integrate_segment(np.convolve(P[:, 0], L[:, 0])[:, None])
                for c in range(3):
                    row[c * nm + mi] = tau[c] * val
            rows.append(row)
    return rows


def _orthonormalise(G: np.ndarray) -> np.ndarray:
    """Rows r of C give q_r = sum_i C[r, i] m_i, orthonormal for the Gram matrix G (Gram-Schmidt
    in the given monomial order, positive leading coefficient): C = L^{-1}, G = L L^T."""
    L = np.linalg.cholesky(G)
    return np.linalg.inv(L)


def _orthonormal_coeffs_triangle(deg: int) -> np.ndarray:
    tm = _face_test_monomials(deg)
    G = np.array([[integrate_triangle(_mono2(a[0] + b[0], a[1] + b[1])) for b in tm] for a in tm])
    return _orthonormalise(G / 0.5)          # mean inner product on T (area 1/2)


def _orthonormal_coeffs_tet(deg: int) -> np.ndarray:
    return _orthonormalise(gram(3, deg) * 6.0)   # mean inner product on K (volume 1/6)


def _mono2(i: int, j: int) -> np.ndarray:
    P = np.zeros((i + 1, j + 1))
    P[i, j] = 1.0
    return P


def _face_test_monomials(deg: int) -> list[tuple[int, int]]:
    """s^i t^j with i + j <= deg: degree ascending, then the power of t ascending."""
    return [(d - j, j) for d in range(deg + 1) for j in range(d + 1)]


def _face_functionals(space: str, k: int, nm: int, ms) -> list[np.ndarray]:
    V = _ref_vertices(3)
    rows = []
    qdeg = k - 2 if space == "hcurl" else k - 1
    if qdeg < 0:
        return rows
    for a, b, c in FACES_3D:
        t1, t2 = V[b] - V[a], V[c] - V[a]
        dirs = [t1, t2] if space == "hcurl" else [np.cross(t1, t2)]
        restricted = [restrict_to_param(m, V[a], [t1, t2]) for m in ms]
        tm = _face_test_monomials(qdeg)
        # ints_mono[i, mi] = int_T m_mi(x(s,t)) s^a t^b ds dt for the i-th face monomial
        ints_mono = np.zeros((len(tm), nm))
        for i, (qi, qj) in enumerate(tm):
            for mi, P in enumerate(restricted):
                pq = np.zeros((P.shape[0] + qi, P.shape[1] + qj))
                pq[qi:, qj:] = P
                ints_mono[i, mi] = integrate_triangle(pq)
        C = _orthonormal_coeffs_triangle(qdeg)          # q_r = sum_i C[r, i] s^a_i t^b_i
        for r in range(len(tm)):
            ints = C[r] @ ints_mono
            for w in dirs:
                row = np.zeros(3 * nm)
                for mi in range(nm):
                    for comp in range(3):
                        row[comp * nm + mi] = w[comp] * ints[mi]
                rows.append(row)
    return rows


def _interior_functionals(qdeg: int, nm: int, ms) -> list[np.ndarray]:
    rows = []
    if qdeg < 0:
        return rows
    qs = monomials(3, qdeg)
    C = _orthonormal_coeffs_tet(qdeg)
    mono_int = np.array([[simplex_monomial_integral(tuple(x + y for x, y in zip(m, q))) for m in ms]
                         for q in qs])                    # [n_q, nm]
    for r in range(len(qs)):
        vals = C[r] @ mono_int
        for comp in range(3):
            row = np.zeros(3 * nm)
            row[comp * nm:(comp + 1) * nm] = vals
            rows.append(row)
    return rows


def _homogeneous(deg: int):
    return [m for m in monomials(3, deg) if sum(m) == deg]


@functools.lru_cache(maxsize=None)
def nedelec1(k: int) -> RefElement:
    ms = monomials(3, k)
    nm = len(ms)
    idx = {m: i for i, m in enumerate(ms)}
    span = [_vec(c, idx[m], nm) for c in range(3) for m in monomials(3, k - 1)]
    for m in _homogeneous(k - 1):
        for c in range(3):
            # x cross (m e_c): components (y w_z - z w_y, z w_x - x w_z, x w_y - y w_x)
            w = np.zeros(3)
            w[c] = 1.0
            v = np.zeros(3 * nm)
            shift = lambda axis: tuple(e + (1 if i == axis else 0) for i, e in enumerate(m))
            v[0 * nm + idx[shift(1)]] += w[2]
            v[0 * nm + idx[shift(2)]] -= w[1]
            v[1 * nm + idx[shift(2)]] += w[0]
            v[1 * nm + idx[shift(0)]] -= w[2]
            v[2 * nm + idx[shift(0)]] += w[1]
            v[2 * nm + idx[shift(1)]] -= w[0]
            span.append(v)
    F = np.array(_edge_functionals(k, nm, ms) + _face_functionals("hcurl", k, nm, ms)
                 + _interior_functionals(k - 3, nm, ms))
    phi = _dualise(np.array(span).T, F, k * (k + 2) * (k + 3) // 2)
    return RefElement("hcurl", 3, k, k, phi, 3)


@functools.lru_cache(maxsize=None)
def raviart_thomas(k: int) -> RefElement:
    ms = monomials(3, k)
    nm = len(ms)
    idx = {m: i for i, m in enumerate(ms)}
    span = [_vec(c, idx[m], nm) for c in range(3) for m in monomials(3, k - 1)]
    for m in _homogeneous(k - 1):
        v = np.zeros(3 * nm)
        for c in range(3):
            v[c * nm + idx[tuple(e + (1 if i == c else 0) for i, e in enumerate(m))]] = 1.0
        span.append(v)
    F = np.array(_face_functionals("hdiv", k, nm, ms) + _interior_functionals(k - 2, nm, ms))
    phi = _dualise(np.array(span).T, F, k * (k + 1) * (k + 3) // 2)
    return RefElement("hdiv", 3, k, k, phi, 3)


def reference_element(space: str, dim: int, order: int) -> RefElement:
    if space == "h1":
        return lagrange(dim, order)
    if dim != 3:
        raise ValueError("H(curl)/H(div) elements are built on tetrahedra")
    if space == "hcurl":
        return nedelec1(order)
    if space == "hdiv":
        return raviart_thomas(order)
    raise ValueError(space)


def dof_functionals(space: str, order: int) -> np.ndarray:
    """The functional matrix F of a vector element (rows = dofs), for tests."""
    k = order
    ms = monomials(3, k)
    nm = len(ms)
    if space == "hcurl":
        return np.array(_edge_functionals(k, nm, ms) + _face_functionals("hcurl", k, nm, ms)
                        + _interior_functionals(k - 3, nm, ms))
    return np.array(_face_functionals("hdiv", k, nm, ms) + _interior_functionals(k - 2, nm, ms))
