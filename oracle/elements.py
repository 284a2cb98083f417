"""Reference elements (Sec. 3 element families) built by dualising a monomial span.

Construction, identical for every family:
  1. a spanning set of the polynomial space written in monomial coefficients;
  2. a basis Q of its span (the first linearly independent members, by exact rational
     elimination; the rank must equal the known dimension);
  3. the dof functionals F as row vectors over the coefficients;
  4. nodal basis Phi = Q (F Q)^{-1}, so that F Phi = I.
All of this runs in exact rationals and 40-digit mpmath; the reference mass blocks are
rounded to FP64 once (the FP64 results are then correctly rounded to about 1e-16, which
keeps the oracle's inverses accurate to cond(M_ref) * 1e-16).

Spaces (reference tetrahedron / triangle with vertices 0, e_1, .., e_d):
  * Lagrange P_p: all monomials of degree <= p; dofs = values at the equispaced nodes
    ``sum alpha_i v_i / p`` (multi-indices in ascending lexicographic order).
  * Lagrange P_p at GLL-based nodes (space "h1g", the "spectral" nodal variant of Sec. 3):
    dofs = values at the recursive nodes of Isaac (2020, "Recursive, parameter-free, explicitly
    defined interpolation nodes for simplices") built on the Gauss-Lobatto-Legendre points
    x_{n,0} < .. < x_{n,n} of [0, 1] (0, 1 and the roots of P_n'): in barycentric coordinates
    b(alpha) = sum_i w_i E_i b(alpha without alpha_i) / sum_i w_i with w_i = x_{n, n - alpha_i},
    n = |alpha|, E_i inserting a zero barycentric coordinate at position i, and b((n)) = (1).
    On every edge and face the nodes are the lower-dimensional ones (so the basis is
    conforming with the same dof map), on an edge the GLL points themselves; for p <= 2
    they coincide with the equispaced nodes.
  * Bernstein P_p (space "h1b", the H1 "Bernstein" family of Table 1): not dualised -- the
    basis is the Bernstein polynomials B_alpha = p!/alpha! prod_i lambda_i^alpha_i themselves
    (barycentric lambda_0 = 1 - sum_c x_c, lambda_c = x_c), over the same multi-indices as
    the Lagrange nodes, expanded into monomial coefficients by the multinomial theorem.
  * Nedelec first kind N1curl_k (3D): P_{k-1}^3 + x cross (homogeneous P_{k-1})^3.
  * Raviart-Thomas RT_k (3D): P_{k-1}^3 + x (homogeneous P_{k-1}).
  * On triangles: N1curl_k = P_{k-1}^2 + (-y, x) (homogeneous P_{k-1}) and RT_k =
    P_{k-1}^2 + x (homogeneous P_{k-1}); edge moments of the tangential component (N1curl) or
    of the normal component n = (t_y, -t_x) (RT, t = v_b - v_a) against L_j, j = 0..k-1, then
    interior moments of the two components against polynomials of degree <= k-2 orthonormal
    for the mean inner product on the reference triangle (the face convention below), q outer,
    component inner.  With this normal, RT_k on triangles is N1curl_k rotated by (v_y, -v_x)
    (interior dofs: the pair of components swapped, one negated).
  * Second kind (N2curl_k: space "n2curl", BDM_k: space "bdm", Tables 2-3): the full vector
    polynomial space P_k^d.  Dofs, in this order: edge moments of the tangential (N2curl) or,
    on triangles, normal (BDM) component against L_j, j = 0..k; BDM face moments of the normal
    component against the orthonormal P_k(face); N2curl face moments int_T phi . (J_f psi)
    over the nodal basis psi of RT_{k-1} on the reference triangle (J_f = [t1 t2], the face
    parametrisation below), face outer; interior moments int phi . psi over the nodal basis
    of RT_{k-1} (N2curl, triangles), RT_{k-2} (N2curl, tetrahedra) or N1curl_{k-1} (BDM).
    The lower-order nodal bases are this module's own.
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
import math
import itertools
from dataclasses import dataclass
from fractions import Fraction

import mpmath
import numpy as np

from .polynomials import (gram, integrate_segment, integrate_triangle, monomials,
                          eval_monomials, restrict_to_param, shifted_legendre,
                          simplex_monomial_integral, to_mpf)

EDGES_3D = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
FACES_3D = [(0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)]


def _np(m: mpmath.matrix) -> np.ndarray:
    return np.array([[float(m[i, j]) for j in range(m.cols)] for i in range(m.rows)])


@dataclass(frozen=True)
class RefElement:
    space: str          # "h1", "hcurl", "hdiv"
    dim: int
    order: int
    degree: int         # max polynomial degree of the basis
    phi_mp: mpmath.matrix   # [n_comp * n_mono, n_loc] nodal basis coefficients
    n_comp: int

    @property
    def n_loc(self) -> int:
        return self.phi_mp.cols

    @functools.cached_property
    def phi(self) -> np.ndarray:
        return _np(self.phi_mp)

    def _component_mp(self, c: int) -> mpmath.matrix:
        nm = len(monomials(self.dim, self.degree))
        return self.phi_mp[c * nm:(c + 1) * nm, :]

    def component(self, c: int) -> np.ndarray:
        nm = len(monomials(self.dim, self.degree))
        return self.phi[c * nm:(c + 1) * nm, :]

    @functools.cached_property
    def _mass_blocks(self) -> np.ndarray:
        G = gram(self.dim, self.degree)
        R = np.empty((self.n_comp, self.n_comp, self.n_loc, self.n_loc))
        comps = [self._component_mp(c) for c in range(self.n_comp)]
        for a in range(self.n_comp):
            GA = comps[a].T * G
            for b in range(self.n_comp):
                R[a, b] = _np(GA * comps[b])
        return R

    def mass_blocks(self) -> np.ndarray:
        """R[a, b] = int_ref phi^a phi^b^T  (shape [n_comp, n_comp, n_loc, n_loc])."""
        return self._mass_blocks.copy()

    def evaluate(self, pts: np.ndarray) -> np.ndarray:
        """Reference basis values [n_pts, n_loc, n_comp] at reference points (FP64)."""
        V = eval_monomials(self.dim, self.degree, pts)
        return np.stack([V @ self.component(c) for c in range(self.n_comp)], axis=2)


def _ref_vertices(d: int) -> list[list[int]]:
    return [[0] * d] + [[1 if i == j else 0 for i in range(d)] for j in range(d)]


def _independent_columns(cols: list[list[Fraction]]) -> list[int]:
    """Indices of the first linearly independent columns (exact Gaussian elimination)."""
    basis: list[tuple[int, list[Fraction]]] = []       # (pivot row, reduced vector)
    keep = []
    for j, v in enumerate(cols):
        v = list(v)
        for piv, b in basis:
            if v[piv] != 0:
                f = v[piv] / b[piv]
                v = [x - f * y for x, y in zip(v, b)]
        nz = next((i for i, x in enumerate(v) if x != 0), None)
        if nz is not None:
            basis.append((nz, v))
            keep.append(j)
    return keep


def _dualise(span: list[list[Fraction]], F: mpmath.matrix, dim_expected: int) -> mpmath.matrix:
    keep = _independent_columns(span)
    if len(keep) != dim_expected:
        raise AssertionError(f"span rank {len(keep)} != {dim_expected}")
    n_coef = len(span[0])
    Q = mpmath.matrix(n_coef, len(keep))
    for jj, j in enumerate(keep):
        for i in range(n_coef):
            Q[i, jj] = to_mpf(span[j][i])
    A = F * Q
    if A.rows != A.cols:
        raise AssertionError(f"{A.rows} functionals for a space of dimension {A.cols}")
    return Q * mpmath.inverse(A)


@functools.lru_cache(maxsize=None)
def lagrange(dim: int, p: int) -> RefElement:
    ms = monomials(dim, p)
    nodes = sorted(a for a in itertools.product(range(p + 1), repeat=dim + 1) if sum(a) == p)
    V = _ref_vertices(dim)
    F = mpmath.matrix(len(nodes), len(ms))                  # point evaluations (exact nodes)
    for r, a in enumerate(nodes):
        pt = [Fraction(sum(a[i] * V[i][c] for i in range(dim + 1)), p) for c in range(dim)]
        for j, m in enumerate(ms):
            val = Fraction(1)
            for c in range(dim):
                val *= pt[c] ** m[c]
            F[r, j] = to_mpf(val)
    eye = [[Fraction(int(i == j)) for i in range(len(ms))] for j in range(len(ms))]
    phi = _dualise(eye, F, len(ms))
    return RefElement("h1", dim, p, p, phi, 1)


@functools.lru_cache(maxsize=None)
def gll_points_01(n: int) -> tuple:
    """The n + 1 Gauss-Lobatto-Legendre points of [0, 1], ascending (40 digits): the end
    points and the roots of the derivative of the Legendre polynomial P_n (mapped from
    [-1, 1])."""
    if n == 1:
        return (mpmath.mpf(0), mpmath.mpf(1))
    # Legendre coefficients by (k + 1) P_{k+1} = (2k + 1) x P_k - k P_{k-1}, exact rationals
    P = [[Fraction(1)], [Fraction(0), Fraction(1)]]
    for k in range(1, n):
        nxt = [Fraction(0)] * (k + 2)
        for i, c in enumerate(P[k]):
            nxt[i + 1] += Fraction(2 * k + 1, k + 1) * c
        for i, c in enumerate(P[k - 1]):
            nxt[i] -= Fraction(k, k + 1) * c
        P.append(nxt)
    dP = [i * c for i, c in enumerate(P[n])][1:]           # ascending powers
    with mpmath.workdps(60):
        roots = mpmath.polyroots([to_mpf(c) for c in reversed(dP)], maxsteps=200, extraprec=200)
        inner = sorted(mpmath.re(r) for r in roots)
        pts = [mpmath.mpf(0)] + [(t + 1) / 2 for t in inner] + [mpmath.mpf(1)]
    return tuple(+x for x in pts)


def _recursive_node(alpha: tuple) -> tuple:
    """Barycentric coordinates of the recursive GLL node of multi-index alpha (Isaac 2020)."""
    d = len(alpha) - 1
    n = sum(alpha)
    if d == 0:
        return (mpmath.mpf(1),)
    if n == 0:                      # a degree-0 facet: its weight below is x_{n,0} = 0
        return tuple(mpmath.mpf(1) / (d + 1) for _ in range(d + 1))
    x = gll_points_01(n)
    acc = [mpmath.mpf(0)] * (d + 1)
    wsum = mpmath.mpf(0)
    for i in range(d + 1):
        w = x[n - alpha[i]]
        sub = _recursive_node(alpha[:i] + alpha[i + 1:])
        emb = sub[:i] + (mpmath.mpf(0),) + sub[i:]
        for j in range(d + 1):
            acc[j] += w * emb[j]
        wsum += w
    return tuple(a / wsum for a in acc)


@functools.lru_cache(maxsize=None)
def lagrange_gll(dim: int, p: int) -> RefElement:
    ms = monomials(dim, p)
    nodes = sorted(a for a in itertools.product(range(p + 1), repeat=dim + 1) if sum(a) == p)
    V = _ref_vertices(dim)
    F = mpmath.matrix(len(nodes), len(ms))                  # point evaluations at the GLL nodes
    for r, a in enumerate(nodes):
        lam = _recursive_node(a)
        pt = [sum(lam[i] * V[i][c] for i in range(dim + 1)) for c in range(dim)]
        for j, m in enumerate(ms):
            val = mpmath.mpf(1)
            for c in range(dim):
                val *= pt[c] ** m[c]
            F[r, j] = val
    eye = [[Fraction(int(i == j)) for i in range(len(ms))] for j in range(len(ms))]
    phi = _dualise(eye, F, len(ms))
    return RefElement("h1g", dim, p, p, phi, 1)


@functools.lru_cache(maxsize=None)
def bernstein(dim: int, p: int) -> RefElement:
    ms = monomials(dim, p)
    col = {m: i for i, m in enumerate(ms)}
    nodes = sorted(a for a in itertools.product(range(p + 1), repeat=dim + 1) if sum(a) == p)
    phi = mpmath.matrix(len(ms), len(nodes))
    for j, a in enumerate(nodes):
        lead = Fraction(math.factorial(p), math.prod(math.factorial(x) for x in a))
        # lambda_0^{a_0} = (1 - x_1 - .. - x_d)^{a_0}: multinomial terms with exponents k_1..k_d
        for k in itertools.product(range(a[0] + 1), repeat=dim):
            if sum(k) > a[0]:
                continue
            k0 = a[0] - sum(k)
            c = Fraction(math.factorial(a[0]), math.factorial(k0) * math.prod(math.factorial(x) for x in k))
            c *= (-1) ** sum(k)
            m = tuple(k[i] + a[i + 1] for i in range(dim))
            phi[col[m], j] += to_mpf(lead * c)
    return RefElement("h1", dim, p, p, phi, 1)


def _vec(c: int, j: int, nm: int) -> list[Fraction]:
    v = [Fraction(0)] * (3 * nm)
    v[c * nm + j] = Fraction(1)
    return v


def _edge_functionals(k: int, nm: int, ms) -> list[list]:
    V = _ref_vertices(3)
    rows = []
    for a, b in EDGES_3D:
        tau = [V[b][c] - V[a][c] for c in range(3)]
        restricted = [restrict_to_param(m, V[a], [tau]) for m in ms]
        for j in range(k):
            L = shifted_legendre(j)
            row = [mpmath.mpf(0)] * (3 * nm)
            for mi, P in enumerate(restricted):
                prod = {}
                for (i, _), cf in P.items():
                    for l, cl in enumerate(L):
                        prod[(i + l, 0)] = prod.get((i + l, 0), 0) + cf * cl
                val = to_mpf(integrate_segment(prod))
                for c in range(3):
                    row[c * nm + mi] = tau[c] * val
            rows.append(row)
    return rows


def _orthonormalise(G: mpmath.matrix) -> mpmath.matrix:
    """Rows r of C give q_r = sum_i C[r, i] m_i, orthonormal for the Gram matrix G (Gram-Schmidt
    in the given monomial order, positive leading coefficient): C = L^{-1}, G = L L^T."""
    return mpmath.inverse(mpmath.cholesky(G))


def _face_test_monomials(deg: int) -> list[tuple[int, int]]:
    """s^i t^j with i + j <= deg: degree ascending, then the power of t ascending."""
    return [(d - j, j) for d in range(deg + 1) for j in range(d + 1)]


@functools.lru_cache(maxsize=None)
def _orthonormal_coeffs_triangle(deg: int) -> mpmath.matrix:
    tm = _face_test_monomials(deg)
    G = mpmath.matrix(len(tm), len(tm))
    for i, a in enumerate(tm):
        for j, b in enumerate(tm):
            G[i, j] = to_mpf(integrate_triangle({(a[0] + b[0], a[1] + b[1]): Fraction(1)}) * 2)
    return _orthonormalise(G)            # mean inner product on T (area 1/2)


@functools.lru_cache(maxsize=None)
def _orthonormal_coeffs_tet(deg: int) -> mpmath.matrix:
    return _orthonormalise(gram(3, deg) * 6)   # mean inner product on K (volume 1/6)


def _face_functionals(space: str, k: int, nm: int, ms) -> list[list]:
    V = _ref_vertices(3)
    rows = []
    qdeg = k - 2 if space == "hcurl" else k - 1
    if qdeg < 0:
        return rows
    tm = _face_test_monomials(qdeg)
    C = _orthonormal_coeffs_triangle(qdeg)          # q_r = sum_i C[r, i] s^a_i t^b_i
    for a, b, c in FACES_3D:
        t1 = [V[b][i] - V[a][i] for i in range(3)]
        t2 = [V[c][i] - V[a][i] for i in range(3)]
        if space == "hcurl":
            dirs = [t1, t2]
        else:
            dirs = [[t1[1] * t2[2] - t1[2] * t2[1], t1[2] * t2[0] - t1[0] * t2[2], t1[0] * t2[1] - t1[1] * t2[0]]]
        restricted = [restrict_to_param(m, V[a], [t1, t2]) for m in ms]
        # ints_mono[i][mi] = int_T m_mi(x(s,t)) s^a t^b ds dt for the i-th face monomial
        ints_mono = [[to_mpf(integrate_triangle({(ii + qi, jj + qj): cf for (ii, jj), cf in P.items()}))
                      for P in restricted] for (qi, qj) in tm]
        for r in range(len(tm)):
            ints = [mpmath.fsum(C[r, i] * ints_mono[i][mi] for i in range(len(tm))) for mi in range(nm)]
            for w in dirs:
                row = [mpmath.mpf(0)] * (3 * nm)
                for mi in range(nm):
                    for comp in range(3):
                        row[comp * nm + mi] = w[comp] * ints[mi]
                rows.append(row)
    return rows


def _interior_functionals(qdeg: int, nm: int, ms) -> list[list]:
    rows = []
    if qdeg < 0:
        return rows
    qs = monomials(3, qdeg)
    C = _orthonormal_coeffs_tet(qdeg)
    mono_int = [[to_mpf(simplex_monomial_integral(tuple(x + y for x, y in zip(m, q)))) for m in ms]
                for q in qs]                                  # [n_q][nm]
    for r in range(len(qs)):
        vals = [mpmath.fsum(C[r, i] * mono_int[i][mi] for i in range(len(qs))) for mi in range(nm)]
        for comp in range(3):
            row = [mpmath.mpf(0)] * (3 * nm)
            row[comp * nm:(comp + 1) * nm] = vals
            rows.append(row)
    return rows


def _homogeneous(deg: int):
    return [m for m in monomials(3, deg) if sum(m) == deg]


def _functional_matrix(space: str, k: int) -> mpmath.matrix:
    ms = monomials(3, k)
    nm = len(ms)
    if space == "hcurl":
        rows = (_edge_functionals(k, nm, ms) + _face_functionals("hcurl", k, nm, ms)
                + _interior_functionals(k - 3, nm, ms))
    else:
        rows = _face_functionals("hdiv", k, nm, ms) + _interior_functionals(k - 2, nm, ms)
    return mpmath.matrix(rows)


@functools.lru_cache(maxsize=None)
def nedelec1(k: int) -> RefElement:
    ms = monomials(3, k)
    nm = len(ms)
    idx = {m: i for i, m in enumerate(ms)}
    span = [_vec(c, idx[m], nm) for c in range(3) for m in monomials(3, k - 1)]
    for m in _homogeneous(k - 1):
        for c in range(3):
            # x cross (m e_c): components (y w_z - z w_y, z w_x - x w_z, x w_y - y w_x)
            w = [0, 0, 0]
            w[c] = 1
            v = [Fraction(0)] * (3 * nm)
            shift = lambda axis: tuple(e + (1 if i == axis else 0) for i, e in enumerate(m))
            v[0 * nm + idx[shift(1)]] += w[2]
            v[0 * nm + idx[shift(2)]] -= w[1]
            v[1 * nm + idx[shift(2)]] += w[0]
            v[1 * nm + idx[shift(0)]] -= w[2]
            v[2 * nm + idx[shift(0)]] += w[1]
            v[2 * nm + idx[shift(1)]] -= w[0]
            span.append(v)
    phi = _dualise(span, _functional_matrix("hcurl", k), k * (k + 2) * (k + 3) // 2)
    return RefElement("hcurl", 3, k, k, phi, 3)


@functools.lru_cache(maxsize=None)
def raviart_thomas(k: int) -> RefElement:
    ms = monomials(3, k)
    nm = len(ms)
    idx = {m: i for i, m in enumerate(ms)}
    span = [_vec(c, idx[m], nm) for c in range(3) for m in monomials(3, k - 1)]
    for m in _homogeneous(k - 1):
        v = [Fraction(0)] * (3 * nm)
        for c in range(3):
            v[c * nm + idx[tuple(e + (1 if i == c else 0) for i, e in enumerate(m))]] = Fraction(1)
        span.append(v)
    phi = _dualise(span, _functional_matrix("hdiv", k), k * (k + 1) * (k + 3) // 2)
    return RefElement("hdiv", 3, k, k, phi, 3)


EDGES_2D = [(0, 1), (0, 2), (1, 2)]


def _functional_matrix_2d(space: str, k: int) -> mpmath.matrix:
    ms = monomials(2, k)
    nm = len(ms)
    V = _ref_vertices(2)
    rows = []
    for a, b in EDGES_2D:
        tau = [V[b][c] - V[a][c] for c in range(2)]
        w = tau if space == "hcurl" else [tau[1], -tau[0]]
        restricted = [restrict_to_param(m, V[a], [tau]) for m in ms]
        for j in range(k):
            L = shifted_legendre(j)
            row = [mpmath.mpf(0)] * (2 * nm)
            for mi, P in enumerate(restricted):
                prod = {}
                for (i, _), cf in P.items():
                    for l, cl in enumerate(L):
                        prod[(i + l, 0)] = prod.get((i + l, 0), 0) + cf * cl
                val = to_mpf(integrate_segment(prod))
                for c in range(2):
                    row[c * nm + mi] = w[c] * val
            rows.append(row)
    qdeg = k - 2
    if qdeg >= 0:
        tm = _face_test_monomials(qdeg)                   # (x, y) = (s, t) on the reference triangle
        C = _orthonormal_coeffs_triangle(qdeg)
        mono_int = [[to_mpf(integrate_triangle({(m[0] + qi, m[1] + qj): Fraction(1)})) for m in ms]
                    for (qi, qj) in tm]
        for r in range(len(tm)):
            vals = [mpmath.fsum(C[r, i] * mono_int[i][mi] for i in range(len(tm))) for mi in range(nm)]
            for comp in range(2):
                row = [mpmath.mpf(0)] * (2 * nm)
                row[comp * nm:(comp + 1) * nm] = vals
                rows.append(row)
    return mpmath.matrix(rows)


@functools.lru_cache(maxsize=None)
def vector_2d(space: str, k: int) -> RefElement:
    ms = monomials(2, k)
    nm = len(ms)
    idx = {m: i for i, m in enumerate(ms)}
    span = [[Fraction(int(c * nm + idx[m] == t)) for t in range(2 * nm)]
            for c in range(2) for m in monomials(2, k - 1)]
    for m in (m for m in monomials(2, k - 1) if sum(m) == k - 1):
        v = [Fraction(0)] * (2 * nm)
        if space == "hcurl":            # (-y m, x m)
            v[0 * nm + idx[(m[0], m[1] + 1)]] = Fraction(-1)
            v[1 * nm + idx[(m[0] + 1, m[1])]] = Fraction(1)
        else:                           # (x m, y m)
            v[0 * nm + idx[(m[0] + 1, m[1])]] = Fraction(1)
            v[1 * nm + idx[(m[0], m[1] + 1)]] = Fraction(1)
        span.append(v)
    phi = _dualise(span, _functional_matrix_2d(space, k), k * (k + 2))
    return RefElement(space, 2, k, k, phi, 2)


def _mono_vec_integrals_2d(ms2, psi: RefElement, comp_dirs) -> list[list]:
    """Rows r: the functional int_T v(x) . (sum_c comp_dirs[c] psi_r^c(x)) dx over the reference
    triangle, evaluated on the monomial vectors x^m e_d of ms2 (2 components, coefficient
    layout [d * nm + m])."""
    nm = len(ms2)
    pm = monomials(2, psi.degree)
    rows = []
    for r in range(psi.n_loc):
        row = [mpmath.mpf(0)] * (2 * nm)
        for d in range(2):
            for mi, m in enumerate(ms2):
                acc = mpmath.mpf(0)
                for c in range(2):
                    w = comp_dirs[c][d]
                    if w == 0:
                        continue
                    for qi, q in enumerate(pm):
                        cf = psi.phi_mp[c * len(pm) + qi, r]
                        if cf != 0:
                            acc += w * cf * to_mpf(integrate_triangle({(m[0] + q[0], m[1] + q[1]): Fraction(1)}))
                row[d * nm + mi] = acc
        rows.append(row)
    return rows


def _second_kind_functionals_2d(space: str, k: int) -> mpmath.matrix:
    ms = monomials(2, k)
    nm = len(ms)
    V = _ref_vertices(2)
    rows = []
    for a, b in EDGES_2D:
        tau = [V[b][c] - V[a][c] for c in range(2)]
        w = tau if space == "n2curl" else [tau[1], -tau[0]]
        restricted = [restrict_to_param(m, V[a], [tau]) for m in ms]
        for j in range(k + 1):
            L = shifted_legendre(j)
            row = [mpmath.mpf(0)] * (2 * nm)
            for mi, P in enumerate(restricted):
                prod = {}
                for (i, _), cf in P.items():
                    for l, cl in enumerate(L):
                        prod[(i + l, 0)] = prod.get((i + l, 0), 0) + cf * cl
                val = to_mpf(integrate_segment(prod))
                for c in range(2):
                    row[c * nm + mi] = w[c] * val
            rows.append(row)
    if k >= 2:
        psi = vector_2d("hdiv" if space == "n2curl" else "hcurl", k - 1)
        rows += _mono_vec_integrals_2d(ms, psi, [[1, 0], [0, 1]])
    return mpmath.matrix(rows)


def _interior_against_basis_3d(ms, psi: RefElement) -> list[list]:
    """Rows r: int_K v . psi_r over the reference tetrahedron on the monomial vectors of ms."""
    nm = len(ms)
    pm = monomials(3, psi.degree)
    rows = []
    for r in range(psi.n_loc):
        row = [mpmath.mpf(0)] * (3 * nm)
        for c in range(3):
            for qi, q in enumerate(pm):
                cf = psi.phi_mp[c * len(pm) + qi, r]
                if cf == 0:
                    continue
                for mi, m in enumerate(ms):
                    row[c * nm + mi] += cf * to_mpf(simplex_monomial_integral(tuple(x + y for x, y in zip(m, q))))
        rows.append(row)
    return rows


def _n2curl_face_functionals(k: int, nm: int, ms) -> list[list]:
    """int_T phi(x(s, t)) . (psi_r^s t1 + psi_r^t t2) ds dt, psi the RT_{k-1} triangle basis."""
    V = _ref_vertices(3)
    psi = vector_2d("hdiv", k - 1)
    pm = monomials(2, psi.degree)
    rows = []
    for a, b, c in FACES_3D:
        t1 = [V[b][i] - V[a][i] for i in range(3)]
        t2 = [V[c][i] - V[a][i] for i in range(3)]
        restricted = [restrict_to_param(m, V[a], [t1, t2]) for m in ms]
        for r in range(psi.n_loc):
            # the face field psi_r as a polynomial per Cartesian component
            field = [{} for _ in range(3)]
            for comp, tv in ((0, t1), (1, t2)):
                for qi, q in enumerate(pm):
                    cf = psi.phi_mp[comp * len(pm) + qi, r]
                    if cf == 0:
                        continue
                    for d in range(3):
                        if tv[d] != 0:
                            field[d][q] = field[d].get(q, mpmath.mpf(0)) + cf * tv[d]
            row = [mpmath.mpf(0)] * (3 * nm)
            for mi, P in enumerate(restricted):
                for d in range(3):
                    acc = mpmath.mpf(0)
                    for q, cf in field[d].items():
                        acc += cf * to_mpf(integrate_triangle({(i + q[0], j + q[1]): c0 for (i, j), c0 in P.items()}))
                    row[d * nm + mi] = acc
            rows.append(row)
    return rows


@functools.lru_cache(maxsize=None)
def second_kind(space: str, dim: int, k: int) -> RefElement:
    """N2curl_k ("n2curl") or BDM_k ("bdm"): P_k^dim dualised against the functionals above."""
    ms = monomials(dim, k)
    nm = len(ms)
    span = [[Fraction(int(t == c * nm + j)) for t in range(dim * nm)] for c in range(dim) for j in range(nm)]
    if dim == 2:
        F = _second_kind_functionals_2d(space, k)
    elif space == "n2curl":
        rows = _edge_functionals(k + 1, nm, ms)
        if k >= 2:
            rows += _n2curl_face_functionals(k, nm, ms)
        if k >= 3:
            rows += _interior_against_basis_3d(ms, raviart_thomas(k - 2))
        F = mpmath.matrix(rows)
    else:
        rows = _face_functionals("hdiv", k + 1, nm, ms)
        if k >= 2:
            rows += _interior_against_basis_3d(ms, nedelec1(k - 1))
        F = mpmath.matrix(rows)
    phi = _dualise(span, F, dim * nm)
    return RefElement(space, dim, k, k, phi, dim)


def reference_element(space: str, dim: int, order: int) -> RefElement:
    if space == "h1":
        return lagrange(dim, order)
    if space == "h1b":
        return bernstein(dim, order)
    if space == "h1g":
        return lagrange_gll(dim, order)
    if space in ("n2curl", "bdm"):
        return second_kind(space, dim, order)
    if dim == 2 and space in ("hcurl", "hdiv"):
        return vector_2d(space, order)
    if space == "hcurl":
        return nedelec1(order)
    if space == "hdiv":
        return raviart_thomas(order)
    raise ValueError(space)
