"""Pins of the oracle's reference elements against closed forms and conformity.

* P1 element mass = |K| (1 + delta_ij) / ((d+1)(d+2))  (closed form).
* Lagrange partition of unity and polynomial reproduction (definition of the nodal basis).
* N1curl_1 = Whitney edge forms, RT_1 = Whitney face forms: element mass matrices from
  the closed form int_K lambda_i lambda_j = |K| (1 + delta_ij) / 20, on a random tetrahedron
  (this also pins the covariant / contravariant Piola metrics, Eq. piola_mass_pullbacks).
* Bernstein: reference mass = (p!)^2 (alpha + beta)! / (alpha! beta! (2p + d)!) (the integral
  of a barycentric monomial over the simplex), partition of unity sum_alpha B_alpha = 1, and
  B_alpha = p!/alpha! lambda^alpha at random points.
* 2D N1curl / RT: on two triangles sharing an edge the tangential / normal trace agrees, and
  RT_k on triangles is N1curl_k rotated by (v_y, -v_x) (interior pairs swapped with a sign).
* Conformity: on two tetrahedra sharing a face, a random global coefficient vector gives
  a field whose value (H1), tangential part (H(curl)) or normal part (H(div)) agrees from
  both sides of the shared face -- this pins the dof functionals, the signs and the
  generator's dof numbering together.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import assembly, elements
from oracle.polynomials import monomials, eval_monomials
from paper_2607_12138_b300 import meshgen as mg


def _rand_tet(seed):
    return mg.single_simplex_mesh(3, seed=seed, jitter=0.25)


@pytest.mark.parametrize("dim", [2, 3])
def test_p1_closed_form(dim):
    mesh = mg.single_simplex_mesh(dim, seed=3)
    Me = assembly.element_matrices(mesh.coords, mesh.cells, "h1", 1)[0]
    J = assembly.jacobians(mesh.coords, mesh.cells)[0]
    vol = abs(np.linalg.det(J)) / math.factorial(dim)
    ref = vol / ((dim + 1) * (dim + 2)) * (np.ones((dim + 1, dim + 1)) + np.eye(dim + 1))
    np.testing.assert_allclose(Me, ref, rtol=1e-13, atol=0)


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (2, 3), (2, 4), (3, 1), (3, 2), (3, 3), (3, 4)])
def test_lagrange_partition_of_unity_and_reproduction(dim, p):
    e = elements.lagrange(dim, p)
    rng = np.random.default_rng(0)
    pts = rng.dirichlet(np.ones(dim + 1), size=50)[:, 1:]
    vals = e.evaluate(pts)[:, :, 0]
    np.testing.assert_allclose(vals.sum(axis=1), 1.0, atol=1e-12)
    # a random polynomial of degree p equals its interpolant
    coef = rng.standard_normal(len(monomials(dim, p)))
    nodes = sorted(a for a in itertools.product(range(p + 1), repeat=dim + 1) if sum(a) == p)
    V = np.vstack([np.zeros(dim), np.eye(dim)])
    npts = np.array([np.asarray(a, float) @ V / p for a in nodes])
    f_nodes = eval_monomials(dim, p, npts) @ coef
    f_pts = eval_monomials(dim, p, pts) @ coef
    np.testing.assert_allclose(vals @ f_nodes, f_pts, atol=1e-11)
    # integral of 1 = |K_ref| = 1/d!
    assert abs(e.mass_blocks()[0, 0].sum() - 1 / math.factorial(dim)) < 1e-12


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_gll_points_are_legendre_derivative_roots(n):
    """The 1D family of the GLL-based nodes: end points and the roots of P_n' (numpy's Legendre
    routines, mapped to [0, 1])."""
    from numpy.polynomial import legendre as L
    c = np.zeros(n + 1)
    c[n] = 1
    inner = np.sort(np.real(L.legroots(L.legder(c))))
    expect = np.concatenate([[0.0], (inner + 1) / 2, [1.0]])
    got = np.array([float(v) for v in elements.gll_points_01(n)])
    np.testing.assert_allclose(got, expect, atol=1e-14)


@pytest.mark.parametrize("dim,p", [(1, 3), (1, 4), (2, 3), (2, 4), (3, 3), (3, 4)])
def test_recursive_gll_nodes_restrict_to_facets(dim, p):
    """A node with a zero barycentric index is the lower-dimensional node of its facet (the
    property that makes the basis conforming); on an edge it is the GLL point; nodes permute
    with their multi-indices."""
    x = [float(v) for v in elements.gll_points_01(p)]
    for a in itertools.product(range(p + 1), repeat=dim + 1):
        if sum(a) != p:
            continue
        b = np.array([float(v) for v in elements._recursive_node(a)])
        assert abs(b.sum() - 1) < 1e-14 and np.all(b >= -1e-15)
        for i in range(dim + 1):
            if a[i] == 0 and dim > 1:
                sub = np.array([float(v) for v in elements._recursive_node(a[:i] + a[i + 1:])])
                np.testing.assert_allclose(np.delete(b, i), sub, atol=1e-14)
                assert abs(b[i]) < 1e-15
        if dim == 1:
            np.testing.assert_allclose(b, [x[a[0]], x[a[1]]], atol=1e-14)
        for perm in itertools.permutations(range(dim + 1)):
            bp = np.array([float(v) for v in elements._recursive_node(tuple(a[j] for j in perm))])
            np.testing.assert_allclose(bp, b[list(perm)], atol=1e-14)


@pytest.mark.parametrize("dim,p", [(2, 3), (2, 4), (3, 3), (3, 4)])
def test_gll_lagrange_interpolates_at_its_nodes(dim, p):
    """phi_i(node_j) = delta_ij, partition of unity, and exact interpolation of P_p."""
    e = elements.reference_element("h1g", dim, p)
    nodes = sorted(a for a in itertools.product(range(p + 1), repeat=dim + 1) if sum(a) == p)
    V = np.vstack([np.zeros(dim), np.eye(dim)])
    npts = np.array([np.array([float(v) for v in elements._recursive_node(a)]) @ V for a in nodes])
    np.testing.assert_allclose(e.evaluate(npts)[:, :, 0], np.eye(len(nodes)), atol=1e-12)
    rng = np.random.default_rng(3)
    pts = rng.dirichlet(np.ones(dim + 1), size=40)[:, 1:]
    vals = e.evaluate(pts)[:, :, 0]
    np.testing.assert_allclose(vals.sum(axis=1), 1.0, atol=1e-12)
    coef = rng.standard_normal(len(monomials(dim, p)))
    np.testing.assert_allclose(vals @ (eval_monomials(dim, p, npts) @ coef), eval_monomials(dim, p, pts) @ coef,
                               atol=1e-11)
    assert abs(e.mass_blocks()[0, 0].sum() - 1 / math.factorial(dim)) < 1e-12


def _bary_grads(J):
    Jinv = np.linalg.inv(J)
    return np.vstack([-Jinv.sum(axis=0), Jinv])          # row i = grad lambda_i


def _lamlam(vol):
    return vol * (np.ones((4, 4)) + np.eye(4)) / 20.0


def test_whitney_edge_forms():
    mesh = _rand_tet(7)
    J = assembly.jacobians(mesh.coords, mesh.cells)[0]
    vol = abs(np.linalg.det(J)) / 6
    g = _bary_grads(J)
    LL = _lamlam(vol)
    E = elements.EDGES_3D
    W = np.zeros((6, 6))
    for i, (a, b) in enumerate(E):
        for j, (c, d) in enumerate(E):
            W[i, j] = (LL[a, c] * g[b] @ g[d] - LL[a, d] * g[b] @ g[c]
                       - LL[b, c] * g[a] @ g[d] + LL[b, d] * g[a] @ g[c])
    Me = assembly.element_matrices(mesh.coords, mesh.cells, "hcurl", 1)[0]
    np.testing.assert_allclose(Me, W, rtol=1e-12, atol=1e-15)


def test_whitney_face_forms():
    mesh = _rand_tet(11)
    J = assembly.jacobians(mesh.coords, mesh.cells)[0]
    vol = abs(np.linalg.det(J)) / 6
    g = _bary_grads(J)
    LL = _lamlam(vol)
    F = elements.FACES_3D

    def terms(a, b, c):   # w = 2 sum_cyc lambda_a grad b x grad c
        return [(a, 2 * np.cross(g[b], g[c])), (b, 2 * np.cross(g[c], g[a])), (c, 2 * np.cross(g[a], g[b]))]

    W = np.zeros((4, 4))
    for i, f in enumerate(F):
        for j, h in enumerate(F):
            W[i, j] = sum(LL[p, q] * u @ v for p, u in terms(*f) for q, v in terms(*h))
    Me = assembly.element_matrices(mesh.coords, mesh.cells, "hdiv", 1)[0]
    S = np.sign(Me[0] / W[0])
    np.testing.assert_allclose(Me, S[:, None] * W * S[None, :], rtol=1e-12, atol=1e-15)


def _two_tets(seed, sort=True):
    rng = np.random.default_rng(seed)
    coords = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1.0]]) + rng.uniform(-0.15, 0.15, (5, 3))
    cells = np.array([[0, 1, 2, 3], [1, 2, 3, 4]], dtype=np.int32)
    if not sort:
        cells = np.array([[2, 0, 3, 1], [4, 3, 1, 2]], dtype=np.int32)
    return mg.Mesh(coords, cells, 3)


def _field(mesh, space, order, l2g, signs, coef, k, x):
    ref = elements.reference_element(space, 3, order)
    X = mesh.coords[mesh.cells[k]]
    J = (X[1:] - X[0]).T
    xh = np.linalg.solve(J, (x - X[0]).T).T
    s = np.ones(l2g.shape[1]) if signs is None else signs[k].astype(float)
    vals = ref.evaluate(xh)                             # [pts, n_loc, comp]
    loc = s * coef[l2g[k]]
    u = np.einsum("pnc,n->pc", vals, loc)
    if space in ("hcurl", "n2curl"):
        return u @ np.linalg.inv(J)                     # J^{-T} u (row vectors)
    if space in ("hdiv", "bdm"):
        return u @ J.T / np.linalg.det(J)
    return u


@pytest.mark.parametrize("dim,p", [(2, 2), (2, 4), (3, 1), (3, 3), (3, 4)])
def test_bernstein_closed_forms(dim, p):
    ref = elements.reference_element("h1b", dim, p)
    nodes = sorted(a for a in itertools.product(range(p + 1), repeat=dim + 1) if sum(a) == p)
    f = math.factorial
    fac = lambda a: math.prod(f(x) for x in a)
    C = np.array([[f(p) ** 2 * math.prod(f(x + y) for x, y in zip(a, b)) / (fac(a) * fac(b) * f(2 * p + dim))
                   for b in nodes] for a in nodes])
    np.testing.assert_allclose(ref.mass_blocks()[0, 0], C, rtol=1e-14, atol=0)
    rng = np.random.default_rng(dim * 10 + p)
    pts = rng.dirichlet(np.ones(dim + 1), size=12)[:, 1:]          # reference points
    vals = ref.evaluate(pts)[:, :, 0]
    np.testing.assert_allclose(vals.sum(axis=1), 1.0, atol=1e-13)   # partition of unity
    lam = np.concatenate([1 - pts.sum(1, keepdims=True), pts], axis=1)
    expect = np.stack([f(p) / fac(a) * np.prod(lam ** np.array(a), axis=1) for a in nodes], axis=1)
    np.testing.assert_allclose(vals, expect, atol=1e-13)


@pytest.mark.parametrize("space,order,sort", [
    ("h1", 1, False), ("h1", 2, False), ("h1", 3, False), ("h1", 4, False), ("h1b", 3, False), ("h1b", 4, False),
    ("h1g", 3, False), ("h1g", 4, False),
    ("hcurl", 1, False), ("hcurl", 1, True), ("hcurl", 2, True), ("hcurl", 3, True), ("hcurl", 4, True),
    ("hdiv", 1, False), ("hdiv", 1, True), ("hdiv", 2, True), ("hdiv", 3, True), ("hdiv", 4, True),
    ("hcurl", 2, False),
    ("n2curl", 1, False), ("n2curl", 2, True), ("n2curl", 3, True), ("n2curl", 4, True), ("bdm", 1, True),
    ("bdm", 2, True), ("bdm", 3, True), ("bdm", 4, True), ("bdm", 1, False), ("n2curl", 2, False)])
def test_conformity_across_shared_face(space, order, sort):
    # several moments per face need the sorted-vertex convention; the dof map says so
    if (space, order, sort) in (("hcurl", 2, False), ("bdm", 1, False), ("n2curl", 2, False)):
        with pytest.raises(ValueError):
            mg.dof_map(_two_tets(0, sort), space, order)
        return
    mesh = _two_tets(5, sort)
    n, l2g, signs = mg.dof_map(mesh, space, order)
    shared = sorted(set(mesh.cells[0]) & set(mesh.cells[1]))
    V = mesh.coords[shared]
    rng = np.random.default_rng(1)
    bc = rng.dirichlet(np.ones(3), size=20)
    x = bc @ V
    nrm = np.cross(V[1] - V[0], V[2] - V[0])
    nrm /= np.linalg.norm(nrm)
    for trial in range(3):
        coef = rng.standard_normal(n)
        u0 = _field(mesh, space, order, l2g, signs, coef, 0, x)
        u1 = _field(mesh, space, order, l2g, signs, coef, 1, x)
        if space in ("h1", "h1b", "h1g"):
            np.testing.assert_allclose(u0, u1, atol=1e-10)
        elif space in ("hcurl", "n2curl"):
            t0 = u0 - np.outer(u0 @ nrm, nrm)
            t1 = u1 - np.outer(u1 @ nrm, nrm)
            np.testing.assert_allclose(t0, t1, atol=1e-10)
            assert np.abs(u0 - u1).max() > 1e-6        # normal part is free to jump
        else:
            np.testing.assert_allclose(u0 @ nrm, u1 @ nrm, atol=1e-10)


def _two_triangles(seed, sort=True):
    rng = np.random.default_rng(seed)
    coords = np.array([[0, 0], [1, 0], [0, 1], [1, 1.0]]) + rng.uniform(-0.15, 0.15, (4, 2))
    cells = np.array([[0, 1, 2], [1, 2, 3]], dtype=np.int32)
    if not sort:
        cells = np.array([[2, 0, 1], [3, 1, 2]], dtype=np.int32)
    return mg.Mesh(coords, cells, 2)


@pytest.mark.parametrize("space,order", [(s, k) for s in ("hcurl", "hdiv") for k in (1, 2, 3, 4)]
                         + [(s, k) for s in ("n2curl", "bdm") for k in (1, 2, 3, 4)])
@pytest.mark.parametrize("sort", [True, False])
def test_conformity_across_shared_edge_2d(space, order, sort):
    mesh = _two_triangles(3, sort)
    n, l2g, signs = mg.dof_map(mesh, space, order)
    ref = elements.reference_element(space, 2, order)
    shared = sorted(set(mesh.cells[0]) & set(mesh.cells[1]))
    V = mesh.coords[shared]
    t = V[1] - V[0]
    nrm = np.array([t[1], -t[0]]) / np.linalg.norm(t)
    x = V[0] + np.outer(np.random.default_rng(1).uniform(0, 1, 15), t)
    rng = np.random.default_rng(2)
    for _ in range(3):
        coef = rng.standard_normal(n)
        u = []
        for k in range(2):
            X = mesh.coords[mesh.cells[k]]
            J = (X[1:] - X[0]).T
            xh = np.linalg.solve(J, (x - X[0]).T).T
            loc = signs[k].astype(float) * coef[l2g[k]]
            v = np.einsum("pnc,n->pc", ref.evaluate(xh), loc)
            u.append(v @ np.linalg.inv(J) if space in ("hcurl", "n2curl") else v @ J.T / np.linalg.det(J))
        if space in ("hcurl", "n2curl"):
            np.testing.assert_allclose(u[0] @ t, u[1] @ t, atol=1e-10)
            assert np.abs(u[0] - u[1]).max() > 1e-6
        else:
            np.testing.assert_allclose(u[0] @ nrm, u[1] @ nrm, atol=1e-10)


@pytest.mark.parametrize("order", [1, 2, 3, 4])
def test_rt_is_rotated_nedelec_2d(order):
    """With n = R t, R v = (v_y, -v_x), the RT edge moments of R psi equal the N1curl edge moments
    of psi, and the RT interior moments of components (0, 1) are the N1curl ones of (1, -0): so
    the RT basis is R of the N1curl basis, with the interior pairs (q, 0), (q, 1) swapped and the
    second negated."""
    pts = np.random.default_rng(order).dirichlet(np.ones(3), size=10)[:, 1:]
    vc = elements.reference_element("hcurl", 2, order).evaluate(pts)
    vd = elements.reference_element("hdiv", 2, order).evaluate(pts)
    rot = np.stack([vc[:, :, 1], -vc[:, :, 0]], axis=2)           # R applied to every N1curl function
    k = order
    expect = rot.copy()
    for r in range((k - 1) * k // 2):
        i0, i1 = 3 * k + 2 * r, 3 * k + 2 * r + 1
        expect[:, i0], expect[:, i1] = rot[:, i1], -rot[:, i0]
    np.testing.assert_allclose(vd, expect, atol=1e-12)


def _simplex_rule(dim, n=6):
    """Collapsed Gauss-Legendre rule on the reference simplex (exact to degree 2n - 2 - dim)."""
    x, w = np.polynomial.legendre.leggauss(n)
    x, w = (x + 1) / 2, w / 2
    if dim == 2:
        u, v = np.meshgrid(x, x, indexing="ij")
        W = np.outer(w, w) * (1 - u)
        return np.stack([u.ravel(), (v * (1 - u)).ravel()], 1), W.ravel()
    u, v, t = np.meshgrid(x, x, x, indexing="ij")
    W = w[:, None, None] * w[None, :, None] * w[None, None, :] * (1 - u) ** 2 * (1 - v)
    return np.stack([u.ravel(), (v * (1 - u)).ravel(), (t * (1 - u) * (1 - v)).ravel()], 1), W.ravel()


@pytest.mark.parametrize("space", ["n2curl", "bdm", "hcurl", "hdiv"])
@pytest.mark.parametrize("dim", [2, 3])
def test_second_kind_reproduces_full_polynomials(space, dim):
    """N2curl_k and BDM_k contain the whole P_k^d: the L2 projection (M c = int phi . f) of a
    random vector field of degree k = 2 onto the assembled space on a jittered mesh gives f back
    at random points.  The first kinds (N1curl_2, RT_2) contain only part of P_2^d, so the same
    projection misses f by a visible amount."""
    k = 2
    mesh = mg.unit_square_mesh(2, jitter=0.2, seed=3) if dim == 2 else mg.unit_cube_mesh(1, jitter=0.15, seed=3)
    n, l2g, signs = mg.dof_map(mesh, space, k)
    ref = elements.reference_element(space, dim, k)
    rng = np.random.default_rng(4)
    from oracle.polynomials import monomials
    ms = monomials(dim, k)
    coef_f = rng.standard_normal((dim, len(ms)))
    f = lambda x: np.stack([np.prod(x[:, None, :] ** np.array(ms)[None], axis=2) @ coef_f[c] for c in range(dim)], 1)
    qx, qw = _simplex_rule(dim)
    vals = ref.evaluate(qx)                                # [q, n_loc, dim]
    M = np.zeros((n, n))
    b = np.zeros(n)
    maps = []
    for K in range(mesh.n_cell):
        X = mesh.coords[mesh.cells[K]]
        J = (X[1:] - X[0]).T
        dJ = np.linalg.det(J)
        s = np.ones(l2g.shape[1]) if signs is None else signs[K].astype(float)
        phys = vals @ np.linalg.inv(J) if space in ("hcurl", "n2curl") else vals @ J.T / dJ
        phys = phys * s[None, :, None]
        xq = qx @ J.T + X[0]
        w = qw * abs(dJ)
        Mk = np.einsum("q,qic,qjc->ij", w, phys, phys)
        bk = np.einsum("q,qic,qc->i", w, phys, f(xq))
        idx = l2g[K]
        M[np.ix_(idx, idx)] += Mk
        np.add.at(b, idx, bk)
        maps.append((X, J, phys, idx, s))
    c = np.linalg.solve(M, b)
    err = 0.0
    for K, (X, J, _, idx, s) in enumerate(maps):
        xh = rng.dirichlet(np.ones(dim + 1), size=10)[:, 1:]
        v = ref.evaluate(xh)
        phys = v @ np.linalg.inv(J) if space in ("hcurl", "n2curl") else v @ J.T / np.linalg.det(J)
        u = np.einsum("pnc,n->pc", phys, s * c[idx])
        err = max(err, np.abs(u - f(xh @ J.T + X[0])).max())
    scale = np.abs(coef_f).max()
    if space in ("n2curl", "bdm"):
        assert err <= 1e-9 * scale
    else:
        assert err >= 1e-3 * scale
