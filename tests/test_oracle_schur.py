"""Pins of the oracle's mixed Poisson Schur complement (Sec. 4, Sec. 5.1):

* the lowest-order divergence block in closed form: with chi = 1 and the RT_1 flux dofs
  (normal t1 x t2 of each sorted face), int_K div phi_f = +-1, the sign saying whether t1 x t2
  points out of the reference tetrahedron: (-1, +1, -1, +1) for faces 012, 013, 023, 123;
* B annihilates the RT interpolant of a constant field (div of a constant is 0; the pullback
  of c is det J J^{-1} c, and the
  interpolant's face moments are c . (t1 x t2) / 2 for the lowest face polynomial, 0 for the
  others);
* BDM_k / DG_{k-1} (the pair of Sec. 5.1): the L2 projection of a constant field onto BDM_k
  reproduces it (BDM_k holds all of P_k^3), so B annihilates it, and B is onto DG_{k-1} on a
  mesh (div maps BDM_k onto P_{k-1} cell by cell);
* on one cell BRAS = M^{-1}, so -S~ = -S;
* the bound of Sec. 4: if the mass pencil's eigenvalues lie in [a, b] then those of
  S~^{-1} S lie in [1/b, 1/a] (for BRAS, a >= 1, so S~^{-1} S <= 1).
"""
import numpy as np
import pytest

from oracle.assembly import Problem, jacobians
from oracle.elements import FACES_3D
from oracle.schur import divergence_matrix, n_dg, reference_divergence, schur_bras, schur_exact_dense
from oracle.solvers import pencil_eigs
from paper_2607_12138_b300 import meshgen as mg


def _problem(mesh, k, space="hdiv"):
    n, l2g, s = mg.dof_map(mesh, space, k)
    return Problem(mesh, space, k, l2g, s, n), l2g, s, n


def test_lowest_order_divergence_closed_form():
    np.testing.assert_allclose(reference_divergence(1), [[-1.0, 1.0, -1.0, 1.0]], atol=1e-14)
    for k in (2, 3, 4):
        assert reference_divergence(k).shape == (n_dg(k), k * (k + 1) * (k + 3) // 2)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_divergence_annihilates_constant_fields(k):
    mesh = mg.unit_cube_mesh(2, jitter=0.15)
    pr, l2g, s, n = _problem(mesh, k)
    B = divergence_matrix(mesh, l2g, s, n, k)
    J = jacobians(mesh.coords, mesh.cells)
    c = np.array([0.3, -1.1, 0.7])
    nf = k * (k + 1) // 2                                  # face dofs per face
    x = np.zeros(n)
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]])
    for K in range(mesh.n_cell):
        ch = np.linalg.det(J[K]) * np.linalg.solve(J[K], c)           # contravariant pullback of c
        for f, (a, b, cc) in enumerate(FACES_3D):
            nrm = np.cross(V[b] - V[a], V[cc] - V[a])
            g = l2g[K, f * nf]
            x[g] = s[K, f * nf] * (ch @ nrm) / 2.0        # q_0 = 1 on the face (area 1/2)
        # interior moments: component integrals against q_r; only q_0 = 1 survives (volume 1/6)
        if k >= 2:
            ni = k * (k - 1) * (k + 1) // 2
            base = 4 * nf
            for comp in range(3):
                x[l2g[K, base + comp]] = ch[comp] / 6.0
            for r in range(3, ni):
                x[l2g[K, base + r]] = 0.0
    assert np.abs(B @ x).max() <= 1e-12 * np.abs(x).max()
    assert np.abs(B @ np.random.default_rng(0).standard_normal(n)).max() > 1e-3   # not identically zero


@pytest.mark.parametrize("k", [1, 2])
def test_one_cell_schur_is_exact(k):
    mesh = mg.single_simplex_mesh(3, seed=5)
    pr, l2g, s, n = _problem(mesh, k)
    B = divergence_matrix(mesh, l2g, s, n, k)
    np.testing.assert_allclose(schur_bras(B, pr.B).toarray(), schur_exact_dense(B, pr.M), rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("k,cells", [(1, 3), (2, 2), (3, 2)])
def test_schur_spectrum_within_mass_bounds(k, cells):
    mesh = mg.unit_cube_mesh(cells, jitter=0.15, seed=k)
    pr, l2g, s, n = _problem(mesh, k)
    B = divergence_matrix(mesh, l2g, s, n, k)
    mass_ev = pencil_eigs(pr.M.toarray(), pr.B.toarray())
    St = schur_bras(B, pr.B).toarray()
    S = schur_exact_dense(B, pr.M)
    ev = pencil_eigs(St, np.linalg.inv(S))               # eigenvalues of (-S)^{-1}(-S~) = 1 / those of S~^{-1} S
    assert ev[0] >= mass_ev[0] * (1 - 1e-9) and ev[-1] <= mass_ev[-1] * (1 + 1e-9)
    assert ev[0] >= 1 - 1e-9                             # S~^{-1} S <= 1 for BRAS


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_bdm_divergence_kernel_and_range(k):
    mesh = mg.unit_cube_mesh(2, jitter=0.15, seed=k)
    pr, l2g, s, n = _problem(mesh, k, "bdm")
    B = divergence_matrix(mesh, l2g, s, n, k, "bdm")
    assert B.shape == (mesh.n_cell * n_dg(k), n)
    # L2 projection of the constant field c: M x = int phi . c, cell by cell with the reference
    # mass blocks (phi . c is linear in phi, so int_K phi_i . c = c . (pulled-back moments))
    from oracle.elements import reference_element
    from oracle.polynomials import monomials, simplex_monomial_integral
    ref = reference_element("bdm", 3, k)
    ms = monomials(3, k)
    mom = ref.phi.reshape(3, len(ms), ref.n_loc)
    ints = np.array([float(simplex_monomial_integral(m)) for m in ms])
    phi_int = np.einsum("cij,i->jc", mom, ints)            # int_ref phi^_j, [n_loc, 3]
    J = jacobians(mesh.coords, mesh.cells)
    c = np.array([0.4, -1.3, 0.9])
    b = np.zeros(n)
    for K in range(mesh.n_cell):
        # phi = J phi^ / det J, dx = |det J| dx^  ->  int_K phi . c = sign(det J) (J phi^_int) . c
        v = np.sign(np.linalg.det(J[K])) * (phi_int @ J[K].T) @ c
        np.add.at(b, l2g[K], s[K] * v)
    x = np.linalg.solve(pr.M.toarray(), b)
    assert np.abs(B @ x).max() <= 1e-10 * np.abs(x).max()
    assert np.linalg.matrix_rank(B.toarray()) == B.shape[0]


@pytest.mark.parametrize("k", [1, 2])
def test_bdm_one_cell_schur_is_exact(k):
    mesh = mg.single_simplex_mesh(3, seed=6)
    pr, l2g, s, n = _problem(mesh, k, "bdm")
    B = divergence_matrix(mesh, l2g, s, n, k, "bdm")
    np.testing.assert_allclose(schur_bras(B, pr.B).toarray(), schur_exact_dense(B, pr.M), rtol=1e-9, atol=1e-12)


def test_bdm_schur_spectrum_within_mass_bounds():
    mesh = mg.unit_cube_mesh(2, jitter=0.15, seed=9)
    pr, l2g, s, n = _problem(mesh, 2, "bdm")
    B = divergence_matrix(mesh, l2g, s, n, 2, "bdm")
    mass_ev = pencil_eigs(pr.M.toarray(), pr.B.toarray())
    ev = pencil_eigs(schur_bras(B, pr.B).toarray(), np.linalg.inv(schur_exact_dense(B, pr.M)))
    assert ev[0] >= mass_ev[0] * (1 - 1e-9) and ev[-1] <= mass_ev[-1] * (1 + 1e-9)
