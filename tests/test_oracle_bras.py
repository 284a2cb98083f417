"""Pins of the oracle's BRAS operator against the paper's theorems and printed values.

* one element: P = D = I, so M_bras^{-1} = M^{-1} (Eq. mhatinvbras_def);
* SPD and lambda_min(M_bras^{-1} M) >= 1 (Corollary bras_lambda_min);
* Lemma bras_exact_inverse_correction, brute force with an explicit constraint matrix C;
* Theorem bras_lambda_max_projector: lambda_max = lambda_max(M_br Q M_br^{-1} Q);
* lambda_min = 1 when n_br < 2n (RT) and for P1 on a uniform mesh (Sec. 2.3);
* Corollary bras_piola_metric_contrast (metric-contrast bound) for H1 and H(div);
* covariance under global dof sign flips (P' = P S, D' = D);
* kappa_hat of Tables 1-3 at lowest order, and of the Bernstein column of Table 1 at every
  order (tests/golden/paper_tables.json).
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import assembly
from oracle.assembly import Problem
from oracle.solvers import kappa_hat, pencil_eigs
from paper_2607_12138_b300 import meshgen as mg

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))


def _problem(mesh, space, order, rho=None):
    n, l2g, s = mg.dof_map(mesh, space, order)
    return Problem(mesh, space, order, l2g, s, n, rho)


@pytest.mark.parametrize("space,order", [("h1", 2), ("h1", 4), ("hcurl", 2), ("hcurl", 3), ("hcurl", 4), ("hdiv", 3),
                                         ("hdiv", 4), ("n2curl", 3), ("bdm", 3), ("n2curl", 4), ("bdm", 4)])
def test_one_element_is_exact_inverse(space, order):
    pr = _problem(mg.single_simplex_mesh(3, seed=2), space, order)
    np.testing.assert_allclose(pr.B.toarray(), np.linalg.inv(pr.M.toarray()), rtol=1e-10, atol=1e-9 * np.abs(pr.B).max())


@pytest.mark.parametrize("space,order", [("hcurl", 1), ("hcurl", 3), ("hdiv", 2), ("hcurl", 4), ("hdiv", 4),
                                         ("n2curl", 2), ("bdm", 3)])
def test_one_triangle_is_exact_inverse(space, order):
    pr = _problem(mg.single_simplex_mesh(2, seed=2), space, order)
    np.testing.assert_allclose(pr.B.toarray(), np.linalg.inv(pr.M.toarray()), rtol=1e-10, atol=1e-9 * np.abs(pr.B).max())


CASES = [(mg.unit_square_mesh(5, jitter=0.2, seed=4), "h1", 2),
         (mg.unit_cube_mesh(2, jitter=0.15), "h1", 1),
         (mg.relabel_mesh(mg.unit_cube_mesh(2), seed=3), "hcurl", 1),
         (mg.unit_cube_mesh(2), "hcurl", 2),
         (mg.relabel_mesh(mg.unit_cube_mesh(2), seed=5), "hdiv", 1),
         (mg.unit_cube_mesh(2), "hdiv", 2),
         (mg.relabel_mesh(mg.unit_square_mesh(4, jitter=0.2, seed=6), seed=7), "hcurl", 2),
         (mg.relabel_mesh(mg.unit_square_mesh(4, jitter=0.2, seed=8), seed=9), "hdiv", 3),
         (mg.unit_cube_mesh(2, jitter=0.1, seed=10), "hcurl", 4),
         (mg.unit_cube_mesh(2, jitter=0.1, seed=11), "hdiv", 4),
         (mg.relabel_mesh(mg.unit_cube_mesh(2, jitter=0.1), seed=12), "n2curl", 1),
         (mg.unit_cube_mesh(2, jitter=0.1, seed=13), "bdm", 2),
         (mg.relabel_mesh(mg.unit_square_mesh(4, jitter=0.2, seed=14), seed=15), "bdm", 3)]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_spd_and_lambda_min(case):
    mesh, space, order = CASES[case]
    pr = _problem(mesh, space, order)
    B = pr.B.toarray()
    np.testing.assert_allclose(B, B.T, atol=1e-12 * np.abs(B).max())
    assert np.linalg.eigvalsh(B)[0] > 0
    ev = pencil_eigs(pr.M.toarray(), B)
    assert ev[0] >= 1 - 1e-9


def _constraints(l2g, signs, n_dof):
    """Rows s_j1 w_j1 - s_jt w_jt = 0 for every further copy jt of a dof (ker C = range P)."""
    s = np.ones(l2g.size) if signs is None else signs.ravel().astype(float)
    flat = l2g.ravel()
    rows, cols, vals = [], [], []
    r = 0
    for i in range(n_dof):
        copies = np.nonzero(flat == i)[0]
        for j in copies[1:]:
            rows += [r, r]
            cols += [copies[0], j]
            vals += [s[copies[0]], -s[j]]
            r += 1
    return sp.csr_matrix((vals, (rows, cols)), shape=(r, l2g.size)).toarray()


@pytest.mark.parametrize("case", [0, 2, 4])
def test_lemma_exact_inverse_correction(case):
    mesh, space, order = CASES[case]
    pr = _problem(mesh, space, order)
    n, nb = pr.n_dof, pr.l2g.size
    C = _constraints(pr.l2g, pr.signs, n)
    assert C.shape[0] == nb - n and np.linalg.matrix_rank(C) == nb - n
    P = assembly.injection(pr.l2g, pr.signs, n).toarray()
    np.testing.assert_allclose(C @ P, 0, atol=1e-14)
    Mbr_inv = np.zeros((nb, nb))
    nl = pr.l2g.shape[1]
    for k in range(pr.l2g.shape[0]):
        Mbr_inv[k * nl:(k + 1) * nl, k * nl:(k + 1) * nl] = pr.Minv_loc[k]
    Dinv = np.diag(1 / pr.d)
    Z = Dinv @ P.T @ Mbr_inv @ C.T
    S = -C @ Mbr_inv @ C.T
    rhs = np.linalg.inv(pr.M.toarray()) - Z @ np.linalg.solve(S, Z.T)
    B = pr.B.toarray()
    np.testing.assert_allclose(B, rhs, atol=1e-9 * np.abs(B).max())


@pytest.mark.parametrize("case", [0, 1, 3, 5])
def test_theorem_lambda_max_projector(case):
    mesh, space, order = CASES[case]
    pr = _problem(mesh, space, order)
    n, nl = pr.n_dof, pr.l2g.shape[1]
    P = assembly.injection(pr.l2g, pr.signs, n).toarray()
    Q = P @ np.diag(1 / pr.d) @ P.T
    nb = P.shape[0]
    Mbr, Mbr_inv = np.zeros((nb, nb)), np.zeros((nb, nb))
    for k in range(pr.l2g.shape[0]):
        sl = slice(k * nl, (k + 1) * nl)
        Mbr[sl, sl] = pr.Me[k]
        Mbr_inv[sl, sl] = pr.Minv_loc[k]
    np.testing.assert_allclose(P.T @ Mbr @ P, pr.M.toarray(), atol=1e-13)
    lam_thm = np.max(np.linalg.eigvals(Mbr @ Q @ Mbr_inv @ Q).real)
    lam = pencil_eigs(pr.M.toarray(), pr.B.toarray())[-1]
    assert abs(lam_thm - lam) <= 1e-8 * lam


def test_lambda_min_equals_one():
    pr = _problem(mg.unit_cube_mesh(3, jitter=0.15), "hdiv", 1)      # n_br < 2 n
    assert pr.l2g.size < 2 * pr.n_dof
    ev = pencil_eigs(pr.M.toarray(), pr.B.toarray())
    assert abs(ev[0] - 1) < 1e-9
    pr = _problem(mg.unit_cube_mesh(3), "h1", 1)                      # uniform P1: M_br P 1 in range P
    ev = pencil_eigs(pr.M.toarray(), pr.B.toarray())
    assert abs(ev[0] - 1) < 1e-9
    pr = _problem(mg.unit_cube_mesh(3, jitter=0.15), "h1", 1)         # jittered: strictly above 1
    assert pencil_eigs(pr.M.toarray(), pr.B.toarray())[0] > 1 + 1e-6


@pytest.mark.parametrize("space", ["h1", "hdiv"])
def test_metric_contrast_bound(space):
    mesh = mg.unit_cube_mesh(3, jitter=0.2, seed=9)
    n, l2g, s = mg.dof_map(mesh, space, 1)
    pr = Problem(mesh, space, 1, l2g, s, n)
    # identity-metric operator on the same P: every M_K the reference mass (G_K = I)
    ref = assembly.reference_element(space, 3, 1).mass_blocks()
    MeI = np.repeat(np.einsum("aaij->ij", ref)[None], mesh.n_cell, axis=0)
    MI = assembly.assemble_mass(l2g, s, MeI, n).toarray()
    BI = assembly.bras_inverse(l2g, s, MeI, n).toarray()
    G = assembly.metrics(space, assembly.jacobians(mesh.coords, mesh.cells))
    ev = np.linalg.eigvalsh(G)
    ratio = ev.max() / ev.min()
    lam_G = pencil_eigs(pr.M.toarray(), pr.B.toarray())[-1]
    lam_I = pencil_eigs(MI, BI)[-1]
    assert lam_G <= ratio * lam_I * (1 + 1e-12)


@pytest.mark.parametrize("space,order", [("h1", 2), ("hcurl", 1), ("hdiv", 2)])
def test_sign_covariance(space, order):
    mesh = mg.unit_cube_mesh(2, jitter=0.1)
    n, l2g, s = mg.dof_map(mesh, space, order)
    pr = Problem(mesh, space, order, l2g, s, n)
    flip = np.random.default_rng(0).choice([-1, 1], size=n)
    s0 = np.ones(l2g.shape, dtype=np.int8) if s is None else s
    s2 = (s0 * flip[l2g]).astype(np.int8)
    pr2 = Problem(mesh, space, order, l2g, s2, n)
    S = np.diag(flip.astype(float))
    np.testing.assert_allclose(pr2.M.toarray(), S @ pr.M.toarray() @ S, atol=1e-14)
    np.testing.assert_allclose(pr2.B.toarray(), S @ pr.B.toarray() @ S, atol=1e-10)


KAPPA_MESHES = {
    "h1_2d_p1": (lambda: mg.unit_square_mesh(30), "h1", 1),
    "h1_2d_p2": (lambda: mg.unit_square_mesh(16), "h1", 2),
    "h1_3d_p1": (lambda: mg.unit_cube_mesh(10), "h1", 1),
    "h1_3d_p2": (lambda: mg.unit_cube_mesh(6), "h1", 2),
    "hcurl_3d_k1": (lambda: mg.unit_cube_mesh(6), "hcurl", 1),
    "hdiv_3d_k1": (lambda: mg.unit_cube_mesh(5), "hdiv", 1),
    "hcurl_2d_k1": (lambda: mg.unit_square_mesh(24), "hcurl", 1),
    "hdiv_2d_k1": (lambda: mg.unit_square_mesh(24), "hdiv", 1),
    "h1b_2d_p2": (lambda: mg.unit_square_mesh(16), "h1b", 2),
    "h1b_2d_p3": (lambda: mg.unit_square_mesh(12), "h1b", 3),
    "h1b_2d_p4": (lambda: mg.unit_square_mesh(9), "h1b", 4),
    "h1b_3d_p2": (lambda: mg.unit_cube_mesh(6), "h1b", 2),
    "h1b_3d_p3": (lambda: mg.unit_cube_mesh(4), "h1b", 3),
    "h1b_3d_p4": (lambda: mg.unit_cube_mesh(4), "h1b", 4),
    "h1g_2d_p3": (lambda: mg.unit_square_mesh(12), "h1g", 3),
    "h1g_2d_p4": (lambda: mg.unit_square_mesh(9), "h1g", 4),
    "h1g_3d_p3": (lambda: mg.unit_cube_mesh(4), "h1g", 3),
    "h1g_3d_p4": (lambda: mg.unit_cube_mesh(3), "h1g", 4),
    "n2curl_2d_k1": (lambda: mg.unit_square_mesh(24), "n2curl", 1),
    "n2curl_2d_k2": (lambda: mg.unit_square_mesh(16), "n2curl", 2),
    "n2curl_3d_k1": (lambda: mg.unit_cube_mesh(5), "n2curl", 1),
    "n2curl_3d_k2": (lambda: mg.unit_cube_mesh(3), "n2curl", 2),
    "bdm_2d_k1": (lambda: mg.unit_square_mesh(24), "bdm", 1),
    "bdm_2d_k2": (lambda: mg.unit_square_mesh(16), "bdm", 2),
    "bdm_3d_k1": (lambda: mg.unit_cube_mesh(5), "bdm", 1),
    "bdm_3d_k2": (lambda: mg.unit_cube_mesh(3), "bdm", 2),
}


@pytest.mark.parametrize("key", sorted(KAPPA_MESHES))
def test_kappa_hat_matches_paper(key):
    """Uniform unit meshes of 1-2e3 dofs; the printed value has two significant digits, so
    accept half a unit of its last digit plus 2% for the smaller mesh."""
    make, space, order = KAPPA_MESHES[key]
    pr = _problem(make(), space, order)
    M = pr.M.toarray()
    kd = kappa_hat(M, np.diag(1 / pr.diag))
    kb = kappa_hat(M, pr.B.toarray())
    for ours, printed in ((kd, GOLD["kappa_hat"][key]["diag"]), (kb, GOLD["kappa_hat"][key]["bras"])):
        unit = 1.0 if printed >= 10 else 0.1
        assert abs(ours - printed) <= 0.5 * unit + 0.02 * printed, (key, ours, printed)
