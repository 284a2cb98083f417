"""GPU parity: the CUDA path through the C-ABI against the FP64 oracle.

Tolerances (max-abs error / max-abs of the oracle result):
  * FP64 applies: 1e-12 (the FP64 target); both sides round the same exact operator, so
    they differ by about cond(M_K) * 1e-16.
  * FP32 applies: 2e-6 for every family (measured at most 5.7e-7 over every case of the
    suite, max-abs over max-abs: FP32 local matrices and products, ~6e-8 per rounding, over
    up to 105 terms; the in-block dof sums are exact, see the block kernels).
  * bf16-stored inverses: 1e-2 (measured at most 3.2e-3; per entry the median is ~1e-3 and
    the 99th percentile ~3e-2 on small entries: an 8-bit mantissa, 4e-3 per stored entry).
Solves are checked by iteration count (oracle +-1) and by the oracle's own FP64 residual of
the GPU solution (<= the requested 1e-10).
"""
import numpy as np
import pytest
import torch

from oracle import gradient as ograd
from oracle import sampled
from oracle.assembly import Problem, element_matrices
from oracle.solvers import cg_lanczos, chebyshev, fixed_point, pcg, power_lambda_max
from paper_2607_12138_b300 import meshgen as mg

from _cases import SMALL_CASES, build, cube, rel_err

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2607_12138_b300 import bras as B

_PROBLEMS = {}


def _setup(case, **kw):
    key = (case, tuple(sorted(kw.items())))
    if key not in _PROBLEMS:
        mesh, space, order, n, l2g, signs = build(case)
        pr = Problem(mesh, space, order, l2g, signs, n)
        ctx = B.Context(mesh.coords, mesh.cells, space, order, n, l2g, signs, **kw)
        _PROBLEMS[key] = (mesh, pr, ctx)
    return _PROBLEMS[key]


def _vec(n, nrhs=1, seed=5, dtype=torch.float64):
    x = mg.rhs(n, nrhs, seed=seed)
    return x, torch.as_tensor(x, dtype=dtype, device="cuda")


TOL32 = {"h1": 2e-6, "h1b": 2e-6, "h1g": 2e-6, "hcurl": 2e-6, "hdiv": 2e-6, "n2curl": 2e-6, "bdm": 2e-6}
TOL16 = 1e-2   # bf16-stored inverses of H(curl) / H(div)


@pytest.mark.parametrize("case", sorted(SMALL_CASES))
def test_fp64_applies(case):
    mesh, pr, ctx = _setup(case)
    x, xt = _vec(pr.n_dof)
    assert rel_err(ctx.mass_apply(xt).cpu(), pr.M @ x) <= 1e-12
    assert rel_err(ctx.bras_apply(xt).cpu(), pr.B @ x) <= 1e-12
    assert rel_err(ctx.jacobi_apply(xt).cpu(), x / pr.diag) <= 1e-12
    # float-float local products (refinement residual form): same 1e-12 bar
    assert rel_err(ctx.mass_apply(xt, B.FP64X).cpu(), pr.M @ x) <= 1e-12


@pytest.mark.parametrize("case", sorted(SMALL_CASES))
def test_fp32_and_bf16_applies(case):
    mesh, pr, ctx = _setup(case)
    space = SMALL_CASES[case][1]
    x, xt = _vec(pr.n_dof, dtype=torch.float32)
    assert rel_err(ctx.mass_apply(xt, B.FP32).cpu(), pr.M @ x) <= TOL32[space]
    assert rel_err(ctx.bras_apply(xt, B.FP32).cpu(), pr.B @ x) <= TOL32[space]
    assert rel_err(ctx.jacobi_apply(xt, B.FP32).cpu(), x / pr.diag) <= 1e-6
    assert rel_err(ctx.bras_apply(xt, B.BF16).cpu(), pr.B @ x) <= (TOL16 if space not in ("h1", "h1b", "h1g") else TOL32[space])


@pytest.mark.parametrize("case", ["3d_p2", "hcurl2", "hdiv1_signed", "c1_2d_p2", "3d_p3", "3d_p4", "hcurl3", "hdiv3",
                                  "hcurl4", "bdm2", "n2curl3"])
@pytest.mark.parametrize("nrhs", [2, 3, 5, 8])
def test_multi_rhs_interleaved(case, nrhs):
    """[n][R] vectors: chunks of up to 4 right-hand sides per CTA (ragged last chunk for R = 3, 5),
    every precision against the oracle, and each column against the single-RHS apply."""
    mesh, pr, ctx = _setup(case)
    space = SMALL_CASES[case][1]
    x, xt = _vec(pr.n_dof, nrhs)
    yb, ym = ctx.bras_apply(xt), ctx.mass_apply(xt)
    assert rel_err(yb.cpu(), pr.B @ x) <= 1e-12
    assert rel_err(ym.cpu(), pr.M @ x) <= 1e-12
    assert rel_err(ctx.mass_apply(xt, B.FP64X).cpu(), pr.M @ x) <= 1e-12
    assert rel_err(ctx.jacobi_apply(xt).cpu(), x / pr.diag[:, None]) <= 1e-12
    x32 = xt.float()
    yb32, ym32 = ctx.bras_apply(x32, B.FP32), ctx.mass_apply(x32, B.FP32)
    assert rel_err(yb32.cpu(), pr.B @ x) <= TOL32[space]
    assert rel_err(ym32.cpu(), pr.M @ x) <= TOL32[space]
    assert rel_err(ctx.bras_apply(x32, B.BF16).cpu(), pr.B @ x) <= (TOL16 if space not in ("h1", "h1b", "h1g") else TOL32[space])
    for r in (0, nrhs - 1):
        col = xt[:, r].contiguous()
        assert rel_err(yb[:, r].cpu(), ctx.bras_apply(col).cpu()) <= 1e-15
        assert rel_err(ym32[:, r].cpu(), ctx.mass_apply(col.float(), B.FP32).cpu()) <= 1e-6


@pytest.mark.parametrize("case", ["hcurl3", "hdiv3", "hdiv1_signed", "hcurl2d_1_signed", "bdm2", "hcurl2"])
@pytest.mark.parametrize("nrhs", [16, 20, 64])
def test_many_rhs_cell_products(case, nrhs):
    """A context built for many right-hand sides (max_nrhs >= 16, n_loc <= 48) applies the
    streamed cell matrices to 32 right-hand sides per warp and sums each dof's copies in its
    dof-sorted order: every precision against the oracle, every column against the one-RHS
    apply (a different summation order: agreement to rounding), ragged last lane group
    (R = 20), bit-identical repeats, and a mixed solve of all right-hand sides."""
    mesh, pr, ctx = _setup(case, max_nrhs=64)
    space = SMALL_CASES[case][1]
    x, xt = _vec(pr.n_dof, nrhs, seed=7)
    yb, ym = ctx.bras_apply(xt), ctx.mass_apply(xt)
    assert rel_err(yb.cpu(), pr.B @ x) <= 1e-12
    assert rel_err(ym.cpu(), pr.M @ x) <= 1e-12
    assert rel_err(ctx.mass_apply(xt, B.FP64X).cpu(), pr.M @ x) <= 1e-12
    x32 = xt.float()
    yb32, ym32 = ctx.bras_apply(x32, B.FP32), ctx.mass_apply(x32, B.FP32)
    assert rel_err(yb32.cpu(), pr.B @ x) <= TOL32[space]
    assert rel_err(ym32.cpu(), pr.M @ x) <= TOL32[space]
    assert rel_err(ctx.bras_apply(x32, B.BF16).cpu(), pr.B @ x) <= TOL16
    for r in (0, 17 % nrhs, nrhs - 1):
        col = xt[:, r].contiguous()
        assert rel_err(yb[:, r].cpu(), ctx.bras_apply(col).cpu()) <= 1e-14
        # two FP32 paths with different summation orders: each is within TOL32 of the oracle
        assert rel_err(yb32[:, r].cpu(), ctx.bras_apply(col.float(), B.FP32).cpu()) <= 2 * TOL32[space]
    assert torch.equal(ctx.bras_apply(x32, B.FP32), yb32) and torch.equal(ctx.mass_apply(xt), ym)
    xs, its, rel, st = ctx.pcg_solve(xt, pc=B.PC_BRAS, mode=B.SOLVE_MIXED, rtol=1e-10)
    assert st == B.OK
    xg = xs.cpu().numpy()
    for r in (0, nrhs - 1):
        assert np.linalg.norm(x[:, r] - pr.M @ xg[:, r]) <= 1e-10 * np.linalg.norm(x[:, r])


@pytest.mark.parametrize("case", ["3d_p4", "hcurl3"])
def test_bit_reproducible(case):
    mesh, pr, ctx = _setup(case)
    _, xt = _vec(pr.n_dof)
    for prec, dt in ((B.FP64, torch.float64), (B.FP32, torch.float32)):
        a = ctx.bras_apply(xt.to(dt), prec)
        b = ctx.bras_apply(xt.to(dt), prec)
        assert torch.equal(a, b)
        assert torch.equal(ctx.mass_apply(xt.to(dt), prec), ctx.mass_apply(xt.to(dt), prec))


@pytest.mark.parametrize("block_elems", [32, 100])
def test_small_blocks_and_single_cell(block_elems):
    mesh, pr, ctx = _setup("3d_p3", block_elems=block_elems)
    x, xt = _vec(pr.n_dof)
    assert rel_err(ctx.bras_apply(xt).cpu(), pr.B @ x) <= 1e-12
    one = mg.single_simplex_mesh(3, seed=4)
    n, l2g, s = mg.dof_map(one, "hcurl", 3)
    p1 = Problem(one, "hcurl", 3, l2g, s, n)
    c1 = B.Context(one.coords, one.cells, "hcurl", 3, n, l2g, s)
    x = mg.rhs(n, 1, seed=2)
    y = c1.bras_apply(torch.as_tensor(x, device="cuda")).cpu().numpy()
    assert rel_err(y, np.linalg.solve(p1.M.toarray(), x)) <= 1e-12   # one cell: BRAS = M^{-1}


@pytest.mark.parametrize("case,pc", [("c1_2d_p2", 2),
                                     ("c1_2d_p2", 1), ("3d_p2", 2), ("hcurl2", 2), ("hdiv2", 2), ("hcurl1_signed", 1),
                                     ("3d_p3_bern", 2), ("3d_p3_bern", 1), ("hcurl2d_3", 2), ("hdiv2d_2_signed", 1)])
def test_pcg_fp64_iterations_and_residual(case, pc):
    mesh, pr, ctx = _setup(case)
    b, bt = _vec(pr.n_dof, seed=1)
    x, its, rel, st = ctx.pcg_solve(bt, pc=pc, mode=B.SOLVE_FP64, rtol=1e-10)
    assert st == B.OK
    pre = pr.bras_apply if pc == 2 else pr.jacobi_apply
    _, its_o, _ = pcg(pr.mass_apply, b, pre, rtol=1e-10)
    assert abs(int(its[0]) - its_o) <= 1
    xg = x.cpu().numpy()
    assert np.linalg.norm(b - pr.M @ xg) <= 1.05e-10 * np.linalg.norm(b)


def test_pcg_fixed_iterations_match_oracle_iterates():
    mesh, pr, ctx = _setup("3d_p2")
    b, bt = _vec(pr.n_dof, seed=1)
    for K in (1, 5, 10):
        x, its, rel, st = ctx.pcg_solve(bt, pc=B.PC_BRAS, mode=B.SOLVE_FP64, rtol=0.0, maxit=K)
        assert st == B.NOT_CONVERGED and its[0] == K
        xo, _, _ = pcg(pr.mass_apply, b, pr.bras_apply, max_its=K)
        assert rel_err(x.cpu(), xo) <= 1e-12 * K


@pytest.mark.parametrize("case,inner", [("c1_2d_p2", 1), ("3d_p3", 1), ("hcurl3", 1), ("hcurl3", 2), ("hdiv3", 2)])
def test_pcg_mixed_refinement_reaches_fp64_residual(case, inner):
    mesh, pr, ctx = _setup(case)
    b, bt = _vec(pr.n_dof, seed=1)
    x, its, rel, st = ctx.pcg_solve(bt, pc=B.PC_BRAS, mode=B.SOLVE_MIXED, inner_precision=inner, rtol=1e-10)
    assert st == B.OK
    xg = x.cpu().numpy()
    true_rel = np.linalg.norm(b - pr.M @ xg) / np.linalg.norm(b)
    assert true_rel <= 1e-10 and abs(true_rel - rel[0]) <= 1e-3 * 1e-10 + 1e-6 * true_rel


@pytest.mark.parametrize("case", ["3d_p3", "hcurl3"])
def test_mixed_solve_runs_as_one_graph(case):
    """The refinement loop (scales, inner tolerance, stopping test) runs from device scalars:
    one graph launch per mixed solve, bit-identical repeats, a zero column left at zero and
    untouched by the inner loop, and the iteration budget honoured."""
    mesh, pr, ctx = _setup(case)
    b, _ = _vec(pr.n_dof, 3, seed=5)
    b[:, 1] = 0.0
    bt = torch.as_tensor(b, device="cuda")
    g0, k0 = B.graph_launches(), B.kernel_launches()
    x1, its1, rel1, st1 = ctx.pcg_solve(bt, pc=B.PC_BRAS, mode=B.SOLVE_MIXED, rtol=1e-10)
    assert B.graph_launches() - g0 == 1 and B.kernel_launches() - k0 > int(its1.max())
    x2, its2, rel2, st2 = ctx.pcg_solve(bt, pc=B.PC_BRAS, mode=B.SOLVE_MIXED, rtol=1e-10)
    assert st1 == st2 == B.OK
    assert torch.equal(x1, x2) and np.array_equal(its1, its2) and np.array_equal(rel1, rel2)
    xg = x1.cpu().numpy()
    assert its1[1] == 0 and rel1[1] == 0.0 and not np.any(xg[:, 1])
    for r in (0, 2):
        assert np.linalg.norm(b[:, r] - pr.M @ xg[:, r]) <= 1e-10 * np.linalg.norm(b[:, r])
    # budget: at most maxit inner iterations in all (each refinement step charges at least one)
    xb, itsb, relb, stb = ctx.pcg_solve(bt, pc=B.PC_BRAS, mode=B.SOLVE_MIXED, rtol=1e-10, maxit=4)
    assert stb == B.NOT_CONVERGED and int(itsb.max()) <= 4 and relb.max() > 1e-10
    x0, its0, rel0, st0 = ctx.pcg_solve(bt, pc=B.PC_BRAS, mode=B.SOLVE_MIXED, rtol=1e-10, maxit=0)
    assert st0 == B.NOT_CONVERGED and not torch.any(x0) and np.array_equal(rel0, [1.0, 0.0, 1.0])
    z = torch.zeros_like(bt)
    xz, itsz, relz, stz = ctx.pcg_solve(z, pc=B.PC_BRAS, mode=B.SOLVE_MIXED, rtol=1e-10)
    assert stz == B.OK and not torch.any(xz) and not np.any(itsz) and not np.any(relz)


@pytest.mark.parametrize("case,nrhs", [("3d_p2", 4), ("3d_p4", 5), ("hcurl3", 3)])
def test_pcg_multi_rhs_and_host_buffers(case, nrhs):
    mesh, pr, ctx = _setup(case)
    b, bt = _vec(pr.n_dof, nrhs, seed=1)
    x, its, rel, st = ctx.pcg_solve(bt, pc=B.PC_BRAS, rtol=1e-10)
    assert st == B.OK
    for r in range(nrhs):
        _, its_o, _ = pcg(pr.mass_apply, b[:, r], pr.bras_apply, rtol=1e-10)
        assert abs(int(its[r]) - its_o) <= 1
        assert np.linalg.norm(b[:, r] - pr.M @ x.cpu().numpy()[:, r]) <= 1.05e-10 * np.linalg.norm(b[:, r])
    bh = torch.as_tensor(b)                               # host buffers through the same call
    xh, its_h, rel_h, st_h = ctx.pcg_solve(bh, pc=B.PC_BRAS, rtol=1e-10)
    assert st_h == B.OK and xh.device.type == "cpu"
    assert torch.equal(xh, x.cpu()) and np.array_equal(its_h, its)
    xm, its_m, rel_m, st_m = ctx.pcg_solve(bt, pc=B.PC_BRAS, mode=B.SOLVE_MIXED, rtol=1e-10)
    assert st_m == B.OK and rel_m.max() <= 1e-10


def test_gradient_and_weight_update():
    mesh = cube(3, 0.1)
    n, l2g, s = mg.dof_map(mesh, "h1", 3)
    z = np.random.default_rng(2).normal(0, 0.5, mesh.n_cell)
    rho = np.exp(z)
    ctx = B.Context(mesh.coords, mesh.cells, "h1", 3, n, l2g, s, rho=rho)
    x = mg.rhs(n, 1, seed=3)
    lam = mg.rhs(n, 1, seed=4)
    g = ctx.grad_rho(torch.as_tensor(x, device="cuda"), torch.as_tensor(lam, device="cuda")).cpu().numpy()
    Me1 = element_matrices(mesh.coords, mesh.cells, "h1", 3)
    assert rel_err(g, ograd.rho_bar(Me1, l2g, s, x, lam)) <= 1e-12
    rho2 = np.exp(-z)
    ctx.update_rho(rho2)
    pr2 = Problem(mesh, "h1", 3, l2g, s, n, rho2)
    xt = torch.as_tensor(x, device="cuda")
    assert rel_err(ctx.mass_apply(xt).cpu(), pr2.M @ x) <= 1e-12
    assert rel_err(ctx.bras_apply(xt).cpu(), pr2.B @ x) <= 1e-12
    assert rel_err(ctx.jacobi_apply(xt).cpu(), x / pr2.diag) <= 1e-12


def test_log_density_weights_and_gradient():
    """rho = exp(z) set from z on the device, and zbar = rhobar * rho from the fused element
    kernel, against the oracle's weighted operators and adjoint gradient."""
    mesh = cube(3, 0.1)
    n, l2g, s = mg.dof_map(mesh, "h1", 3)
    z = np.random.default_rng(5).normal(0, 0.5, mesh.n_cell)
    ctx = B.Context(mesh.coords, mesh.cells, "h1", 3, n, l2g, s)
    ctx.update_log_rho(torch.as_tensor(z, device="cuda"))
    rho = np.exp(z)
    pr = Problem(mesh, "h1", 3, l2g, s, n, rho)
    x = mg.rhs(n, 1, seed=3)
    lam = mg.rhs(n, 1, seed=4)
    xt, lt = torch.as_tensor(x, device="cuda"), torch.as_tensor(lam, device="cuda")
    assert rel_err(ctx.mass_apply(xt).cpu(), pr.M @ x) <= 1e-12
    assert rel_err(ctx.bras_apply(xt).cpu(), pr.B @ x) <= 1e-12
    Me1 = element_matrices(mesh.coords, mesh.cells, "h1", 3)
    zbar = ctx.grad_log_rho(xt, lt).cpu().numpy()
    assert rel_err(zbar, ograd.rho_bar(Me1, l2g, s, x, lam) * rho) <= 1e-12


def test_error_codes():
    mesh = cube(2)
    n, l2g, s = mg.dof_map(mesh, "h1", 2)
    bad = l2g.copy()
    bad[3, 4] = n
    with pytest.raises(B.BrasError) as e:
        B.Context(mesh.coords, mesh.cells, "h1", 2, n, bad)
    assert e.value.code == -2 and e.value.detail == 3 * 10 + 4
    with pytest.raises(B.BrasError) as e:
        B.Context(mesh.coords, mesh.cells, "h1", 2, n + 1, l2g)
    assert e.value.code == -3 and e.value.detail == n
    flat = mesh.coords.copy()
    flat[mesh.cells[5]] = flat[mesh.cells[5][0]]                  # collapse cell 5
    with pytest.raises(B.BrasError) as e:
        B.Context(flat, mesh.cells, "h1", 2, n, l2g)
    assert e.value.code == -4
    with pytest.raises(B.BrasError) as e:
        B.Context(mesh.coords, mesh.cells, "h1", 2, n, l2g, rho=-np.ones(mesh.n_cell))
    assert e.value.code == -4
    n1, l1, s1 = mg.dof_map(mesh, "hcurl", 1)
    s1 = s1.copy()
    s1[0, 0] = 0
    with pytest.raises(B.BrasError) as e:
        B.Context(mesh.coords, mesh.cells, "hcurl", 1, n1, l1, s1)
    assert e.value.code == -1
    neg = np.ones_like(l2g, dtype=np.int8)
    neg[7, 2] = -1                                                # Lagrange dofs carry no sign
    with pytest.raises(B.BrasError) as e:
        B.Context(mesh.coords, mesh.cells, "h1", 2, n, l2g, neg)
    assert e.value.code == -1 and e.value.detail == 7 * 10 + 2
    ctx = B.Context(mesh.coords, mesh.cells, "hcurl", 1, n1, l1, precisions=1)
    with pytest.raises(B.BrasError) as e:
        ctx.bras_apply(torch.zeros(n1, dtype=torch.float32, device="cuda"), B.FP32)
    assert e.value.code == -9


FULL = {
    "c2_p2": (48, "h1", 2),
    "c2_p4": (48, "h1", 4),
    "c2_p3_gll": (48, "h1g", 3),
    "c2_p4_gll": (48, "h1g", 4),
    "c3_k3": (40, "hcurl", 3),
}


@pytest.mark.parametrize("key", sorted(FULL))
def test_full_size_sampled_parity(key):
    """Full-size meshes in the launch configuration of the benchmark; 200 sampled dofs are
    computed one at a time by the oracle."""
    ncell, space, order = FULL[key]
    mesh = cube(ncell, 0.15, seed=0)
    n, l2g, s = mg.dof_map(mesh, space, order)
    ctx = B.Context(mesh.coords, mesh.cells, space, order, n, l2g, s)
    x = mg.rhs(n, 1, seed=1)
    xt = torch.as_tensor(x, device="cuda")
    dofs = np.random.default_rng(3).choice(n, 200, replace=False)
    yb = ctx.bras_apply(xt).cpu().numpy()[dofs]
    ym = ctx.mass_apply(xt).cpu().numpy()[dofs]
    ob = sampled.bras_apply_at(mesh, space, order, l2g, s, n, x, dofs)
    om = sampled.mass_apply_at(mesh, space, order, l2g, s, n, x, dofs)
    assert rel_err(yb, ob) <= 1e-12 and rel_err(ym, om) <= 1e-12
    y32 = ctx.bras_apply(xt.float(), B.FP32).cpu().numpy()[dofs]
    assert rel_err(y32, ob) <= TOL32[space]
    if space not in ("h1", "h1g"):   # bf16-stored inverses of the streamed spaces
        y16 = ctx.bras_apply(xt.float(), B.BF16).cpu().numpy()[dofs]
        assert rel_err(y16, ob) <= TOL16


def test_full_size_multi_rhs_sampled_parity():
    """32 right-hand sides on the full C2 mesh (H1 p = 4, GLL-based nodes) in the launch
    configuration of the benchmark's 32-RHS rows: 64 sampled dofs of every column against the
    oracle, FP64 and FP32 (multi-RHS tensor-core kernel)."""
    mesh = cube(48, 0.15, seed=0)
    n, l2g, s = mg.dof_map(mesh, "h1g", 4)
    R = 32
    ctx = B.Context(mesh.coords, mesh.cells, "h1g", 4, n, l2g, s, max_nrhs=R)
    X = mg.rhs(n, R, seed=1)
    Xt = torch.as_tensor(X, device="cuda")
    dofs = np.random.default_rng(5).choice(n, 64, replace=False)
    Y64 = ctx.bras_apply(Xt).cpu().numpy()[dofs]
    Y32 = ctx.bras_apply(Xt.float(), B.FP32).cpu().numpy()[dofs]
    M32 = ctx.mass_apply(Xt.float(), B.FP32).cpu().numpy()[dofs]
    for r in range(R):
        ob = sampled.bras_apply_at(mesh, "h1g", 4, l2g, s, n, X[:, r], dofs)
        om = sampled.mass_apply_at(mesh, "h1g", 4, l2g, s, n, X[:, r], dofs)
        assert rel_err(Y64[:, r], ob) <= 1e-12
        assert rel_err(Y32[:, r], ob) <= TOL32["h1g"] and rel_err(M32[:, r], om) <= TOL32["h1g"]


def test_full_size_gradient_sampled_parity():
    """The weighted-solve gradient at the C5 size (32^3 x 6 tets, H1 p = 3, GLL-based nodes,
    rho = exp(z), z ~ N(0, 0.5^2)): rhobar and zbar = rhobar * rho of 300 sampled cells against
    the oracle's element formula on those cells."""
    mesh = cube(32, 0.15, seed=0)
    n, l2g, s = mg.dof_map(mesh, "h1g", 3)
    z = np.random.default_rng(2).normal(0, 0.5, mesh.n_cell)
    ctx = B.Context(mesh.coords, mesh.cells, "h1g", 3, n, l2g, s)
    ctx.update_log_rho(torch.as_tensor(z, device="cuda"))
    x, lam = mg.rhs(n, 1, seed=3), mg.rhs(n, 1, seed=4)
    xt, lt = torch.as_tensor(x, device="cuda"), torch.as_tensor(lam, device="cuda")
    rb = ctx.grad_rho(xt, lt).cpu().numpy()
    zb = ctx.grad_log_rho(xt, lt).cpu().numpy()
    cells = np.random.default_rng(6).choice(mesh.n_cell, 300, replace=False)
    Me1 = element_matrices(mesh.coords, mesh.cells[cells], "h1g", 3)
    orb = ograd.rho_bar(Me1, l2g[cells], None if s is None else s[cells], x, lam)
    assert rel_err(rb[cells], orb) <= 1e-12
    assert rel_err(zb[cells], orb * np.exp(z[cells])) <= 1e-12


def test_autograd_weighted_solve():
    """x = M(exp z)^{-1} b as a torch.autograd.Function: gradients against the oracle's exact
    adjoint gradient and against central differences of the GPU loss (h = 1e-6, FP64)."""
    from paper_2607_12138_b300.autograd import WeightedMassSolver
    mesh = cube(3, 0.1)
    n, l2g, s = mg.dof_map(mesh, "h1", 3)
    rng = np.random.default_rng(2)
    z0 = rng.normal(0, 0.5, mesh.n_cell)
    b0 = mg.rhs(n, 1, seed=1)
    xs0 = mg.rhs(n, 1, seed=3)
    solver = WeightedMassSolver(mesh.coords, mesh.cells, 3, n, l2g, rtol=1e-14)
    z = torch.tensor(z0, device="cuda", requires_grad=True)
    b = torch.tensor(b0, device="cuda", requires_grad=True)
    xs = torch.tensor(xs0, device="cuda")
    x = solver(z, b)
    loss = 0.5 * ((x - xs) ** 2).sum()
    loss.backward()
    L_o, bbar_o, zbar_o, _ = ograd.loss_and_grad(mesh, "h1", 3, l2g, s, n, z0, b0, xs0)
    assert abs(loss.item() - L_o) <= 1e-11 * abs(L_o)
    assert rel_err(z.grad.cpu(), zbar_o) <= 1e-9
    assert rel_err(b.grad.cpu(), bbar_o) <= 1e-9
    h = 1e-6
    with torch.no_grad():
        for trial in range(3):
            v = torch.tensor(rng.standard_normal(mesh.n_cell), device="cuda")
            lp = 0.5 * ((solver(z + h * v, b) - xs) ** 2).sum().item()
            lm = 0.5 * ((solver(z - h * v, b) - xs) ** 2).sum().item()
            fd = (lp - lm) / (2 * h)
            assert abs(fd - (z.grad @ v).item()) <= 1e-6 * max(1.0, abs(fd))


def _batch(space, order, sizes, seed0=10):
    meshes, probs = [], []
    for i, (nx, nz) in enumerate(sizes):
        mesh = mg.unit_cube_mesh(nx, jitter=0.15, seed=seed0 + i, nz=nz)
        n, l2g, s = mg.dof_map(mesh, space, order)
        meshes.append((mesh.coords, mesh.cells, n, l2g, s))
        probs.append(Problem(mesh, space, order, l2g, s, n))
    return meshes, probs


@pytest.mark.parametrize("space,order", [("hdiv", 1), ("hdiv", 2), ("h1", 2), ("n2curl", 1)])
def test_batched_multi_mesh(space, order):
    """Several uneven meshes in one context: applies equal the per-mesh oracle operators and
    one solve reaches each mesh's own tolerance with the oracle's iteration count."""
    sizes = [(2, 1), (4, 3), (3, 5), (1, 1), (5, 2)]
    meshes, probs = _batch(space, order, sizes)
    ctx = B.Context.batched(meshes, space, order)
    off = ctx.offsets
    assert ctx.n_mesh == len(sizes) and off[-1] == sum(p.n_dof for p in probs)
    b = np.concatenate([mg.rhs(p.n_dof, 1, seed=20 + i) for i, p in enumerate(probs)])
    bt = torch.as_tensor(b, device="cuda")
    yb = ctx.bras_apply(bt).cpu().numpy()
    ym = ctx.mass_apply(bt).cpu().numpy()
    for i, p in enumerate(probs):
        seg = slice(off[i], off[i + 1])
        assert rel_err(yb[seg], p.B @ b[seg]) <= 1e-12
        assert rel_err(ym[seg], p.M @ b[seg]) <= 1e-12
    for mode in (B.SOLVE_FP64, B.SOLVE_MIXED):
        x, its, rel, st = ctx.pcg_solve(bt, pc=B.PC_BRAS, mode=mode, rtol=1e-10)
        assert st == B.OK and len(its) == len(sizes)
        xg = x.cpu().numpy()
        for i, p in enumerate(probs):
            seg = slice(off[i], off[i + 1])
            assert np.linalg.norm(b[seg] - p.M @ xg[seg]) <= 1.05e-10 * np.linalg.norm(b[seg])
            if mode == B.SOLVE_FP64:
                _, its_o, _ = pcg(p.mass_apply, b[seg], p.bras_apply, rtol=1e-10)
                assert abs(int(its[i]) - its_o) <= 1


@pytest.mark.parametrize("case", ["2d_p3", "2d_p4", "3d_p3", "3d_p4", "c1_2d_p2", "3d_p4_bern"])
def test_tensor_core_vs_simt_fp32(case):
    """H1 FP32 applies: 3xTF32 tcgen05 local GEMM against the FP32-unit path and the oracle."""
    mesh, space, order, n, l2g, signs = build(case)
    pr = Problem(mesh, space, order, l2g, signs, n)
    tc = B.Context(mesh.coords, mesh.cells, space, order, n, l2g, signs)
    simt = B.Context(mesh.coords, mesh.cells, space, order, n, l2g, signs, simt_only=True)
    x, xt = _vec(n, dtype=torch.float32)
    for op, ref in (("bras_apply", pr.B @ x), ("mass_apply", pr.M @ x)):
        a = getattr(tc, op)(xt, B.FP32).cpu()
        s = getattr(simt, op)(xt, B.FP32).cpu()
        assert rel_err(a, ref) <= TOL32[space] and rel_err(s, ref) <= TOL32[space]
        assert rel_err(a, s) <= 2 * TOL32[space]


@pytest.mark.parametrize("case", ["3d_p3", "3d_p4"])
@pytest.mark.parametrize("block_elems", [64, 128, 160, 256])
def test_tensor_core_block_variants(case, block_elems):
    """The tensor-core kernel's launch variants on 750 tets: blocks of <= 128 cells (two threads
    per cell, one TMEM tile, four CTAs per SM), 160 and 256 (one thread per cell, two tiles);
    one and four (multi-RHS kernel) right-hand sides."""
    mesh, space, order, n, l2g, signs = build(case)
    pr = Problem(mesh, space, order, l2g, signs, n)
    ctx = B.Context(mesh.coords, mesh.cells, space, order, n, l2g, signs, block_elems=block_elems, max_nrhs=4)
    x, xt = _vec(n, dtype=torch.float32)
    for op, ref in (("bras_apply", pr.B @ x), ("mass_apply", pr.M @ x)):
        assert rel_err(getattr(ctx, op)(xt, B.FP32).cpu(), ref) <= TOL32[space]
    x4, xt4 = _vec(n, nrhs=4, seed=9, dtype=torch.float32)
    y4 = ctx.bras_apply(xt4, B.FP32).cpu().numpy().reshape(n, 4)
    assert rel_err(y4, pr.B @ x4.reshape(n, 4)) <= TOL32[space]


@pytest.mark.parametrize("case", ["3d_p2", "hcurl2", "c1_2d_p2", "3d_p4", "hdiv1_signed"])
def test_stationary_iterations(case):
    """Power iteration, damped fixed point and Chebyshev semi-iteration (Sec. 3) against the
    oracle: lambda_max from the same start vector, iteration counts (oracle +-1), the oracle's
    FP64 residual of the GPU solution, and the iterates after a fixed number of steps."""
    mesh, pr, ctx = _setup(case)
    n = pr.n_dof
    v0 = mg.rhs(n, 1, seed=4)
    v0t = torch.as_tensor(v0, device="cuda")
    for pc, P in ((B.PC_JACOBI, pr.jacobi_apply), (B.PC_BRAS, pr.bras_apply)):
        lam = ctx.lambda_max(v0t, pc, iters=40)[0]
        assert abs(lam - power_lambda_max(pr.mass_apply, P, v0, 40)) <= 1e-10 * lam
    lam_b = ctx.lambda_max(v0t, B.PC_BRAS, iters=100)[0]
    omega = 2.0 / (1.0 + lam_b)
    b, bt = _vec(n, 1, seed=1)
    for name, run, ref in (
            ("fixed point", lambda **k: ctx.fixed_point_solve(bt, omega, B.PC_BRAS, **k),
             lambda **k: fixed_point(pr.mass_apply, b, pr.bras_apply, omega, **k)),
            ("chebyshev", lambda **k: ctx.chebyshev_solve(bt, 1.0, lam_b, B.PC_BRAS, **k),
             lambda **k: chebyshev(pr.mass_apply, b, pr.bras_apply, 1.0, lam_b, **k))):
        x, its, rel, st = run(rtol=1e-10)
        _, its_o = ref(rtol=1e-10)
        assert st == B.OK and abs(int(its[0]) - its_o) <= 1, (name, its, its_o)
        assert np.linalg.norm(b - pr.M @ x.cpu().numpy()) <= 1.05e-10 * np.linalg.norm(b), name
        x6, its6, _, st6 = run(rtol=0.0, maxit=6)
        u6, _ = ref(max_its=6)
        assert st6 == B.NOT_CONVERGED and int(its6[0]) == 6
        assert rel_err(x6.cpu().numpy(), u6) <= 1e-12, name
    xh, itsh, _, sth = ctx.chebyshev_solve(bt.cpu(), 1.0, lam_b, B.PC_BRAS)   # host buffers
    assert sth == B.OK and xh.device.type == "cpu"


def test_stationary_multi_rhs_and_batched():
    mesh, pr, ctx = _setup("3d_p2")
    b, bt = _vec(pr.n_dof, 3, seed=1)
    lam = ctx.lambda_max(torch.as_tensor(mg.rhs(pr.n_dof, 3, seed=4), device="cuda"), B.PC_BRAS, iters=60)
    assert lam.shape == (3,)
    x, its, rel, st = ctx.chebyshev_solve(bt, 1.0, lam, B.PC_BRAS)
    assert st == B.OK
    for r in range(3):
        assert np.linalg.norm(b[:, r] - pr.M @ x.cpu().numpy()[:, r]) <= 1.05e-10 * np.linalg.norm(b[:, r])
    sizes = [(2, 1), (4, 3), (3, 5), (1, 1)]
    meshes, probs = _batch("hdiv", 1, sizes)
    bc = B.Context.batched(meshes, "hdiv", 1)
    off = bc.offsets
    v0 = np.concatenate([mg.rhs(p.n_dof, 1, seed=40 + i) for i, p in enumerate(probs)])
    lam = bc.lambda_max(torch.as_tensor(v0, device="cuda"), B.PC_BRAS, iters=50)
    assert lam.shape == (len(sizes),)
    for i, p in enumerate(probs):
        seg = slice(off[i], off[i + 1])
        assert abs(lam[i] - power_lambda_max(p.mass_apply, p.bras_apply, v0[seg], 50)) <= 1e-10 * lam[i]
    bb = np.concatenate([mg.rhs(p.n_dof, 1, seed=20 + i) for i, p in enumerate(probs)])
    x, its, rel, st = bc.fixed_point_solve(torch.as_tensor(bb, device="cuda"), 2.0 / (1.0 + lam), B.PC_BRAS)
    assert st == B.OK and len(its) == len(sizes)
    xg = x.cpu().numpy()
    for i, p in enumerate(probs):
        seg = slice(off[i], off[i + 1])
        _, its_o = fixed_point(p.mass_apply, bb[seg], p.bras_apply, 2.0 / (1.0 + lam[i]))
        assert abs(int(its[i]) - its_o) <= 1
        assert np.linalg.norm(bb[seg] - p.M @ xg[seg]) <= 1.05e-10 * np.linalg.norm(bb[seg])


@pytest.mark.parametrize("case", ["3d_p3", "hcurl2", "c1_2d_p2"])
def test_autotuned_block_size(case):
    """A setup that times the admissible cell-block sizes keeps one of them, and the context
    it leaves behind (re-installed tables, diag(M) recomputed) matches the oracle like any other."""
    mesh, space, order, n, l2g, signs = build(case)
    pr = Problem(mesh, space, order, l2g, signs, n)
    ctx = B.Context(mesh.coords, mesh.cells, space, order, n, l2g, signs, autotune=True)
    be, timed = ctx.block_tuning
    assert len(timed) >= 1 and be in [s for s, _ in timed] and all(us > 0 for _, us in timed)
    x, xt = _vec(n)
    assert rel_err(ctx.bras_apply(xt).cpu(), pr.B @ x) <= 1e-12
    assert rel_err(ctx.mass_apply(xt).cpu(), pr.M @ x) <= 1e-12
    assert rel_err(ctx.jacobi_apply(xt).cpu(), x / pr.diag) <= 1e-12
    assert rel_err(ctx.bras_apply(xt.float(), B.FP32).cpu(), pr.B @ x) <= TOL32[space]
    b, bt = _vec(n, 1, seed=1)
    xs, its, rel, st = ctx.pcg_solve(bt, pc=B.PC_BRAS, rtol=1e-10)
    _, its_o, _ = pcg(pr.mass_apply, b, pr.bras_apply, rtol=1e-10)
    assert st == B.OK and abs(int(its[0]) - its_o) <= 1
    plain = B.Context(mesh.coords, mesh.cells, space, order, n, l2g, signs)
    assert plain.block_tuning[1] == []


@pytest.mark.parametrize("case", ["3d_p2", "hcurl2", "c1_2d_p2", "hdiv2d_2_signed", "3d_p4_bern"])
def test_cg_lanczos_kappa(case):
    """Extreme Ritz values of the CG-Lanczos tridiagonal: the GPU's (FP64 PCG coefficients,
    bisection) against the oracle's (same start vector and step count, dense eigvalsh)."""
    mesh, pr, ctx = _setup(case)
    b, bt = _vec(pr.n_dof, 1, seed=1)
    for pc, P in ((B.PC_BRAS, pr.bras_apply), (B.PC_JACOBI, pr.jacobi_apply)):
        lo, hi, k = ctx.cg_lanczos(bt, pc, steps=15)
        lo_o, hi_o, k_o = cg_lanczos(pr.mass_apply, b, P, 15)
        assert k == k_o == 15
        assert abs(lo - lo_o) <= 1e-8 * lo_o and abs(hi - hi_o) <= 1e-8 * hi_o
    lo, hi, k = ctx.cg_lanczos(bt.cpu(), B.PC_BRAS, steps=400)    # host start vector; early stop
    assert k < 400 and lo >= 1.0 - 1e-9                             # lambda_min >= 1 for BRAS


@pytest.mark.parametrize("case", ["hdiv1_signed", "hdiv2", "hdiv3", "hdiv4", "bdm2", "bdm4"])
def test_schur_complement_apply(case):
    """-S~ x = B M_bras^{-1} B^T x (mixed Poisson, RT_k or BDM_k / DG_{k-1}) against the oracle's
    assembled B and BRAS, in FP64 and FP32; other spaces are rejected."""
    from oracle.schur import divergence_matrix, n_dg, schur_bras
    mesh, pr, ctx = _setup(case)
    space, k = SMALL_CASES[case][1], SMALL_CASES[case][2]
    n, l2g, signs = mg.dof_map(mesh, space, k)
    St = schur_bras(divergence_matrix(mesh, l2g, signs, n, k, space), pr.B)
    x = np.random.default_rng(7).standard_normal(mesh.n_cell * n_dg(k))
    xt = torch.as_tensor(x, device="cuda")
    ref = St @ x
    assert rel_err(ctx.schur_apply(xt).cpu(), ref) <= 1e-12
    assert rel_err(ctx.schur_apply(xt).cpu(), ctx.schur_apply(xt).cpu()) == 0.0
    assert rel_err(ctx.schur_apply(xt.float(), B.FP32).cpu(), ref) <= 1e-4
    _, pr2, c2 = _setup("hcurl2")
    with pytest.raises(B.BrasError) as e:
        c2.schur_apply(torch.zeros(10, dtype=torch.float64, device="cuda"))
    assert e.value.code == -1
