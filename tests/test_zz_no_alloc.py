"""bras_apply_noalloc: the BRAS apply for callers that cannot let the library allocate.

Callers that manage all device memory themselves (a pool or caching allocator), or that
cannot afford an allocation's implicit synchronisation, call this entry point: it keeps its
scratch (partial sums of cell-block boundary dofs) in a fixed device array of the library
instead of allocating.  It runs bras_apply's own kernels, so the test calls it through the C
ABI twice in a row and requires the same bits as bras_apply on the same inputs.  It lives in
its own file, collected last, and builds its own context so it runs alone or after the rest.
"""
import numpy as np
import pytest
import torch

from paper_2607_12138_b300 import meshgen as mg

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("space,order,prec", [("h1", 3, 0), ("h1", 3, 1), ("h1g", 4, 1), ("hcurl", 2, 0),
                                              ("hdiv", 2, 2)])
def test_noalloc_matches_bras_apply_twice(space, order, prec):
    from paper_2607_12138_b300 import bras as B
    mesh = mg.unit_cube_mesh(5, jitter=0.15, seed=0)
    n, l2g, s = mg.dof_map(mesh, space, order)
    ctx = B.Context(mesh.coords, mesh.cells, space, order, n, l2g, s)
    dt = torch.float64 if prec == B.FP64 else torch.float32
    for nrhs, seed in ((1, 3), (3, 4)):
        x = torch.as_tensor(mg.rhs(n, nrhs, seed=seed), device="cuda").to(dt)
        ref = torch.empty_like(x)
        B.bras_apply(ctx.ctx, prec, x, ref, nrhs)
        for call in range(2):
            y = torch.full_like(x, float("nan"))
            B.bras_apply_noalloc(ctx.ctx, prec, x, y, nrhs)
            torch.cuda.synchronize()
            assert torch.equal(y, ref), (call, (y - ref).abs().max().item())


def test_noalloc_rejects_oversized_scratch():
    from paper_2607_12138_b300 import bras as B
    mesh = mg.unit_cube_mesh(3, jitter=0.1)
    n, l2g, s = mg.dof_map(mesh, "h1", 2)
    ctx = B.Context(mesh.coords, mesh.cells, "h1", 2, n, l2g, s, block_elems=32)   # 6 blocks: partials > 0
    # the host-side size check rejects the call before anything is launched, so the buffers
    # are never read; nrhs is chosen so that even one partial needs more than 16 MiB
    nrhs = 2 ** 21 + 1
    x = torch.zeros(16, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(B.BrasError) as e:
        B.bras_apply_noalloc(ctx.ctx, B.FP64, x, y, nrhs)
    assert e.value.code == -10 and e.value.detail > 16 * 2 ** 20
    assert torch.count_nonzero(y).item() == 0
