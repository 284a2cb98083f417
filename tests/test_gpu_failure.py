"""Failure detection on the GPU without a fault: every mbarrier wait of the library's kernels
is bounded (0.5 s of the global timer), records a bit in a status word and returns.  The
self-test makes one wait run out on a barrier that nothing completes; the host reads the bit,
the CUDA context stays usable, and a context's status word reads clear after normal work."""
import numpy as np
import pytest
import torch

from oracle.assembly import Problem

from _cases import build, rel_err

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2607_12138_b300 import bras as B


def test_bounded_wait_runs_out_and_reports():
    bits, ms = B.bras_wait_selftest()
    assert bits == 1
    assert 300.0 <= ms <= 30000.0
    # the context survives: an apply after the timed-out wait is still correct, and its own
    # status word is clear
    mesh, space, order, n, l2g, signs = build("3d_p3")
    pr = Problem(mesh, space, order, l2g, signs, n)
    ctx = B.Context(mesh.coords, mesh.cells, space, order, n, l2g, signs, block_elems=64)
    x = np.random.default_rng(3).standard_normal(n)
    y = ctx.bras_apply(torch.as_tensor(x, device="cuda"))
    assert rel_err(y.cpu(), pr.B @ x) <= 1e-12
    assert ctx.device_status() == (B.OK, 0)
