"""Run one apply kernel of the library repeatedly on a fixed case (for profilers).

    python -m paper_2607_12138_b300.profile_case --space h1 --order 4 --cells 48 \
        --op bras --prec fp32 --reps 5

Builds the jittered unit-cube mesh (cells^3 x 6 tetrahedra, jitter 0.15h, seed 0), sets up
one context and launches the chosen apply `reps` times on the current stream.
"""
from __future__ import annotations

import argparse
import time

import torch

from . import bras as B
from . import meshgen as mg


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--space", default="h1", choices=["h1", "h1g", "h1b", "hcurl", "hdiv"])
    ap.add_argument("--order", type=int, default=4)
    ap.add_argument("--cells", type=int, default=48)
    ap.add_argument("--op", default="bras", choices=["bras", "mass", "jacobi"])
    ap.add_argument("--prec", default="fp32", choices=["fp64", "fp32", "bf16", "fp64x"])
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--block-elems", type=int, default=0)
    ap.add_argument("--autotune", action="store_true", help="let setup time the cell block sizes")
    ap.add_argument("--precisions", type=int, default=0,
                    help="bit mask of precisions the context builds (1 << FP64 | 1 << FP32 | 1 << BF16); 0 = all")
    a = ap.parse_args()
    mesh = mg.unit_cube_mesh(a.cells, jitter=0.15, seed=0)
    n, l2g, s = mg.dof_map(mesh, a.space, a.order)
    ctx = B.Context(mesh.coords, mesh.cells, a.space, a.order, n, l2g, s, max_nrhs=a.nrhs,
                    block_elems=a.block_elems, precisions=a.precisions, autotune=a.autotune)
    prec = {"fp64": B.FP64, "fp32": B.FP32, "bf16": B.BF16, "fp64x": B.FP64X}[a.prec]
    dt = torch.float64 if prec in (B.FP64, B.FP64X) else torch.float32
    x = torch.as_tensor(mg.rhs(n, a.nrhs, seed=1), device="cuda").to(dt)
    y = torch.empty_like(x)
    fn = {"bras": ctx.bras_apply, "mass": ctx.mass_apply, "jacobi": ctx.jacobi_apply}[a.op]
    fn(x, prec, out=y)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.reps):
        fn(x, prec, out=y)
    e1.record()
    torch.cuda.synchronize()
    dt_s = e0.elapsed_time(e1) / 1e3 / a.reps
    print(f"{a.space} p={a.order} cells={mesh.n_cell} dofs={n} op={a.op} prec={a.prec} nrhs={a.nrhs} "
          f"blocks={ctx.n_blocks} tuning={ctx.block_tuning} avg_event_us={dt_s * 1e6:.1f} alg_bytes={ctx.algorithmic_bytes(prec, a.nrhs, a.op == 'bras')}")


if __name__ == "__main__":
    main()
