"""Shared case builders for the parity tests (inputs from the seeded generator only)."""
from __future__ import annotations

import numpy as np

from paper_2607_12138_b300 import meshgen as mg


def cube(n, jitter=0.15, seed=0):
    return mg.unit_cube_mesh(n, jitter=jitter, seed=seed)


def square(n, jitter=0.2, seed=0):
    return mg.unit_square_mesh(n, jitter=jitter, seed=seed)


# name -> (mesh factory, space, order); sizes span several 256-cell blocks and a ragged tail
SMALL_CASES = {
    "c1_2d_p2": (lambda: square(32), "h1", 2),          # configuration C1 at full size
    "2d_p1": (lambda: square(23), "h1", 1),
    "2d_p3": (lambda: square(17), "h1", 3),
    "2d_p4": (lambda: square(13), "h1", 4),
    "3d_p1": (lambda: cube(6), "h1", 1),
    "3d_p2": (lambda: cube(6), "h1", 2),
    "3d_p3": (lambda: cube(5), "h1", 3),
    "3d_p4": (lambda: cube(5), "h1", 4),
    "hcurl1_signed": (lambda: mg.relabel_mesh(cube(5), seed=7), "hcurl", 1),
    "hcurl2": (lambda: cube(4), "hcurl", 2),
    "hcurl3": (lambda: cube(4), "hcurl", 3),
    "hdiv1_signed": (lambda: mg.relabel_mesh(cube(5), seed=8), "hdiv", 1),
    "hdiv2": (lambda: cube(4), "hdiv", 2),
    "hdiv3": (lambda: cube(4), "hdiv", 3),
    "hcurl2d_1_signed": (lambda: mg.relabel_mesh(square(16), seed=11), "hcurl", 1),   # triangles
    "hdiv2d_2_signed": (lambda: mg.relabel_mesh(square(12), seed=12), "hdiv", 2),
    "hcurl2d_3": (lambda: square(12), "hcurl", 3),
    "hcurl4": (lambda: cube(3), "hcurl", 4),             # order 4: n_loc 84 / 70 / 24
    "hdiv4": (lambda: cube(3), "hdiv", 4),
    "hdiv2d_4_signed": (lambda: mg.relabel_mesh(square(8), seed=13), "hdiv", 4),
    "n2curl1_signed": (lambda: mg.relabel_mesh(cube(4), seed=14), "n2curl", 1),   # second kind: n_loc 12
    "n2curl3": (lambda: cube(3), "n2curl", 3),           # n_loc 60
    "bdm2": (lambda: cube(3), "bdm", 2),                 # n_loc 30
    "n2curl2d_2": (lambda: square(10), "n2curl", 2),     # n_loc 12 (triangles)
    "bdm2d_3_signed": (lambda: mg.relabel_mesh(square(8), seed=15), "bdm", 3),   # n_loc 20
    "bdm4": (lambda: cube(2), "bdm", 4),                 # n_loc 105
    "n2curl4": (lambda: cube(2), "n2curl", 4),
    "n2curl2d_4": (lambda: square(6), "n2curl", 4),      # n_loc 30
    "2d_p4_bern": (lambda: square(13), "h1b", 4),        # Bernstein basis (Table 1)
    "3d_p3_bern": (lambda: cube(5), "h1b", 3),
    "3d_p4_bern": (lambda: cube(5), "h1b", 4),
    "2d_p4_gll": (lambda: square(13), "h1g", 4),         # Lagrange at GLL-based nodes (Table 1)
    "3d_p3_gll": (lambda: cube(5), "h1g", 3),
    "3d_p4_gll": (lambda: cube(5), "h1g", 4),
}


def build(case):
    make, space, order = SMALL_CASES[case]
    mesh = make()
    n, l2g, signs = mg.dof_map(mesh, space, order)
    return mesh, space, order, n, l2g, signs


def rel_err(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
