"""BRAS / mass outputs computed one dof at a time, for meshes too large to assemble.

y_i = (1/d_i) sum_{(K,a): l2g[K,a] = i} s_{K,a} (M_K^{-1} xt_K)_a,
xt_K[b] = s_{K,b} x[l2g[K,b]] / d_{l2g[K,b]}       (Eq. mhatinvbras_def, element-sum form)
and (M x)_i = sum_{(K,a)} s_{K,a} (M_K x_K)_a       (Eq. M_PMbrP).
Only the element matrices of the cells touching the sampled dofs are formed.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .assembly import element_matrices, signed_values


def _touching(l2g: np.ndarray, dofs: np.ndarray):
    hit = np.isin(l2g, dofs)
    cells = np.nonzero(hit.any(axis=1))[0]
    return cells


def _apply_at(mesh, space, order, l2g, signs, n_dof, x, dofs, rho, inverse: bool):
    dofs = np.asarray(dofs)
    cells = _touching(l2g, dofs)
    sub = type(mesh)(mesh.coords, mesh.cells[cells], mesh.dim)
    r = None if rho is None else np.asarray(rho)[cells]
    Me = element_matrices(sub.coords, sub.cells, space, order, r)
    s = signed_values(l2g[cells], None if signs is None else signs[cells])
    g = l2g[cells]
    x = np.asarray(x, dtype=np.float64)
    if inverse:
        d = np.bincount(l2g.ravel(), minlength=n_dof).astype(np.float64)
        xt = s * x[g] / d[g]
        z = np.stack([sla.cho_solve(sla.cho_factor(Me[k], lower=True), xt[k]) for k in range(len(cells))])
    else:
        z = np.einsum("kab,kb->ka", Me, s * x[g])
    contrib = s * z
    out = np.zeros(dofs.size)
    pos = {int(v): i for i, v in enumerate(dofs)}
    for k in range(len(cells)):
        for a in range(g.shape[1]):
            i = pos.get(int(g[k, a]))
            if i is not None:
                out[i] += contrib[k, a]
    if inverse:
        out /= d[dofs]
    return out


def bras_apply_at(mesh, space, order, l2g, signs, n_dof, x, dofs, rho=None):
    return _apply_at(mesh, space, order, l2g, signs, n_dof, x, dofs, rho, True)


def mass_apply_at(mesh, space, order, l2g, signs, n_dof, x, dofs, rho=None):
    return _apply_at(mesh, space, order, l2g, signs, n_dof, x, dofs, rho, False)
