"""Seeded synthetic inputs: simplicial unit meshes, local-to-global dof maps, signs, RHS.

This module builds only the *inputs* of the mass solve (Sec. 3 workloads: simplicial
unit meshes, a random right-hand side).  It holds none of the method's arithmetic: no
element matrix, no multiplicity, no inverse, no solver.  Both the CUDA path and the
test oracle consume what it returns.

Conventions (shared by every consumer; stated once here):

* Meshes.  2D: unit square, ``nx x ny`` cells, each split along the lower-left ->
  upper-right diagonal.  3D: unit cube, ``n^3`` cells, each split into the 6 Kuhn
  tetrahedra along the main diagonal.  Vertex ids are lexicographic
  (``i + (n+1)*(j + (n+1)*k)``).  Every cell lists its vertices in ascending global id
  (the sorted-vertex convention), so every shared entity is seen with the same vertex
  order from both sides.  Jitter moves interior vertices only, each coordinate by
  ``U(-a*h, a*h)``.
* Local dof order.  H1 Lagrange of order p: one node per multi-index
  ``alpha = (alpha_0..alpha_d)``, ``|alpha| = p``, in ascending lexicographic order of the
  tuple; node position ``sum_i alpha_i v_i / p``.  N1curl_k (3D): edges
  (0,1),(0,2),(0,3),(1,2),(1,3),(2,3) with k dofs each (moment index j = 0..k-1), then
  faces (0,1,2),(0,1,3),(0,2,3),(1,2,3) with k(k-1) dofs each (test polynomial outer,
  tangent m = 1,2 inner), then k(k-1)(k-2)/2 interior dofs (test polynomial outer,
  component inner).  RT_k (3D): faces in the same order with k(k+1)/2 dofs each (test
  polynomial), then interior dofs (test polynomial outer, component inner).  Second kind
  (N2curl_k "n2curl", BDM_k "bdm"): the same entity order with k+1 dofs per edge
  (N2curl; BDM on triangles), (k-1)(k+1) tangential (N2curl) or (k+1)(k+2)/2 normal (BDM)
  dofs per face, then the interior dofs.  The dof functionals themselves are defined where
  the elements are built.
* Signs.  An edge moment j seen with the reversed orientation (local a->b runs from the
  higher to the lower global id) changes by ``(-1)^(j+1)``; a lowest-order face flux
  changes by the parity of the permutation that sorts the face's global ids.  Face
  moments of order >= 2 need the sorted-vertex convention (raises otherwise).
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "Mesh", "unit_square_mesh", "unit_cube_mesh", "single_simplex_mesh", "relabel_mesh",
    "h1_local_nodes", "n_local_dofs", "dof_map", "rhs", "batch_mesh_sizes",
]

# Kuhn split: one tetrahedron per permutation of the axes (walk v000 -> v111).
_KUHN_PERMS = list(itertools.permutations(range(3)))
EDGES_3D = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
FACES_3D = [(0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)]
EDGES_2D = [(0, 1), (0, 2), (1, 2)]


@dataclass
class Mesh:
    coords: np.ndarray   # [n_vert, dim] float64
    cells: np.ndarray    # [n_cell, dim+1] int32
    dim: int

    @property
    def n_vert(self) -> int:
        return int(self.coords.shape[0])

    @property
    def n_cell(self) -> int:
        return int(self.cells.shape[0])


def _jitter(coords: np.ndarray, idx: np.ndarray, n: tuple, amount: float, seed: int) -> np.ndarray:
    if amount == 0.0:
        return coords
    rng = np.random.default_rng(seed)
    h = np.array([1.0 / m for m in n])
    off = rng.uniform(-amount, amount, size=coords.shape) * h
    interior = np.all((idx > 0) & (idx < np.array(n)), axis=1)
    coords = coords.copy()
    coords[interior] += off[interior]
    return coords


def unit_square_mesh(nx: int, ny: int | None = None, jitter: float = 0.0, seed: int = 0) -> Mesh:
    ny = nx if ny is None else ny
    i, j = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="xy")
    idx = np.stack([i.ravel(), j.ravel()], axis=1)          # gid = i + (nx+1) j
    coords = idx / np.array([nx, ny], dtype=np.float64)
    coords = _jitter(coords, idx, (nx, ny), jitter, seed)
    ci, cj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    ci, cj = ci.ravel(), cj.ravel()
    v00 = ci + (nx + 1) * cj
    v10, v01, v11 = v00 + 1, v00 + nx + 1, v00 + nx + 2
    t1 = np.stack([v00, v10, v11], axis=1)
    t2 = np.stack([v00, v01, v11], axis=1)
    cells = np.stack([t1, t2], axis=1).reshape(-1, 3)
    return Mesh(coords, np.sort(cells, axis=1).astype(np.int32), 2)


def unit_cube_mesh(n: int, jitter: float = 0.0, seed: int = 0, ny: int | None = None,
                   nz: int | None = None) -> Mesh:
    nx = n
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    idx = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)   # gid = i + (nx+1)(j + (ny+1)k)
    coords = idx / np.array([nx, ny, nz], dtype=np.float64)
    coords = _jitter(coords, idx, (nx, ny, nz), jitter, seed)
    ck, cj, ci = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    base = (ci + (nx + 1) * (cj + (ny + 1) * ck)).ravel()
    stride = np.array([1, nx + 1, (nx + 1) * (ny + 1)])
    tets = []
    for perm in _KUHN_PERMS:
        v = [base]
        cur = base.copy()
        for ax in perm:
            cur = cur + stride[ax]
            v.append(cur)
        tets.append(np.stack(v, axis=1))
    cells = np.stack(tets, axis=1).reshape(-1, 4)
    return Mesh(coords, np.sort(cells, axis=1).astype(np.int32), 3)


def single_simplex_mesh(dim: int, seed: int = 0, jitter: float = 0.2) -> Mesh:
    """One reference-like simplex with seeded vertex perturbations."""
    rng = np.random.default_rng(seed)
    coords = np.vstack([np.zeros(dim), np.eye(dim)]) + rng.uniform(-jitter, jitter, size=(dim + 1, dim))
    return Mesh(coords, np.arange(dim + 1, dtype=np.int32)[None, :], dim)


def relabel_mesh(mesh: Mesh, seed: int, shuffle_local: bool = True, shuffle_cells: bool = True) -> Mesh:
    """Random vertex relabelling, cell order and local vertex order (unsorted cells)."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(mesh.n_vert)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(mesh.n_vert)
    coords = mesh.coords[perm]                 # new vertex v is old vertex perm[v]
    cells = inv[mesh.cells]
    if shuffle_local:
        cells = np.take_along_axis(cells, np.argsort(rng.random(cells.shape), axis=1), axis=1)
    if shuffle_cells:
        cells = cells[rng.permutation(cells.shape[0])]
    return Mesh(coords, cells.astype(np.int32), mesh.dim)


def h1_local_nodes(dim: int, p: int) -> list[tuple[int, ...]]:
    """Multi-indices of the Lagrange nodes, ascending lexicographic order."""
    return sorted(a for a in itertools.product(range(p + 1), repeat=dim + 1) if sum(a) == p)


def n_local_dofs(space: str, dim: int, order: int) -> int:
    if space in ("h1", "h1b", "h1g"):
        return math.comb(order + dim, dim)
    if space in ("n2curl", "bdm"):                       # the full P_k^dim
        return dim * math.comb(order + dim, dim)
    if dim == 2:
        return order * (order + 2)                       # N1curl_k and RT_k on triangles
    k = order
    if space == "hcurl":
        return k * (k + 2) * (k + 3) // 2
    if space == "hdiv":
        return k * (k + 1) * (k + 3) // 2
    raise ValueError(space)


def _entity_index(keys: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    uniq, inv = np.unique(keys, return_inverse=True)
    return uniq, inv.reshape(keys.shape)


def _h1_dof_map(mesh: Mesh, p: int):
    dim, cells, nv = mesh.dim, mesh.cells.astype(np.int64), mesh.n_vert
    E = cells.shape[0]
    nodes = h1_local_nodes(dim, p)
    # canonical position of a node inside its entity: rank of the positive composition
    comps = {m: sorted(a for a in itertools.product(range(1, p + 1), repeat=m) if sum(a) == p)
             for m in range(1, dim + 2)}
    rank = {m: {a: r for r, a in enumerate(c)} for m, c in comps.items()}
    # entity tables (sorted global vertex tuples)
    ent_keys = {}
    for m in range(2, dim + 2):
        if m == dim + 1:
            continue
        subs = list(itertools.combinations(range(dim + 1), m))
        g = np.sort(cells[:, subs], axis=2)          # [E, nsub, m]
        key = np.zeros(g.shape[:2], dtype=np.int64)
        for c in range(m):
            key = key * nv + g[:, :, c]
        ent_keys[m] = np.unique(key)
    counts = {1: nv, dim + 1: E}
    for m, u in ent_keys.items():
        counts[m] = u.size
    base, acc = {}, 0
    for m in range(1, dim + 2):
        base[m] = acc
        acc += counts[m] * len(comps[m])
    n_dof = acc
    l2g = np.empty((E, len(nodes)), dtype=np.int64)
    for a, alpha in enumerate(nodes):
        sup = [i for i in range(dim + 1) if alpha[i] > 0]
        m = len(sup)
        g = cells[:, sup]
        order = np.argsort(g, axis=1, kind="stable")
        gs = np.take_along_axis(g, order, axis=1)
        beta = np.array([alpha[i] for i in sup])[order]   # alpha values in gid order
        code = np.zeros(E, dtype=np.int64)
        for c in range(m):
            code = code * (p + 1) + beta[:, c]
        table = np.full((p + 1) ** m, -1, dtype=np.int64)
        for comp, rr in rank[m].items():
            cc = 0
            for v in comp:
                cc = cc * (p + 1) + v
            table[cc] = rr
        r = table[code]
        if m == 1:
            ent = gs[:, 0]
        elif m == dim + 1:
            ent = np.arange(E)
        else:
            key = np.zeros(E, dtype=np.int64)
            for c in range(m):
                key = key * nv + gs[:, c]
            ent = np.searchsorted(ent_keys[m], key)
        l2g[:, a] = base[m] + ent * len(comps[m]) + r
    return n_dof, l2g.astype(np.int32), None


def _perm_parity(g: np.ndarray) -> np.ndarray:
    """Parity (+1/-1) of the permutation that sorts each row of g (distinct entries)."""
    s = np.ones(g.shape[0], dtype=np.int64)
    m = g.shape[1]
    for i in range(m):
        for j in range(i + 1, m):
            s *= np.where(g[:, i] < g[:, j], 1, -1)
    return s


def _hcurl_hdiv_dof_map_2d(mesh: Mesh, k: int, second: bool = False):
    """Triangles (N1curl and RT share it): k moments per edge, oriented from the lower to the
    higher global vertex id (moment j flips by (-1)^(j+1) on reversal), then k(k-1) interior
    dofs per cell.  Second kind (N2curl and BDM share it): k+1 moments per edge, then
    (k-1)(k+1) interior dofs."""
    cells, nv = mesh.cells.astype(np.int64), mesh.n_vert
    E = cells.shape[0]
    n_i = (k - 1) * (k + 1) if second else k * (k - 1)
    n_e = k + 1 if second else k
    cols, sgns = [], []
    g = cells[:, EDGES_2D]                               # [E, 3, 2]
    gs = np.sort(g, axis=2)
    uniq, inv = _entity_index(gs[:, :, 0] * nv + gs[:, :, 1])
    rev = g[:, :, 0] > g[:, :, 1]
    for e in range(3):
        for j in range(n_e):
            cols.append(inv[:, e] * n_e + j)
            flip = -1 if (j % 2 == 0) else 1             # (-1)^(j+1)
            sgns.append(np.where(rev[:, e], flip, 1))
    base = uniq.size * n_e
    for j in range(n_i):
        cols.append(base + np.arange(E) * n_i + j)
        sgns.append(np.ones(E, dtype=np.int64))
    base += E * n_i
    l2g = np.stack(cols, axis=1).astype(np.int32)
    signs = np.stack(sgns, axis=1).astype(np.int8)
    return base, l2g, signs


def _hcurl_hdiv_dof_map(mesh: Mesh, space: str, k: int):
    if mesh.dim == 2:
        return _hcurl_hdiv_dof_map_2d(mesh, k, second=space in ("n2curl", "bdm"))
    cells, nv = mesh.cells.astype(np.int64), mesh.n_vert
    E = cells.shape[0]
    if space == "hcurl":
        n_e, n_f, n_i = k, k * (k - 1), k * (k - 1) * (k - 2) // 2
    elif space == "hdiv":
        n_e, n_f, n_i = 0, k * (k + 1) // 2, k * (k - 1) * (k + 1) // 2
    elif space == "n2curl":
        n_e, n_f, n_i = k + 1, (k - 1) * (k + 1), (k - 2) * (k - 1) * (k + 1) // 2
    else:                                                 # bdm
        n_e, n_f, n_i = 0, (k + 1) * (k + 2) // 2, (k - 1) * (k + 1) * (k + 2) // 2
    cols, sgns = [], []
    base = 0
    if n_e:
        g = cells[:, EDGES_3D]                           # [E, 6, 2]
        gs = np.sort(g, axis=2)
        uniq, inv = _entity_index(gs[:, :, 0] * nv + gs[:, :, 1])
        rev = g[:, :, 0] > g[:, :, 1]
        for e in range(6):
            for j in range(n_e):
                cols.append(base + inv[:, e] * n_e + j)
                flip = -1 if (j % 2 == 0) else 1         # (-1)^(j+1)
                sgns.append(np.where(rev[:, e], flip, 1))
        base += uniq.size * n_e
    if n_f:
        g = cells[:, FACES_3D]                           # [E, 4, 3]
        gs = np.sort(g, axis=2)
        uniq, inv = _entity_index((gs[:, :, 0] * nv + gs[:, :, 1]) * nv + gs[:, :, 2])
        for f in range(4):
            par = _perm_parity(g[:, f, :])
            sorted_ok = np.all(g[:, f, :] == gs[:, f, :], axis=1)
            higher = n_f > 1
            if higher and not np.all(sorted_ok):
                raise ValueError("face moments of order >= 2 need cells with sorted vertex ids")
            for j in range(n_f):
                cols.append(base + inv[:, f] * n_f + j)
                sgns.append(par if not higher else np.ones(E, dtype=np.int64))
        base += uniq.size * n_f
    if n_i:
        for j in range(n_i):
            cols.append(base + np.arange(E) * n_i + j)
            sgns.append(np.ones(E, dtype=np.int64))
        base += E * n_i
    l2g = np.stack(cols, axis=1).astype(np.int32)
    signs = np.stack(sgns, axis=1).astype(np.int8)
    return base, l2g, signs


def dof_map(mesh: Mesh, space: str, order: int):
    """Returns (n_dof, l2g [E, n_loc] int32, signs [E, n_loc] int8 or None).  "h1g" (Lagrange
    at GLL-based nodes) and "h1b" (Bernstein) share the Lagrange map: their nodes / B_alpha sit
    on the same multi-index lattice, and the trace on an entity depends only on that entity's
    components of alpha."""
    if space in ("h1", "h1b", "h1g"):
        return _h1_dof_map(mesh, order)
    if space in ("hcurl", "hdiv", "n2curl", "bdm"):
        return _hcurl_hdiv_dof_map(mesh, space, order)
    raise ValueError(space)


def rhs(n: int, nrhs: int = 1, seed: int = 1) -> np.ndarray:
    """N(0,1) right-hand sides, RHS-interleaved layout [n][nrhs] (plain [n] if nrhs == 1)."""
    rng = np.random.default_rng(seed)
    b = rng.standard_normal((n, nrhs))
    return b[:, 0].copy() if nrhs == 1 else b


def batch_mesh_sizes(n_mesh: int, t_min: float = 2e3, t_max: float = 2e5, seed: int = 0):
    """Uneven batch: target tet counts log-uniform in [t_min, t_max]; box sizes (nx, nz)."""
    rng = np.random.default_rng(seed)
    t = np.exp(rng.uniform(math.log(t_min), math.log(t_max), size=n_mesh))
    out = []
    for tt in t:
        nx = max(1, int(round((tt / 6.0) ** (1.0 / 3.0))))
        nz = max(1, int(round(tt / (6.0 * nx * nx))))
        out.append((nx, nz))
    return out
