"""Host logic of the library's block tables (csrc/tables.cpp), on the CPU.

``tests/host/tables_dump.cpp`` runs the library's own table builder on a mesh and writes every
table; the tests below read the table packets back and

* check their invariants: the cell order is a permutation, each block's copies are listed
  once, interior dofs have all their copies in the block (and come by ascending id), a group's dofs are exactly the shared dofs with one block set, listed
  contiguously by ascending id in each of its blocks, its partial slots in ascending block
  order, d = the copy counts;
* replay the block apply from the packets alone -- gather with the sign bits and 1/d, local
  products, per-dof sums through the local indices, interior stores, partials, and
  the group sums of the last block -- with the oracle's element matrices, and compare with
  the oracle's assembled M and M_bras^{-1} (Eq. M_PMbrP, Eq. mhatinvbras_def);
* check the error codes of a bad map (an l2g entry out of range, a dof with no copy).
"""
import os
import struct
import subprocess

import numpy as np
import pytest

from oracle.assembly import Problem
from paper_2607_12138_b300 import meshgen as mg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2607_12138_b300", "csrc")


@pytest.fixture(scope="module")
def dump_exe(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("tables") / "tables_dump")
    cmd = ["g++", "-O1", "-std=c++17", "-fopenmp", "-I/usr/local/cuda/include", "-I" + CSRC,
           os.path.join(ROOT, "tests", "host", "tables_dump.cpp"), os.path.join(CSRC, "tables.cpp"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail("g++ failed:\n" + r.stderr)
    return exe


def _pad16(b):
    return (b + 15) & ~15


def build_tables(exe, tmp, mesh, l2g, signs, n, BE, groups=None, scatter=False):
    E, nloc = l2g.shape
    dim = mesh.dim
    inp, out = str(tmp / "in.bin"), str(tmp / "out.bin")
    with open(inp, "wb") as f:
        f.write(struct.pack("<qiqiiqiii", E, nloc, n, dim, BE, mesh.n_vert, signs is not None, groups is not None,
                            scatter))
        f.write(np.ascontiguousarray(l2g, dtype=np.int32).tobytes())
        if signs is not None:
            f.write(np.ascontiguousarray(signs, dtype=np.int8).tobytes())
        f.write(np.ascontiguousarray(mesh.coords, dtype=np.float64).tobytes())
        f.write(np.ascontiguousarray(mesh.cells, dtype=np.int32).tobytes())
        if groups is not None:
            f.write(np.ascontiguousarray(groups, dtype=np.int32).tobytes())
    r = subprocess.run([exe, inp, out], capture_output=True)
    assert r.returncode == 0
    buf = open(out, "rb").read()
    rc, detail = struct.unpack_from("<iq", buf, 0)
    if rc != 0:
        return rc, detail, None
    o = 12
    BE_, nblk, max_u, max_ne, max_bg, max_copies, max_pkt = struct.unpack_from("<iiiiiiI", buf, o)
    o += 28
    npart, U_tot, nsh = struct.unpack_from("<qqq", buf, o)
    o += 24
    t = {"BE": BE_, "nblk": nblk, "max_u": max_u, "max_ne": max_ne, "max_bg": max_bg, "max_copies": max_copies,
         "max_pkt": max_pkt,
         "npart": npart, "U_tot": U_tot, "nsh": nsh}
    for name, dt in (("perm", np.int32), ("blk_e0", np.int32), ("blk_u0", np.int32), ("blk_nint", np.int32),
                     ("blk_p0", np.int32), ("grp_size", np.int32), ("grp_cnt", np.int32), ("grp_slot0", np.int32),
                     ("grp_slots", np.int32), ("blk_g0", np.int32), ("bg_gid", np.int32), ("bg_u", np.int32),
                     ("grp_item0", np.int32), ("sh_ids", np.int32), ("sh_d", np.uint16),
                     ("blk_pkt", np.int64), ("pkt", np.uint8), ("dinv", np.float64)):
        (cnt,) = struct.unpack_from("<q", buf, o)
        o += 8
        size = cnt * np.dtype(dt).itemsize
        t[name] = np.frombuffer(buf, dtype=dt, count=cnt, offset=o).copy()
        o += size
    assert o == len(buf)
    t["scatter"] = scatter
    return rc, detail, t


def packet(t, b, nloc):
    """The sections of block b's packet (layout of csrc/packet.h): ids, d, loc, and with the
    scatter sections also incoff and pos (None otherwise)."""
    ne = int(t["blk_e0"][b + 1] - t["blk_e0"][b])
    nu = int(t["blk_u0"][b + 1] - t["blk_u0"][b])
    p = t["pkt"][t["blk_pkt"][b]:t["blk_pkt"][b + 1]]
    sc = t["scatter"]
    off_d = _pad16(4 * nu)
    off_inc = off_d + _pad16(2 * nu)
    sa = off_inc + (_pad16(2 * nu + 2) if sc else 0)
    m = ne * nloc
    assert p.size == sa + (2 if sc else 1) * _pad16(2 * m)
    ids = p[:4 * nu].view(np.int32)
    d = p[off_d:off_d + 2 * nu].view(np.uint16)
    loc = p[sa:sa + 2 * m].view(np.uint16)
    incoff = p[off_inc:off_inc + 2 * (nu + 1)].view(np.uint16) if sc else None
    pos = p[sa + _pad16(2 * m):sa + _pad16(2 * m) + 2 * m].view(np.uint16) if sc else None
    return ne, nu, ids, d, loc, incoff, pos


def check_invariants(t, l2g, signs, n, groups=None):
    E, nloc = l2g.shape
    perm = t["perm"]
    assert np.array_equal(np.sort(perm), np.arange(E))
    if groups is not None:
        assert np.all(np.diff(groups[perm]) >= 0)              # each mesh of a batch contiguous
    d = np.bincount(l2g.ravel(), minlength=n)
    np.testing.assert_allclose(t["dinv"], 1.0 / d, rtol=0, atol=0)
    seen_interior = []
    shared_slots = {}
    groups_seen = {}
    for b in range(t["nblk"]):
        ne, nu, ids, dm, loc, incoff, pos = packet(t, b, nloc)
        e0, nint = int(t["blk_e0"][b]), int(t["blk_nint"][b])
        assert 0 < ne <= t["BE"] and nu <= t["max_u"] and ne <= t["max_ne"]
        cells = perm[e0:e0 + ne]
        assert np.array_equal(dm, d[ids])
        assert len(set(ids.tolist())) == nu
        # loc: every copy (a, e) names its block-local dof and carries P's sign in bit 15
        u_of = (loc & 0x7FFF).astype(np.int64)
        neg = (loc & 0x8000) != 0
        for a in range(nloc):
            g = l2g[cells, a]
            assert np.array_equal(ids[u_of[a * ne:(a + 1) * ne]], g)
            s = np.ones(ne, bool) if signs is None else signs[cells, a] < 0
            assert np.array_equal(neg[a * ne:(a + 1) * ne], s if signs is not None else np.zeros(ne, bool))
        counts = np.bincount(u_of, minlength=nu)
        assert counts.max() <= t["max_copies"]
        if pos is not None:
            # pos: a permutation of the slots; dof u's copies fill [incoff[u], incoff[u+1]) by ascending slot
            assert np.array_equal(np.sort(pos), np.arange(ne * nloc))
            assert incoff[0] == 0 and incoff[nu] == ne * nloc
            assert np.array_equal(np.diff(incoff.astype(np.int64)), counts)
            for u in range(nu):
                slots = np.nonzero(u_of == u)[0]               # ascending slot a * ne + e
                assert np.array_equal(pos[slots], np.arange(incoff[u], incoff[u + 1]))
        assert np.array_equal(counts[:nint], d[ids[:nint]])   # interior: every copy in the block
        assert np.all(counts[nint:] < d[ids[nint:]])
        assert np.all(np.diff(ids[:nint]) > 0)                 # interior dofs by ascending id
        seen_interior += ids[:nint].tolist()
        for j, g in enumerate(ids[nint:]):
            shared_slots.setdefault(int(g), []).append((b, int(t["blk_p0"][b]) + j))
        # the block's groups cover its shared dofs in order, each a contiguous run
        g0, g1 = int(t["blk_g0"][b]), int(t["blk_g0"][b + 1])
        assert g1 - g0 <= t["max_bg"]
        u = nint
        for k in range(g0, g1):
            g = int(t["bg_gid"][k])
            assert int(t["bg_u"][k]) == u
            size = int(t["grp_size"][g])
            assert np.all(np.diff(ids[u:u + size]) > 0)           # ascending ids inside a group
            groups_seen.setdefault(g, []).append((b, ids[u:u + size].tolist(), int(t["blk_p0"][b]) + u - nint))
            u += size
        assert u == nu
    assert sorted(seen_interior + list(shared_slots)) == list(range(n))   # each dof ends somewhere once
    assert t["nsh"] == len(shared_slots)
    assert t["npart"] == sum(len(v) for v in shared_slots.values())
    ngrp = t["grp_size"].size
    assert sorted(groups_seen) == list(range(ngrp))
    block_set = {}
    for g, members in groups_seen.items():
        blocks = [mb for mb, _, _ in members]
        assert blocks == sorted(blocks) and len(blocks) == int(t["grp_cnt"][g])    # ascending block order
        assert all(lst == members[0][1] for _, lst, _ in members)             # same dofs, same order
        sl = t["grp_slots"][t["grp_slot0"][g]:t["grp_slot0"][g + 1]].tolist()
        assert sl == [s0 for _, _, s0 in members]
        # the combine pass's group-major items: the group's dofs in order, with their d
        items = t["sh_ids"][t["grp_item0"][g]:t["grp_item0"][g + 1]].tolist()
        assert items == members[0][1]
        assert t["sh_d"][t["grp_item0"][g]:t["grp_item0"][g + 1]].tolist() == [int(d[v]) for v in items]
        for dof in members[0][1]:
            assert [bb for bb, _ in shared_slots[dof]] == blocks               # the dof's blocks = the group's
            block_set[dof] = tuple(blocks)
    # a group holds every shared dof of its block set: no two groups share one
    sets = {}
    for g, members in groups_seen.items():
        key = tuple(mb for mb, _, _ in members)
        assert key not in sets
        sets[key] = g


def replay(t, A, x, nloc, bras):
    """The block apply from the packets alone; A[K] = the cell operator (M_K or M_K^{-1})."""
    perm = t["perm"]
    y = np.zeros_like(x)
    part = np.zeros(t["npart"])
    for b in range(t["nblk"]):
        ne, nu, ids, dm, loc, incoff, pos = packet(t, b, nloc)
        e0, nint = int(t["blk_e0"][b]), int(t["blk_nint"][b])
        xs = x[ids] / dm if bras else x[ids]
        ys = np.zeros(nu)
        sign = np.where(loc & 0x8000, -1.0, 1.0)
        u_of = (loc & 0x7FFF).astype(np.int64)
        if pos is None:     # fixed-point path: products straight into the dofs' accumulators
            for e in range(ne):
                sl = np.arange(nloc) * ne + e
                xl = sign[sl] * xs[u_of[sl]]
                np.add.at(ys, u_of[sl], sign[sl] * (A[perm[e0 + e]] @ xl))
        else:               # scatter path: products to the dof-sorted slots, then each dof's run
            zs = np.zeros(ne * nloc)
            for e in range(ne):
                sl = np.arange(nloc) * ne + e
                xl = sign[sl] * xs[u_of[sl]]
                zs[pos[sl]] = sign[sl] * (A[perm[e0 + e]] @ xl)
            for u in range(nu):
                ys[u] = zs[incoff[u]:incoff[u + 1]].sum()
        for u in range(nu):
            acc = ys[u]
            if u < nint:
                y[ids[u]] = acc / dm[u] if bras else acc
            else:
                part[t["blk_p0"][b] + u - nint] = acc
    # the combine pass: every group's dofs, partials in ascending block order
    for g in range(t["grp_item0"].size - 1):
        i0, i1 = t["grp_item0"][g], t["grp_item0"][g + 1]
        slots = t["grp_slots"][t["grp_slot0"][g]:t["grp_slot0"][g + 1]]
        for i in range(i1 - i0):
            acc = 0.0
            for sl in slots:
                acc += part[sl + i]
            y[t["sh_ids"][i0 + i]] = acc / t["sh_d"][i0 + i] if bras else acc
    return y


CASES = {
    "2d_p2_be32": (lambda: mg.unit_square_mesh(9, jitter=0.2, seed=1), "h1", 2, 32),
    "3d_p3_be64": (lambda: mg.unit_cube_mesh(3, jitter=0.15, seed=2), "h1", 3, 64),
    "hcurl2_signed_be96": (lambda: mg.relabel_mesh(mg.unit_cube_mesh(3), seed=3), "hcurl", 1, 96),
    "hdiv2_be256": (lambda: mg.unit_cube_mesh(3), "hdiv", 2, 256),
    "bdm2d_be32": (lambda: mg.relabel_mesh(mg.unit_square_mesh(6, jitter=0.1, seed=4), seed=5), "bdm", 2, 32),
    "one_cell": (lambda: mg.single_simplex_mesh(3, seed=6), "hcurl", 2, 32),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_tables_replay_the_oracle_operators(dump_exe, tmp_path, case):
    make, space, order, BE = CASES[case]
    mesh = make()
    n, l2g, signs = mg.dof_map(mesh, space, order)
    rc, _, t = build_tables(dump_exe, tmp_path, mesh, l2g, signs, n, BE, scatter=space != "h1")
    assert rc == 0
    assert t["nblk"] == -(-mesh.n_cell // BE)
    check_invariants(t, l2g, signs, n)
    pr = Problem(mesh, space, order, l2g, signs, n)
    x = mg.rhs(n, 1, seed=7)
    ym = replay(t, pr.Me, x, l2g.shape[1], bras=False)
    yb = replay(t, pr.Minv_loc, x, l2g.shape[1], bras=True)
    scale = lambda v: np.abs(v).max()
    assert np.abs(ym - pr.M @ x).max() <= 1e-12 * scale(pr.M @ x)
    assert np.abs(yb - pr.B @ x).max() <= 1e-12 * scale(pr.B @ x)


def test_batched_groups_stay_contiguous(dump_exe, tmp_path):
    """Cells of one mesh of a batch stay contiguous in the cell order (a block may straddle
    two meshes: their dofs are disjoint, so its sums never mix them)."""
    a, b = mg.unit_cube_mesh(2, jitter=0.1, seed=8), mg.unit_cube_mesh(3, jitter=0.1, seed=9)
    coords = np.concatenate([a.coords, b.coords])
    cells = np.concatenate([a.cells, b.cells + a.n_vert]).astype(np.int32)
    mesh = mg.Mesh(coords, cells, 3)
    n, l2g, signs = mg.dof_map(mesh, "h1", 2)
    groups = np.repeat([0, 1], [a.n_cell, b.n_cell]).astype(np.int32)
    rc, _, t = build_tables(dump_exe, tmp_path, mesh, l2g, signs, n, 64, groups)
    assert rc == 0
    check_invariants(t, l2g, signs, n, groups)


def test_error_codes_of_a_bad_map(dump_exe, tmp_path):
    mesh = mg.unit_square_mesh(3)
    n, l2g, signs = mg.dof_map(mesh, "h1", 1)
    bad = l2g.copy()
    bad[4, 2] = n                                           # out of range: detail = flat index
    rc, detail, _ = build_tables(dump_exe, tmp_path, mesh, bad, signs, n, 32)
    assert rc == -2 and detail == 4 * l2g.shape[1] + 2
    rc, detail, _ = build_tables(dump_exe, tmp_path, mesh, l2g, signs, n + 1, 32)
    assert rc == -3 and detail == n                         # dof n has no copy
