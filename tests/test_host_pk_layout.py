"""The per-cell packed-matrix layout (csrc/packet.h, pk_index), compiled on the host: tiles of
32 cells in which 16-byte group g of the tile's cells forms one 512-byte row and the rows
follow in g order.  Checked: the map is one-to-one into the allocation of (cells rounded up to
32) x ceil(npk / G) x G elements, each cell's G consecutive entries share one 16-byte group,
and the 32 cells of a tile fill each row contiguously (what a warp of consecutive cells reads
as one 512-byte row)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(__file__)
CSRC = os.path.join(HERE, "..", "paper_2607_12138_b300", "csrc")


@pytest.fixture(scope="module")
def tool(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("pk") / "pk_layout")
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", CSRC, os.path.join(HERE, "host", "pk_layout.cpp"), "-o", exe],
                   check=True)
    return exe


@pytest.mark.parametrize("E,npk,G", [(1, 10, 4), (37, 10, 4), (64, 1035, 4), (70, 210, 2), (45, 1035, 8), (33, 3, 8)])
def test_tile_layout(tool, E, npk, G):
    out = subprocess.run([tool, str(E), str(npk), str(G)], check=True, capture_output=True, text=True).stdout
    idx = np.array(out.split(), dtype=np.int64).reshape(E, npk)
    ng = -(-npk // G)
    epad = -(-E // 32) * 32
    assert len(np.unique(idx)) == idx.size                     # one-to-one
    assert idx.min() >= 0 and idx.max() < epad * ng * G         # inside the allocation
    grp = idx // G
    for i in range(npk):                                        # entries of one group: one 16-byte run
        assert np.all(idx[:, i] % G == i % G)
        assert np.all(grp[:, i] == grp[:, (i // G) * G])
    # row g of a tile: the tile's 32 cells at consecutive group positions
    for e in range(E):
        t, c = divmod(e, 32)
        for g in range(ng):
            i = g * G
            assert grp[e, i] == (t * ng + g) * 32 + c
