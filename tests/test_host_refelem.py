"""The library's reference-element construction (csrc/refelem.cpp) against the oracle, on the CPU.

``tests/host/refelem_dump.cpp`` writes the library's reference mass blocks
R_ab = int_ref phi^a phi^b (and, for RT_k / BDM_k on tetrahedra, the divergence block against
the orthonormal DG_{k-1} basis).  The two sides build them differently (Whitney-form spans,
Silvester products and Gauss rules in long double against exact rationals and 40-digit
arithmetic), so agreement to ~1e-13 pins the library's dof functionals, spans and quadrature
to the oracle's, family by family and order by order.
"""
import os
import subprocess

import numpy as np
import pytest

from oracle import elements
from oracle.schur import reference_divergence

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2607_12138_b300", "csrc")
SPACE = {"h1": (0, 0), "h1b": (0, 1), "h1g": (0, 2), "hcurl": (1, 0), "hdiv": (2, 0), "n2curl": (1, 1),
         "bdm": (2, 1)}


@pytest.fixture(scope="module")
def dump_exe(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("refelem") / "refelem_dump")
    cmd = ["g++", "-O2", "-std=c++17", "-I" + CSRC, os.path.join(ROOT, "tests", "host", "refelem_dump.cpp"),
           os.path.join(CSRC, "refelem.cpp"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail("g++ failed:\n" + r.stderr)
    return exe


def library_tables(exe, tmp, dim, space, order):
    s, basis = SPACE[space]
    out = str(tmp / "ref.bin")
    assert subprocess.run([exe, str(dim), str(s), str(order), str(basis), out]).returncode == 0
    buf = open(out, "rb").read()
    rc = np.frombuffer(buf, np.int32, 1)[0]
    if rc != 0:
        return None
    nloc, ncomp, nq = np.frombuffer(buf, np.int32, 3, 4)
    R = np.frombuffer(buf, np.float64, 9 * nloc * nloc if ncomp == 3 else nloc * nloc, 16)
    Bd = np.frombuffer(buf, np.float64, nq * nloc, 16 + R.nbytes)
    R = R.reshape(3, 3, nloc, nloc) if ncomp == 3 else R.reshape(1, 1, nloc, nloc)
    return R, Bd.reshape(nq, nloc)


FAMILIES = ([("h1", d, p) for d in (2, 3) for p in (1, 2, 3, 4)] + [("h1b", d, p) for d in (2, 3) for p in (2, 4)]
            + [("h1g", d, p) for d in (2, 3) for p in (3, 4)]
            + [(s, d, k) for s in ("hcurl", "hdiv") for d in (2, 3) for k in (1, 2, 3, 4)]
            + [(s, d, k) for s in ("n2curl", "bdm") for d in (2, 3) for k in (1, 2, 3, 4)])


@pytest.mark.parametrize("space,dim,order", FAMILIES)
def test_reference_mass_blocks_match_the_oracle(dump_exe, tmp_path, space, dim, order):
    R, Bd = library_tables(dump_exe, tmp_path, dim, space, order)
    ref = elements.reference_element(space, dim, order).mass_blocks()
    c = ref.shape[0]
    got = R[:c, :c]
    assert got.shape == ref.shape
    assert np.abs(got - ref).max() <= 5e-13 * np.abs(ref).max()
    if R.shape[0] == 3 and c < 3:                      # triangles: the third component is zero
        assert np.abs(R[2]).max() == 0 and np.abs(R[:, 2]).max() == 0
    if space in ("hdiv", "bdm") and dim == 3:
        Bo = reference_divergence(order, space)
        assert Bd.shape == Bo.shape
        assert np.abs(Bd - Bo).max() <= 5e-13 * np.abs(Bo).max()
    else:
        assert Bd.size == 0


def test_unsupported_orders_are_refused(dump_exe, tmp_path):
    assert library_tables(dump_exe, tmp_path, 3, "hcurl", 5) is None
    assert library_tables(dump_exe, tmp_path, 3, "bdm", 5) is None
    assert library_tables(dump_exe, tmp_path, 3, "h1", 0) is None
