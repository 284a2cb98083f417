"""The FP32 fixed-point arithmetic of the H1 block kernels, restated on the host
(tests/host/fixed_split.cpp, IEEE binary32 with round to nearest even): a scaled product s with
|s| < 2^(L + 22) splits into integers (qh, ql) with qh 2^L + ql = rint(s) exactly and
|ql| <= 2^(L-1), by the form that takes s and by the form that takes t = s 2^-L (the kernels
fold 2^-L into the cell's scale factor) with the same two integers, ties included; and a
total (hi word |hi| < 2^22, lo word |lo| <= 2^29) converts back by one FMA within half an ulp
plus 32 units, exactly rounded whenever |lo| <= 2^24."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(__file__)


@pytest.fixture(scope="module")
def tool(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("fx") / "fixed_split")
    subprocess.run([cxx, "-O1", "-std=c++17", "-ffp-contract=off", os.path.join(HERE, "host", "fixed_split.cpp"),
                    "-o", exe], check=True)
    return exe


@pytest.mark.parametrize("L", [10, 14, 18, 22])
def test_split_and_conversion(tool, L):
    r = subprocess.run([tool, str(L), "200000", str(17 + L)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    _, nsplit, _, nconv, _, nexact = r.stdout.split()
    assert int(nsplit) > 190000 and int(nconv) == 200000 and int(nexact) > 10000
