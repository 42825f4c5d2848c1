"""The O(n) host passes of the matrix assembly (threads over row ranges)
give exactly the serial results: compiled with the library's host source and
run as a small program (no GPU)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2212_09642_gb300", "csrc")


def test_threaded_relabel_matches_serial(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path / "relabel_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-pthread", "-I", CSRC,
                    os.path.join(ROOT, "tests", "host_relabel_check.cpp"), os.path.join(CSRC, "host_graph.cpp"),
                    "-o", exe], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=300).stdout
    assert "ALL OK" in out, out
