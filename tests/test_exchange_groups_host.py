"""Host check of the sweep kernels' tile layouts and exchange barriers.

Compiles tests/exchange_groups_check.cpp against paper_2407_13012_gb300/csrc/tile_layout.cuh
and runs it: every layout is a bijection, every value read in a move was written inside the
move's barrier set, and every named barrier id joins the same warps with a matching count.
"""
import shutil
import subprocess
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent


def test_exchange_groups(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "exchange_groups_check"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", str(ROOT / "paper_2407_13012_gb300" / "csrc"),
                    str(ROOT / "tests" / "exchange_groups_check.cpp"), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().endswith("OK")
