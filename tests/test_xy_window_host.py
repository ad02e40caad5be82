"""Host check of the windowed XY-mixer passes.

Compiles tests/xy_window_check.cpp against paper_2407_13012_gb300/csrc/xy_window.cuh and runs
it: the windows hold every ring pair once and in the ring's parity order, and every tile
element addresses the right state of F_k exactly once (exhaustively for n <= 16, by sampled
tiles up to n = 40), within the kernel's fixed shared-memory arrays.
"""
import shutil
import subprocess
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent


def test_xy_window_tiles(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "xy_window_check"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", str(ROOT / "paper_2407_13012_gb300" / "csrc"),
                    str(ROOT / "tests" / "xy_window_check.cpp"), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().endswith("OK")
