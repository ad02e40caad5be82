"""Host (CPU) check of the complex128 fixed-point helpers the sweep kernels use.

Compiles tests/fixedpoint_check.cpp against paper_2407_13012_gb300/csrc/fixedpoint.cuh
with the host C++ compiler and runs it: the limb-product complex multiply against exact
128-bit rounding, and the integer-only float64 conversions against the C library's
correctly rounded ones.
"""
import shutil
import subprocess
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent


def test_fixedpoint_helpers(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "fixedpoint_check"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", str(ROOT / "paper_2407_13012_gb300" / "csrc"),
                    str(ROOT / "tests" / "fixedpoint_check.cpp"), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().endswith("OK")
