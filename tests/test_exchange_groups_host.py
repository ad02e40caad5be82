"""Host check of the sweep kernels' tile layouts and exchange barriers.

Compiles tests/exchange_groups_check.cpp against paper_2407_13012_gb300/csrc/tile_layout.cuh,
with every configuration the kernel sources declare, and runs it: every layout is a bijection, every value read in a move was written inside the
move's barrier set, and every named barrier id joins the same warps with a matching count.
"""
import re
import shutil
import subprocess
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent


def test_exchange_groups(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    csrc = ROOT / "paper_2407_13012_gb300" / "csrc"
    cfgs = []
    for f in ("sweeper.cuh", "batch_kernel.cuh"):
        cfgs += re.findall(r"using (Cfg\w+) = (Cfg<\d+, \d+, \d+, \d+, \d+>);", (csrc / f).read_text())
    assert {"CfgF1", "CfgF3", "CfgX1", "CfgX2", "CfgXB", "CfgXS", "CfgFB", "CfgFS"} <= {c[0] for c in cfgs}
    (tmp_path / "exchange_cfgs.inc").write_text("".join(f'check<{t}>("{n}");\n' for n, t in cfgs))
    exe = tmp_path / "exchange_groups_check"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", str(csrc), "-I", str(tmp_path),
                    str(ROOT / "tests" / "exchange_groups_check.cpp"), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().endswith("OK")
