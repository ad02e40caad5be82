"""CPU check of the register/thread layouts and shared-memory swizzles of every tile
configuration the kernels instantiate (read from the CUDA sources): idx(k, tid, r) is a
bijection onto [0, 2^B) in every layout, the layouts' new bit ranges cover all B bits,
phys() is a bijection, and each warp-wide shared-memory access (fixed r) is free of bank
conflicts for the element size (8 bytes complex64, 16 bytes complex128)."""
import re
from pathlib import Path

import pytest

CSRC = Path(__file__).resolve().parent.parent / "paper_2407_13012_gb300" / "csrc"


def configs():
    out = {}
    for f in ("sweeper.cuh", "batch_kernel.cuh"):
        for name, b, rb, sw, sww, minb in re.findall(
                r"using (Cfg\w+) = Cfg<(\d+), (\d+), (\d+), (\d+), (\d+)>;", (CSRC / f).read_text()):
            elem = 8 if name.startswith("CfgF") else 16  # F: complex64, X: complex128 fixed point
            out[name] = (int(b), int(rb), int(sw), int(sww), elem)
    return out


def lo(B, RB, k):
    return max(0, B - RB * (k + 1))


def idx(B, RB, k, tid, r):
    l = lo(B, RB, k)
    return (tid & ((1 << l) - 1)) | (r << l) | ((tid >> l) << (l + RB))


def test_config_list_is_complete():
    names = set(configs())
    assert {"CfgF1", "CfgF3", "CfgX1", "CfgX2", "CfgXB", "CfgXS", "CfgFB", "CfgFS"} <= names


@pytest.mark.parametrize("name", sorted(configs()))
def test_layouts_and_swizzle(name):
    B, RB, SW, SWW, es = configs()[name]
    R, NT = 1 << RB, 1 << (B - RB)
    NR = (B + RB - 1) // RB

    def phys(i):
        return i ^ ((i >> SW) & ((1 << SWW) - 1))

    assert sorted(phys(i) for i in range(1 << B)) == list(range(1 << B))
    covered = set()
    for k in range(NR):
        assert {idx(B, RB, k, t, r) for t in range(NT) for r in range(R)} == set(range(1 << B)), k
        newhi = B if k == 0 else lo(B, RB, k - 1)
        covered |= set(range(lo(B, RB, k), newhi))
        per_row = 128 // es  # slots per 128-byte wavefront
        for r in range(R):
            for w0 in range(0, NT, 32):
                lanes = [phys(idx(B, RB, k, t, r)) for t in range(w0, min(w0 + 32, NT))]
                for g0 in range(0, len(lanes), per_row):
                    banks = [x % per_row for x in lanes[g0:g0 + per_row]]
                    assert len(set(banks)) == len(banks), (name, k, r)
    assert covered == set(range(B))
