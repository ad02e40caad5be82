"""Write the oracle's <C>, norm and adjoint gradient for sizes too slow to recompute in a test.

Calls only ``oracle/`` (and the seeded input generators in ``synth/``); nothing
here comes from the CUDA path.  Each case is the plain-workload family at a size
where the oracle's adjoint pass (Sec. II-B, IV-C) takes minutes on one core:

  reg3_int_n26_p6   random 3-regular, n = 26, integer weights {1..10}, seed 0,
                    p = 6, angles U(0, pi) from seed 0 (the bench workload's
                    family and seeds at n = 26)

Run:  python tests/golden/make_fullsize_golden.py [case ...]
Output: tests/golden/<case>.txt, one "key value" line per quantity, values
written with repr() so they round-trip exactly.
"""
from __future__ import annotations

import sys
import time
from pathlib import Path

HERE = Path(__file__).resolve().parent
ROOT = HERE.parent.parent
sys.path.insert(0, str(ROOT))

import numpy as np  # noqa: E402

import synth  # noqa: E402
from oracle import qaoa  # noqa: E402

CASES = {
    "reg3_int_n26_p6": dict(family="reg3", n=26, seed=0, weights="int", p=6, angle_seed=0),
}


def instance(spec):
    e, w, integer = synth.graph(spec["family"], spec["n"], spec["seed"], weights=spec["weights"])
    gam, bet = synth.angles(spec["p"], spec["angle_seed"])
    return e, w, integer, gam, bet


def write_case(name: str) -> Path:
    spec = CASES[name]
    n = spec["n"]
    e, w, integer, gam, bet = instance(spec)
    C = qaoa.cut_values(n, e, w, integer=integer)
    t0 = time.time()
    E, dg, db, back = qaoa.adjoint_gradient(n, C, gam, bet)
    secs = time.time() - t0
    out = HERE / f"{name}.txt"
    lines = [
        f"# oracle.qaoa.adjoint_gradient, {spec}",
        f"# written by tests/golden/make_fullsize_golden.py ({secs:.0f} s on one core)",
        f"n {n}",
        f"p {spec['p']}",
        f"W {float(np.sum(np.abs(w)))!r}",
        f"E {E!r}",
    ]
    lines += [f"dgamma{l} {float(v)!r}" for l, v in enumerate(dg)]
    lines += [f"dbeta{l} {float(v)!r}" for l, v in enumerate(db)]
    lines.append(f"uncompute_residual {float(np.linalg.norm(back - qaoa.plus_state(n)))!r}")
    out.write_text("\n".join(lines) + "\n")
    return out


def read_case(name: str) -> dict:
    vals = {}
    for line in (HERE / f"{name}.txt").read_text().splitlines():
        if not line or line.startswith("#"):
            continue
        k, v = line.split()
        vals[k] = float(v)
    return vals


if __name__ == "__main__":
    for name in sys.argv[1:] or list(CASES):
        print(write_case(name))
