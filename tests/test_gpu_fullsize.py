"""Parity at the sizes the full workload runs, through the C ABI, against the FP64 oracle.

* Sampling (Sec. IV-D) with a multi-chunk prefix scan: the scan groups 4096 leaves of
  1024 amplitudes per chunk, so n = 24 and n = 26 cross 4 and 16 chunk boundaries.
  The oracle's sampler reads the same (uploaded) amplitudes under the same uniforms;
  a crafted state puts its mass on both sides of chunk boundaries with zero-mass
  leaves between, so a wrong cross-chunk offset cannot pass.
* complex128 layers at p = 6 on the plain workload's family (random 3-regular,
  integer weights {1..10}, seed 0, angles from seed 0) for n = 20..26: the state
  element by element, <C> within 1e-10 max(1, W).  The state is held in int64
  fixed point (value = integer 2^-54) inside a call; each rounding of a group mixer
  2^-t W D W adds an error of 2-norm 0.41 2^((n + t)/2 - 54) (t <= 12 qubits per
  group, three groups per layer), so the bound checked is three times the
  root-sum-square of those terms over the 3p group mixers.
* The adjoint gradient at n = 26, p = 6 against the oracle's adjoint pass
  (Sec. II-B, IV-C), whose values tests/golden/make_fullsize_golden.py wrote.
* The p = 1 gradient at n = 28, 30, 31 (complex128) and 32 (complex64) against the
  analytic derivative of the per-edge closed form (oracle/closed_form.py).

Setting QAOA_TEST_REPORT to a file path appends the measured errors as JSON lines.
"""
import json
import math
import os
import sys
from pathlib import Path

import numpy as np
import pytest

import synth
from oracle import closed_form, qaoa

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2407_13012_gb300 as q  # noqa: E402

sys.path.insert(0, str(Path(__file__).resolve().parent / "golden"))
import make_fullsize_golden as golden  # noqa: E402

LEAF = 1 << 10                 # amplitudes per sampling leaf
CHUNK_AMPS = (1 << 12) * LEAF  # amplitudes covered by one scan chunk


def report(**kv):
    path = os.environ.get("QAOA_TEST_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(kv) + "\n")
    print(kv)


def to_np(t):
    return t.detach().cpu().numpy()


def scale_of(w):
    return max(1.0, float(np.sum(np.abs(w))))


def free():
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


# ------------------------------------------------------------------ sampling across scan chunks

def _sample_check(n, psi_ref, graph, C, dtype, shots, seed):
    tdt = torch.complex128 if dtype == "c128" else torch.complex64
    psi = torch.as_tensor(psi_ref).to(tdt).cuda()
    ref_in = to_np(psi.cpu()).astype(np.complex128)  # exactly the values the sampler reads
    cv = q.cost_vector(graph, "i32")
    z, cz = q.sample(psi, cv, shots, seed)
    z = to_np(z).astype(np.int64)
    cz = to_np(cz)
    zr, _ = qaoa.sample(ref_in, C, synth.sample_uniforms(seed, shots))
    mism = float(np.mean(zr.astype(np.int64) != z))
    assert np.all((z >= 0) & (z < (1 << n)))
    assert np.array_equal(cz, C[z].astype(np.float64))
    assert np.all(np.abs(ref_in[z]) > 0)
    assert mism <= 1e-5
    del psi, cv
    free()
    return z, mism


@pytest.mark.parametrize("n,dtype", [(24, "c64"), (24, "c128"), (26, "c64")])
def test_sample_multichunk_parity(n, dtype):
    e, w, integer = synth.graph("reg3", n, 3, weights="int")
    C = qaoa.cut_values(n, e, w)
    psi_ref = synth.random_state(n, 17 + n)
    z, mism = _sample_check(n, psi_ref, q.Graph(n, e, w, integer), C, dtype, 200_000, 4242 + n)
    chunks = np.unique(z >> 22)
    assert len(chunks) == 1 << (n - 22)  # every chunk was hit
    report(test="sample_multichunk", n=n, dtype=dtype, chunks=1 << (n - 22), mismatch=mism)


def test_sample_mass_across_chunk_boundaries():
    """Mass in the last leaves of chunk 0, none in chunk 1 and the first half of chunk 2,
    mass straddling the chunk 2 / chunk 3 boundary, and in the last 100 amplitudes."""
    n = 24
    e, w, integer = synth.graph("gnp", n, 5, weights="int", prob=0.1)
    C = qaoa.cut_values(n, e, w)
    rng_u = synth.uniforms(77, "state", 2 << n).reshape(-1, 2) - 0.5
    psi = np.zeros(1 << n, dtype=np.complex128)
    spans = [(CHUNK_AMPS - 3000, CHUNK_AMPS), (3 * CHUNK_AMPS - 5000, 3 * CHUNK_AMPS + 2000),
             ((1 << n) - 100, 1 << n)]
    for lo, hi in spans:
        psi[lo:hi] = rng_u[lo:hi, 0] + 1j * rng_u[lo:hi, 1]
    psi /= np.linalg.norm(psi)
    for dtype in ("c128", "c64"):
        z, mism = _sample_check(n, psi, q.Graph(n, e, w, integer), C, dtype, 100_000, 9)
        inside = np.zeros(len(z), dtype=bool)
        for lo, hi in spans:
            inside |= (z >= lo) & (z < hi)
        assert inside.all()
        # each span receives close to its probability mass
        for lo, hi in spans:
            pm = float(np.sum(np.abs(psi[lo:hi]) ** 2))
            got = float(np.mean((z >= lo) & (z < hi)))
            assert abs(got - pm) <= 5 * math.sqrt(pm * (1 - pm) / len(z)) + 1e-3
        report(test="sample_chunk_boundaries", n=n, dtype=dtype, mismatch=mism)


# ------------------------------------------------------------------ complex128 state, <C> and gradient at p = 6

FX_SHIFT = 54   # fixed-point scale 2^-54 of the complex128 state inside a call
T_MAX = 12      # largest qubit group of a complex128 sweep


def fx_state_error_bound(n, p, groups=3):
    per_mixer = 0.41 * 2.0 ** ((n + T_MAX) / 2 - FX_SHIFT)
    return 3.0 * math.sqrt(groups * p) * per_mixer


def bench_family(n, p):
    e, w, integer = synth.graph("reg3", n, 0, weights="int")
    gam, bet = synth.angles(p, 0)
    return e, w, integer, gam, bet


@pytest.mark.parametrize("n", [20, 22, 24, 26])
def test_c128_state_and_expectation_p6(n):
    p = 6
    e, w, integer, gam, bet = bench_family(n, p)
    C = qaoa.cut_values(n, e, w)
    cv = q.cost_vector(q.Graph(n, e, w, integer), "i32")
    psi = q.new_state(n, "c128")
    out = to_np(q.apply_layers(psi, cv, gam, bet, expect=True))
    got = to_np(psi.cpu())
    del psi, cv
    free()
    ref = qaoa.qaoa_state(n, C, gam, bet)
    Eref = qaoa.expectation(ref, C)
    err = float(np.linalg.norm(got - ref))
    bound = fx_state_error_bound(n, p)
    report(test="c128_state_p6", n=n, p=p, state_err_2norm=err, bound=bound, dE=float(out[0] - Eref),
           W=float(np.sum(w)), max_abs_err=float(np.max(np.abs(got - ref))))
    assert err <= bound
    assert abs(out[0] - Eref) <= 1e-10 * scale_of(w)
    assert abs(out[1] - 1.0) <= 1e-12


def test_c128_gradient_n26_p6_against_oracle():
    name = "reg3_int_n26_p6"
    ref = golden.read_case(name)
    spec = golden.CASES[name]
    n, p = spec["n"], spec["p"]
    e, w, integer, gam, bet = golden.instance(spec)
    assert int(ref["n"]) == n and int(ref["p"]) == p and ref["W"] == float(np.sum(np.abs(w)))
    cv = q.cost_vector(q.Graph(n, e, w, integer), "i32")
    psi = q.new_state(n, "c128")
    lam = q.new_state(n, "c128")
    out = to_np(q.gradient(psi, lam, cv, gam, bet))
    back = to_np(psi.cpu())
    del psi, lam, cv
    free()
    tol = 1e-10 * scale_of(w)
    dg = np.array([ref[f"dgamma{l}"] for l in range(p)])
    db = np.array([ref[f"dbeta{l}"] for l in range(p)])
    report(test="c128_gradient_n26_p6", dE=float(out[0] - ref["E"]),
           max_dgamma=float(np.max(np.abs(out[2:2 + p] - dg))), max_dbeta=float(np.max(np.abs(out[2 + p:] - db))),
           tol=tol, uncompute_residual=float(np.linalg.norm(back - qaoa.plus_state(n))))
    assert abs(out[0] - ref["E"]) <= tol and abs(out[1] - 1.0) <= 1e-12
    assert np.max(np.abs(out[2:2 + p] - dg)) <= tol
    assert np.max(np.abs(out[2 + p:] - db)) <= tol
    assert np.linalg.norm(back - qaoa.plus_state(n)) <= 10 * fx_state_error_bound(n, 2 * p)


# ------------------------------------------------------------------ p = 1 gradient against the closed form

@pytest.mark.parametrize("n,dtype,fam,kind", [(28, "c128", "reg3", "u01"), (30, "c128", "reg3", "u01"),
                                              (30, "c128", "reg3", "int"), (31, "c128", "gnp", "u01"),
                                              (32, "c64", "reg3", "int")])
def test_p1_gradient_against_closed_form(n, dtype, fam, kind):
    e, w, integer = synth.graph(fam, n, 2, weights=kind, prob=0.1)
    cv = q.cost_vector(q.Graph(n, e, w, integer), "i32" if integer else "f64")
    gam, bet = synth.angles(1, 5 + n)
    psi = q.new_state(n, dtype)
    lam = q.new_state(n, dtype)
    out = to_np(q.gradient(psi, lam, cv, gam, bet))
    del psi, lam, cv
    free()
    E = closed_form.expectation_p1(n, e, w, gam[0], bet[0])
    dg, db = closed_form.gradient_p1_exact(n, e, w, gam[0], bet[0])
    report(test="p1_gradient_closed_form", n=n, dtype=dtype, dE=float(out[0] - E), ddg=float(out[2] - dg),
           ddb=float(out[3] - db))
    if dtype == "c128":
        tol = 1e-10 * scale_of(w)
        assert abs(out[0] - E) <= tol and abs(out[2] - dg) <= tol and abs(out[3] - db) <= tol
    else:
        assert abs(out[0] - E) <= 1e-4 * max(1.0, abs(E))
        assert abs(out[2] - dg) <= 1e-4 * max(1.0, abs(dg))
        assert abs(out[3] - db) <= 1e-4 * max(1.0, abs(db))
