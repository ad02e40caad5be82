"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (derived from the arithmetic, stated per check):
* cost vector: bit-exact for integer weights; float weights within
  (m + 1) 2^-52 max(1, sum|w|) (the oracle sums in edge order, the kernel sums a
  fixed-point quantisation exactly and rounds once).
* complex128: <C> and every gradient entry within 1e-10 max(1, sum|w|);
  state 2-norm error <= 1e-11.
* complex64: <C> and every gradient entry within 1e-4 max(1, |value|);
  state 2-norm error <= 1e-5.
* sampling: under the same uniforms the bitstrings agree except where the
  target lands within rounding of a CDF step (allowed fraction 1e-5); every
  returned cost equals C[z] exactly.
"""
import math

import numpy as np
import pytest

import synth
from oracle import closed_form, qaoa

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2407_13012_gb300 as q  # noqa: E402


def instance(fam, n, seed, weights, prob=0.5, lo=1, hi=10):
    if fam == "reg3" and (n % 2 or n < 4):
        fam = "gnp"
    e, w, integer = synth.graph(fam, n, seed, weights=weights, prob=prob, lo=lo, hi=hi)
    return q.Graph(n, e, w, integer), e, w, integer


def to_np(t):
    return t.detach().cpu().numpy()


def state_np(psi):
    return to_np(psi).astype(np.complex128)


def scale_of(w):
    return max(1.0, float(np.sum(np.abs(w))))


# ------------------------------------------------------------------ S1 cost vector

@pytest.mark.parametrize("n", [1, 2, 3, 5, 9, 10, 11, 12, 14, 17])
@pytest.mark.parametrize("fam", ["gnp", "reg3", "complete"])
def test_cost_vector_integer_bit_exact(n, fam):
    g, e, w, integer = instance(fam, n, n, "int", prob=0.4)
    ref = qaoa.cut_values(n, e, w, integer=True)
    cv = q.cost_vector(g, "i32")
    assert np.array_equal(to_np(cv.C).astype(np.int64), ref)
    assert cv.cmin <= ref.min() and ref.max() <= cv.cmax
    cf = q.cost_vector(g, "f64")
    assert np.array_equal(to_np(cf.C), ref.astype(np.float64))


def test_cost_vector_negative_weights_and_empty():
    g, e, w, integer = instance("gnp", 13, 3, "int", prob=0.5, lo=-5, hi=5)
    assert np.array_equal(to_np(q.cost_vector(g, "i32").C), qaoa.cut_values(13, e, w))
    g0 = q.Graph(6, np.zeros((0, 2), np.int32), None, True)
    assert not to_np(q.cost_vector(g0, "i32").C).any()


@pytest.mark.parametrize("n", [4, 11, 16])
def test_cost_vector_float_weights(n):
    g, e, w, integer = instance("gnp", n, 5, "u01", prob=0.6)
    ref = qaoa.cut_values(n, e, w, integer=False)
    got = to_np(q.cost_vector(g, "f64").C)
    tol = (len(e) + 1) * 2.0 ** -52 * scale_of(w)
    assert np.max(np.abs(got - ref)) <= tol


@pytest.mark.parametrize("scale", [1e-12, 1e-300, 1e12])
def test_cost_vector_float_weights_any_scale(scale):
    """The common fixed point follows sum|w|: tiny or huge weights keep their relative precision
    (the bound is relative to sum|w| itself, not to max(1, sum|w|))."""
    n = 13
    e, w, integer = synth.graph("gnp", n, 8, weights="u01", prob=0.5)
    w = w * scale
    g = q.Graph(n, e, w, False)
    ref = qaoa.cut_values(n, e, w, integer=False)
    got = to_np(q.cost_vector(g, "f64").C)
    assert np.max(np.abs(got - ref)) <= (len(e) + 1) * 2.0 ** -52 * float(np.sum(np.abs(w)))


def test_cost_vector_sampled_at_n30():
    n = 30
    g, e, w, integer = instance("reg3", n, 1, "int")
    cv = q.cost_vector(g, "i32")
    zs = np.concatenate([np.arange(64), (1 << n) - 1 - np.arange(64),
                         synth.draws_u64(4, "state", 4000).astype(np.uint64) % np.uint64(1 << n)]).astype(np.int64)
    got = to_np(cv.C[torch.as_tensor(zs, device="cuda")]).astype(np.int64)
    ref = np.zeros(len(zs), dtype=np.int64)
    for (u, v), we in zip(e, w):  # C(z) one z at a time, edge by edge
        ref += int(we) * (((zs >> u) ^ (zs >> v)) & 1)
    assert np.array_equal(got, ref)
    del cv


# ------------------------------------------------------------------ S2-S4 layers

LAYER_CASES = [(n, p) for n in (1, 2, 4, 7, 11, 12, 13, 16, 19) for p in (0, 1, 3)]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n,p", LAYER_CASES)
def test_layers_parity(n, p, dtype):
    kind = "int" if (n + p) % 2 else "u01"
    g, e, w, integer = instance("gnp", n, n + 7 * p, kind, prob=0.5)
    C = qaoa.cut_values(n, e, w, integer=integer)
    cv = q.cost_vector(g, "i32" if integer else "f64")
    gam, bet = synth.angles(p, 100 + n + p)
    psi = q.new_state(n, dtype)
    out = q.apply_layers(psi, cv, gam, bet, init=True, expect=True)
    ref = qaoa.qaoa_state(n, C, gam, bet)
    Eref = qaoa.expectation(ref, C)
    got = state_np(psi)
    E, nrm = to_np(out)
    if dtype == "c128":
        assert np.linalg.norm(got - ref) <= 1e-11
        assert abs(E - Eref) <= 1e-10 * scale_of(w)
        assert abs(nrm - 1.0) <= 1e-12
    else:
        assert np.linalg.norm(got - ref) <= 1e-5
        assert abs(E - Eref) <= 1e-4 * max(1.0, abs(Eref))
        assert abs(nrm - 1.0) <= 1e-5


@pytest.mark.parametrize("n,dtype,kind", [(22, "c128", "int"), (22, "c128", "u01"), (24, "c64", "int")])
def test_layers_three_groups(n, dtype, kind):
    """Sizes whose qubits split into three tile groups, compared element by element."""
    g, e, w, integer = instance("reg3", n, 9, kind)
    C = qaoa.cut_values(n, e, w, integer=integer)
    cv = q.cost_vector(g, "i32" if integer else "f64")
    gam, bet = synth.angles(3, 31)
    psi = q.new_state(n, dtype)
    out = to_np(q.apply_layers(psi, cv, gam, bet, expect=True))
    ref = qaoa.qaoa_state(n, C, gam, bet)
    Eref = qaoa.expectation(ref, C)
    got = state_np(psi)
    if dtype == "c128":
        assert np.linalg.norm(got - ref) <= 1e-11
        assert abs(out[0] - Eref) <= 1e-10 * scale_of(w)
    else:
        assert np.linalg.norm(got - ref) <= 1e-5
        assert abs(out[0] - Eref) <= 1e-4 * max(1.0, abs(Eref))


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n", [5, 12, 15])
def test_layers_continue_from_state(n, dtype):
    g, e, w, integer = instance("gnp", n, 3, "int", prob=0.5)
    C = qaoa.cut_values(n, e, w)
    cv = q.cost_vector(g, "i32")
    psi0 = synth.random_state(n, 11)
    gam, bet = synth.angles(2, 8)
    tdt = torch.complex128 if dtype == "c128" else torch.complex64
    psi = torch.as_tensor(psi0).to(tdt).cuda()
    q.apply_layers(psi, cv, gam, bet, init=False)
    ref = qaoa.qaoa_state(n, C, gam, bet, psi0=psi0)
    assert np.linalg.norm(state_np(psi) - ref) <= (1e-11 if dtype == "c128" else 1e-5)
    out = q.expectation(psi, cv)
    assert abs(to_np(out)[0] - qaoa.expectation(ref, C)) <= (1e-10 * scale_of(w) if dtype == "c128"
                                                              else 1e-4 * scale_of(w))


def test_table_bounds_wrong_still_correct():
    # a descriptor whose bounds do not cover every entry must still give the right state
    n = 10
    g, e, w, integer = instance("gnp", n, 2, "int", prob=0.5)
    C = qaoa.cut_values(n, e, w)
    cv = q.cost_vector(g, "i32")
    cv.cmax = max(cv.cmin, int(C.max()) // 2)
    gam, bet = synth.angles(2, 3)
    psi = q.new_state(n, "c128")
    q.apply_layers(psi, cv, gam, bet)
    assert np.linalg.norm(state_np(psi) - qaoa.qaoa_state(n, C, gam, bet)) <= 1e-11


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_table_bounds_outside_int32_still_correct(dtype):
    # bounds no int32 cost can reach: the kernels skip the table and compute every phase
    n = 10
    g, e, w, integer = instance("gnp", n, 4, "int", prob=0.5)
    C = qaoa.cut_values(n, e, w)
    cv = q.cost_vector(g, "i32")
    cv.cmin, cv.cmax = (1 << 40) - 3, (1 << 40) + 50
    gam, bet = synth.angles(2, 5)
    psi = q.new_state(n, dtype)
    q.apply_layers(psi, cv, gam, bet)
    err = np.linalg.norm(state_np(psi) - qaoa.qaoa_state(n, C, gam, bet))
    assert err <= (1e-11 if dtype == "c128" else 1e-5)


def test_empty_graph_and_zero_angles():
    n = 9
    g = q.Graph(n, np.zeros((0, 2), np.int32), None, True)
    cv = q.cost_vector(g, "i32")
    psi = q.new_state(n, "c128")
    out = q.apply_layers(psi, cv, [0.7, 1.1], [0.3, 0.2], expect=True)
    assert abs(to_np(out)[0]) == 0.0
    # |+> is an eigenvector of the mixer: amplitudes all equal
    a = state_np(psi)
    assert np.max(np.abs(a - a[0])) < 1e-14


@pytest.mark.parametrize("n,dtype", [(24, "c128"), (28, "c128"), (30, "c128"), (28, "c64"), (32, "c64")])
def test_large_p1_against_closed_form(n, dtype):
    fam = "reg3"
    g, e, w, integer = instance(fam, n, 2, "int" if dtype == "c64" else "u01")
    cv = q.cost_vector(g, "i32" if integer else "f64")
    gam, bet = synth.angles(1, 5)
    psi = q.new_state(n, dtype)
    out = to_np(q.apply_layers(psi, cv, gam, bet, expect=True))
    ref = closed_form.expectation_p1(n, e, w, gam[0], bet[0])
    if dtype == "c128":
        assert abs(out[0] - ref) <= 1e-10 * scale_of(w)
        assert abs(out[1] - 1.0) <= 1e-12
    else:
        assert abs(out[0] - ref) <= 1e-4 * max(1.0, abs(ref))
        assert abs(out[1] - 1.0) <= 1e-4
    del psi, cv
    torch.cuda.empty_cache()


def test_n31_complex128_p1_and_p2_invariants():
    """The largest complex128 size (34 GB state): G(31, 0.1), U(0,1) weights.  p = 1 against
    the closed form; p = 2 keeps the norm and, with beta_2 shifted by pi/2 (RX(pi) = -iX on
    every qubit, which commutes with C's bit-flip symmetry), the same <C>."""
    n = 31
    g, e, w, integer = instance("gnp", n, 4, "u01", prob=0.1)
    cv = q.cost_vector(g, "f64")
    gam, bet = synth.angles(2, 6)
    psi = q.new_state(n, "c128")
    out = to_np(q.apply_layers(psi, cv, gam[:1], bet[:1], expect=True))
    ref = closed_form.expectation_p1(n, e, w, gam[0], bet[0])
    assert abs(out[0] - ref) <= 1e-10 * scale_of(w) and abs(out[1] - 1.0) <= 1e-12
    a = to_np(q.apply_layers(psi, cv, gam, bet, expect=True))
    b = to_np(q.apply_layers(psi, cv, gam, bet + np.array([0.0, np.pi / 2]), expect=True))
    assert abs(a[1] - 1.0) <= 1e-12 and abs(b[1] - 1.0) <= 1e-12
    assert abs(a[0] - b[0]) <= 1e-10 * scale_of(w)
    del psi, cv
    torch.cuda.empty_cache()


# ------------------------------------------------------------------ S5-S6 sampling

def upload(psi_ref, dtype):
    """An oracle state rounded to the test dtype, on the device (sampler input)."""
    tdt = torch.complex128 if dtype == "c128" else torch.complex64
    return torch.as_tensor(psi_ref).to(tdt).cuda()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n,shots", [(1, 500), (3, 2000), (10, 4096), (14, 20000), (18, 100000)])
def test_sample_parity(n, shots, dtype):
    g, e, w, integer = instance("gnp", n, n, "int", prob=0.5)
    C = qaoa.cut_values(n, e, w)
    cv = q.cost_vector(g, "i32")
    ref = qaoa.qaoa_state(n, C, *synth.angles(2, n))
    psi = upload(ref, dtype)
    ref_in = to_np(psi.cpu()).astype(np.complex128)  # exactly the values the sampler reads
    seed = 1234 + n
    z, cz = q.sample(psi, cv, shots, seed)
    z = to_np(z).astype(np.int64)
    cz = to_np(cz)
    assert np.all((z >= 0) & (z < (1 << n)))
    assert np.array_equal(cz, C[z].astype(np.float64))
    zr, _ = qaoa.sample(ref_in, C, synth.sample_uniforms(seed, shots))
    assert np.mean(zr.astype(np.int64) != z) <= 1e-5
    assert np.all(np.abs(ref_in[z]) > 0)


def test_sample_chi_square_and_determinism():
    n = 12
    g, e, w, integer = instance("reg3", n, 4, "int")
    C = qaoa.cut_values(n, e, w)
    cv = q.cost_vector(g, "i32")
    ref = qaoa.qaoa_state(n, C, *synth.angles(3, 1))
    psi = upload(ref, "c64")
    shots = 200000
    z1, c1 = q.sample(psi, cv, shots, 99)
    z2, _ = q.sample(psi, cv, shots, 99)
    assert torch.equal(z1, z2)
    prob = np.abs(ref) ** 2
    vals = np.unique(C)
    pv = np.array([prob[C == v].sum() for v in vals])
    c1 = to_np(c1)
    obs = np.array([np.sum(c1 == v) for v in vals])
    keep = pv * shots > 5
    chi2 = np.sum((obs[keep] - shots * pv[keep]) ** 2 / (shots * pv[keep]))
    dof = keep.sum() - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof)


def test_sample_zero_shots_and_basis_state():
    n = 11
    g, e, w, integer = instance("gnp", n, 1, "int")
    C = qaoa.cut_values(n, e, w)
    cv = q.cost_vector(g, "i32")
    psi = torch.zeros(1 << n, dtype=torch.complex128, device="cuda")
    psi[1234] = 1j
    z, cz = q.sample(psi, cv, 1000, 5)
    assert np.all(to_np(z) == 1234) and np.all(to_np(cz) == C[1234])
    z, cz = q.sample(psi, cv, 0, 5)
    assert z.numel() == 0


# ------------------------------------------------------------------ S7 gradient

@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n,p", [(3, 1), (8, 2), (12, 3), (15, 2), (17, 4), (22, 2)])
def test_gradient_parity(n, p, dtype):
    kind = "u01" if n % 2 else "int"
    g, e, w, integer = instance("gnp", n, n + p, kind, prob=0.4)
    C = qaoa.cut_values(n, e, w, integer=integer)
    cv = q.cost_vector(g, "i32" if integer else "f64")
    gam, bet = synth.angles(p, 7 * n + p)
    psi = q.new_state(n, dtype)
    lam = q.new_state(n, dtype)
    out = to_np(q.gradient(psi, lam, cv, gam, bet))
    E, dg, db, back = qaoa.adjoint_gradient(n, C, gam, bet)
    s = scale_of(w)
    if dtype == "c128":
        tol = 1e-10 * s
        assert abs(out[0] - E) <= tol and abs(out[1] - 1.0) <= 1e-12
        assert np.max(np.abs(out[2:2 + p] - dg)) <= tol
        assert np.max(np.abs(out[2 + p:] - db)) <= tol
        assert np.linalg.norm(state_np(psi) - qaoa.plus_state(n)) <= 1e-11
    else:
        # 1e-4 relative to each value (absolute below 1)
        assert abs(out[0] - E) <= 1e-4 * max(1.0, abs(E))
        assert np.all(np.abs(out[2:2 + p] - dg) <= 1e-4 * np.maximum(1.0, np.abs(dg)))
        assert np.all(np.abs(out[2 + p:] - db) <= 1e-4 * np.maximum(1.0, np.abs(db)))


# ------------------------------------------------------------------ the small configuration end to end

def test_n10_gnp05_seed0_p2_config():
    """n = 10, G(10, 0.5) from seed 0, unweighted, p = 2, complex128: C, <C>, 4096 samples."""
    n, p = 10, 2
    e = synth.gnp_edges(n, 0.5, 0)
    g = q.Graph(n, e, None, True)
    gam, bet = synth.angles(p, 0)
    C = qaoa.cut_values(n, e)
    cv = q.cost_vector(g, "i32")
    assert np.array_equal(to_np(cv.C), C)
    psi = q.new_state(n, "c128")
    E = to_np(q.apply_layers(psi, cv, gam, bet, expect=True))[0]
    ref = qaoa.qaoa_state(n, C, gam, bet)
    assert abs(E - qaoa.expectation(ref, C)) <= 1e-10 * max(1, len(e))
    z, cz = q.sample(psi, cv, 4096, 0)
    zr, cr = qaoa.sample(ref, C, synth.sample_uniforms(0, 4096))
    assert np.mean(to_np(z).astype(np.int64) != zr.astype(np.int64)) <= 1e-5
    assert np.array_equal(to_np(cz), C[to_np(z).astype(np.int64)].astype(np.float64))
