"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each check is chosen so that a plausible mistake in the oracle (a dropped term,
a wrong sign, a transposed operand, a wrong bit order) fails at least one of
them; ``test_pins_detect_planted_*`` plant such mistakes in the oracle on the
CPU and show that the pins catch them.
"""
import math
from pathlib import Path

import numpy as np
import pytest

import synth
from oracle import closed_form, dense, qaoa

GOLDEN = Path(__file__).parent / "golden"


def load_known_maxcuts():
    rows = []
    for line in (GOLDEN / "known_maxcuts.txt").read_text().splitlines():
        if not line.strip() or line.startswith("#"):
            continue
        name, n, val, edges = [x.strip() for x in line.split("|")]
        e = [tuple(map(int, p.split("-"))) for p in edges.split()] if edges else []
        rows.append((name, int(n), int(val), np.array(e, dtype=np.int64).reshape(-1, 2)))
    return rows


# ------------------------------------------------------------------ cut values

@pytest.mark.parametrize("name,n,val,edges", load_known_maxcuts())
def test_known_max_cuts(name, n, val, edges):
    C = qaoa.cut_values(n, edges)
    assert C.max() == val, name


def test_cut_values_match_pubo_eq3_integer():
    for seed in range(4):
        e, w, _ = synth.graph("gnp", 9, seed, weights="int", prob=0.5, lo=-3, hi=7)
        C = qaoa.cut_values(9, e, w, integer=True)
        F = qaoa.pubo_values(9, qaoa.maxcut_pubo_terms(e, w), integer=True)
        assert np.array_equal(C, F)


def test_cut_values_invariants():
    for seed in range(3):
        n = 10
        e, w, _ = synth.graph("gnp", n, seed, weights="int", prob=0.4)
        C = qaoa.cut_values(n, e, w)
        mask = (1 << n) - 1
        z = np.arange(1 << n)
        assert np.array_equal(C, C[z ^ mask])                    # complement symmetry
        assert C.sum() == int(w.sum()) * (1 << (n - 1))          # each edge cut in half the states
        assert C[0] == 0 and C.min() == 0


def test_cut_values_bit_order():
    # one edge (0, 2) of weight 5 on 3 qubits: cut exactly when bit 0 != bit 2
    C = qaoa.cut_values(3, [[0, 2]], [5.0])
    assert list(C) == [0, 5, 0, 5, 5, 0, 5, 0]


def test_float_cut_values_exact_on_dyadic_weights():
    n = 8
    e, w, _ = synth.graph("gnp", n, 7, weights="int", prob=0.6)
    Ci = qaoa.cut_values(n, e, w, integer=True)
    Cf = qaoa.cut_values(n, e, w / 4.0, integer=False)
    assert np.array_equal(Cf * 4.0, Ci.astype(np.float64))


def test_pubo_literal_reading_differs():
    # Eq. 3 read as "x subset of mask" would count terms when the bits are 0; the
    # reading (x AND mask) == mask is the one that reproduces the cut.
    e = np.array([[0, 1]])
    terms = qaoa.maxcut_pubo_terms(e, [1.0])
    F = qaoa.pubo_values(2, terms)
    assert list(F) == [0, 1, 1, 0]


def random_pubo_terms(n, nterms, seed, integer=True):
    """Terms of degree 0..4 over n variables with weights in {-5..5} (or U(-1, 1))."""
    u = synth.uniforms(seed, "weights", 6 * nterms).reshape(nterms, 6)
    terms = []
    for r in u:
        deg = int(r[0] * 5)
        vars_ = sorted({int(x * n) for x in r[1:1 + deg]})
        wk = float(int(r[5] * 11) - 5) if integer else 2.0 * r[5] - 1.0
        terms.append((wk, vars_))
    return terms


def test_pubo_closed_forms_higher_degree():
    """Eq. 3 with terms of degree up to 4: a term of degree d is 1 on exactly 2^(n-d) of
    the 2^n assignments, so sum_z f = sum_t w_t 2^(n - d_t); f(all ones) = sum_t w_t;
    f(0) = the constant terms; and a single monomial is 1 exactly on the supersets of
    its variable set."""
    n = 9
    for seed in range(4):
        terms = random_pubo_terms(n, 25, seed)
        F = qaoa.pubo_values(n, terms, integer=True)
        assert F.sum() == sum(int(w) * 2 ** (n - len(t)) for w, t in terms)
        assert F[(1 << n) - 1] == sum(int(w) for w, _ in terms)
        assert F[0] == sum(int(w) for w, t in terms if not t)
    F = qaoa.pubo_values(5, [(3.0, [1, 3, 4])], integer=True)
    z = np.arange(32)
    want = np.where(((z >> 1) & 1) & ((z >> 3) & 1) & ((z >> 4) & 1), 3, 0)
    assert np.array_equal(F, want)


# ------------------------------------------------------------------ states

def small_instances():
    out = []
    for seed in range(3):
        for fam, kind in (("gnp", "int"), ("gnp", "u01"), ("complete", "unit")):
            n = 4 + seed
            e, w, integer = synth.graph(fam, n, seed, weights=kind, prob=0.6)
            out.append((n, e, w, integer, seed))
    return out


@pytest.mark.parametrize("n,e,w,integer,seed", small_instances())
def test_state_matches_dense_expm(n, e, w, integer, seed):
    C = qaoa.cut_values(n, e, w, integer=integer)
    for p in (1, 2, 3):
        g, b = synth.angles(p, seed * 10 + p)
        psi = qaoa.qaoa_state(n, C, g, b)
        ref = dense.dense_state(n, C, g, b)
        assert np.max(np.abs(psi - ref)) < 1e-12


def test_mixer_sign_identity():
    n = 6
    e, w, integer = synth.graph("gnp", n, 3, weights="u01", prob=0.5)
    C = qaoa.cut_values(n, e, w, integer=False)
    g, b = synth.angles(3, 11)
    paper = qaoa.expectation(qaoa.qaoa_state(n, C, g, b, mixer_sign=-1), C)
    ours_negb = qaoa.expectation(qaoa.qaoa_state(n, C, g, -b), C)
    ours_negg = qaoa.expectation(qaoa.qaoa_state(n, C, -g, b), C)
    assert abs(paper - ours_negb) < 1e-13
    assert abs(paper - ours_negg) < 1e-12
    assert abs(paper - dense.dense_expectation(n, C, g, b, mixer_sign=-1)) < 1e-12


def test_norm_and_uniform_identities():
    e, w, _ = synth.graph("reg3", 10, 2, weights="int")
    n = 10
    C = qaoa.cut_values(n, e, w)
    W = float(w.sum())
    g, b = synth.angles(4, 5)
    psi = qaoa.plus_state(n)
    for l in range(4):
        psi = qaoa.apply_rx_all(qaoa.apply_cost_unitary(psi, C, g[l]), n, b[l])
        assert abs(qaoa.norm2(psi) - 1.0) < 1e-12
    assert abs(qaoa.expectation(qaoa.plus_state(n), C) - W / 2) < 1e-12
    assert abs(qaoa.expectation(qaoa.qaoa_state(n, C, [0.0] * 3, b[:3]), C) - W / 2) < 1e-11
    assert abs(qaoa.expectation(qaoa.qaoa_state(n, C, g[:3], [0.0] * 3), C) - W / 2) < 1e-11


def test_flip_symmetry_and_quarter_turn():
    n = 8
    e, w, integer = synth.graph("gnp", n, 4, weights="u01", prob=0.5)
    C = qaoa.cut_values(n, e, w, integer=False)
    g, b = synth.angles(3, 9)
    psi = qaoa.qaoa_state(n, C, g, b)
    z = np.arange(1 << n)
    assert np.max(np.abs(psi - psi[z ^ ((1 << n) - 1)])) < 1e-13
    E = qaoa.expectation(psi, C)
    b2 = b.copy()
    b2[1] += np.pi / 2  # RX(pi) on every qubit = (-i)^n X^n commutes with C up to the flip symmetry
    assert abs(qaoa.expectation(qaoa.qaoa_state(n, C, g, b2), C) - E) < 1e-12


def test_p1_closed_form_against_dense():
    for seed in range(4):
        n = 5 + (seed % 2)
        e, w, integer = synth.graph("gnp", n, seed, weights="u01" if seed % 2 else "int", prob=0.6)
        C = qaoa.cut_values(n, e, w, integer=integer)
        g, b = synth.angles(1, seed)
        ref = dense.dense_expectation(n, C, g, b)
        assert abs(closed_form.expectation_p1(n, e, w, g[0], b[0]) - ref) < 1e-12


def test_p1_closed_form_against_state_at_n14():
    for fam, kind in (("reg3", "u01"), ("gnp", "int")):
        n = 14
        e, w, integer = synth.graph(fam, n, 1, weights=kind, prob=0.3)
        C = qaoa.cut_values(n, e, w, integer=integer)
        g, b = synth.angles(1, 21)
        E = qaoa.expectation(qaoa.qaoa_state(n, C, g, b), C)
        assert abs(closed_form.expectation_p1(n, e, w, g[0], b[0]) - E) < 1e-11


def test_dense_operators():
    n = 3
    B = dense.b_matrix(n)
    ev = np.sort(np.linalg.eigvalsh(B))
    assert np.allclose(ev, np.sort([n - 2 * bin(z).count("1") for z in range(8)]))
    # X on qubit 1 flips bit 1 of the index
    X1 = dense.x_on(n, 1)
    for z in range(8):
        assert X1[z ^ 2, z] == 1


# ------------------------------------------------------------------ sampling

def test_sample_basis_and_uniform_states():
    n = 6
    C = qaoa.cut_values(n, [[0, 1], [2, 5]], [1.0, 2.0])
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[37] = 1j
    u = synth.sample_uniforms(3, 500)
    z, c = qaoa.sample(psi, C, u)
    assert np.all(z == 37) and np.all(c == C[37])
    z, c = qaoa.sample(qaoa.plus_state(n), C, u)
    assert np.array_equal(z.astype(np.int64), np.floor(u * 64).astype(np.int64))
    assert np.array_equal(c, C[z.astype(np.int64)])


def test_sample_edge_uniforms():
    # probabilities 1/4 at z = 1, 3, 4, 6 (exact in binary): P = [0, .25, .25, .5, .75, .75, 1, 1]
    psi = np.zeros(8, dtype=np.complex128)
    psi[[1, 3, 4, 6]] = [0.5, 0.5j, -0.5, 0.5]
    C = np.arange(8.0)
    z, _ = qaoa.sample(psi, C, np.array([0.0, 0.2499, 0.25, 0.5, 0.75, 1.0 - 2 ** -53]))
    assert list(z) == [1, 1, 3, 4, 6, 6]


def test_sample_chi_square():
    n = 8
    e, w, integer = synth.graph("gnp", n, 2, weights="int", prob=0.5)
    C = qaoa.cut_values(n, e, w)
    psi = qaoa.qaoa_state(n, C, *synth.angles(2, 4))
    shots = 200000
    z, c = qaoa.sample(psi, C, synth.sample_uniforms(7, shots))
    vals = np.unique(C)
    prob = np.array([np.sum(np.abs(psi[C == v]) ** 2) for v in vals])
    obs = np.array([np.sum(c == v) for v in vals])
    keep = prob * shots > 5
    chi2 = np.sum((obs[keep] - shots * prob[keep]) ** 2 / (shots * prob[keep]))
    dof = keep.sum() - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof)


# ------------------------------------------------------------------ gradient

def test_adjoint_matches_finite_differences():
    n = 8
    e, w, integer = synth.graph("gnp", n, 5, weights="u01", prob=0.5)
    C = qaoa.cut_values(n, e, w, integer=False)
    g, b = synth.angles(3, 13)
    E, dg, db, psi_back = qaoa.adjoint_gradient(n, C, g, b)
    fg, fb = qaoa.finite_difference_gradient(n, C, g, b, h=1e-6)
    scale = max(1.0, float(np.sum(np.abs(w))))
    assert np.max(np.abs(dg - fg)) < 1e-7 * scale
    assert np.max(np.abs(db - fb)) < 1e-7 * scale
    assert abs(E - qaoa.expectation(qaoa.qaoa_state(n, C, g, b), C)) < 1e-12
    assert np.linalg.norm(psi_back - qaoa.plus_state(n)) < 1e-12


def test_adjoint_p1_matches_closed_form_derivative():
    n = 10
    e, w, integer = synth.graph("reg3", n, 3, weights="int")
    C = qaoa.cut_values(n, e, w)
    g, b = synth.angles(1, 2)
    _, dg, db, _ = qaoa.adjoint_gradient(n, C, g, b)
    cg, cb = closed_form.gradient_p1(n, e, w, g[0], b[0], h=1e-5)
    assert abs(dg[0] - cg) < 1e-6 and abs(db[0] - cb) < 1e-6


@pytest.mark.parametrize("n,fam,kind,seed", [(3, "gnp", "u01", 1), (4, "gnp", "int", 2), (5, "gnp", "u01", 3),
                                          (6, "reg3", "int", 4), (6, "gnp", "u01", 5), (6, "complete", "unit", 6)])
def test_dense_gradient_against_finite_differences(n, fam, kind, seed):
    """The dense forward-mode derivative equals central differences of the dense expm state."""
    e, w, integer = synth.graph(fam, n, seed, weights=kind, prob=0.6)
    C = qaoa.cut_values(n, e, w, integer=integer)
    g, b = synth.angles(2, seed)
    dg, db = dense.dense_gradient(n, C, g, b)
    h = 1e-6
    for l in range(2):
        d = np.zeros(2)
        d[l] = h
        fg = (dense.dense_expectation(n, C, g + d, b) - dense.dense_expectation(n, C, g - d, b)) / (2 * h)
        fb = (dense.dense_expectation(n, C, g, b + d) - dense.dense_expectation(n, C, g, b - d)) / (2 * h)
        scale = max(1.0, float(np.sum(np.abs(w))))
        assert abs(dg[l] - fg) < 1e-7 * scale and abs(db[l] - fb) < 1e-7 * scale


@pytest.mark.parametrize("n,fam,kind,seed", [(2, "gnp", "int", 0), (4, "gnp", "u01", 1), (5, "gnp", "int", 2),
                                          (6, "reg3", "int", 3), (6, "gnp", "u01", 4), (6, "complete", "unit", 5)])
def test_p1_gradient_closed_form_against_dense(n, fam, kind, seed):
    """The analytic derivative of the p = 1 closed form equals the dense expm derivative."""
    e, w, integer = synth.graph(fam, n, seed, weights=kind, prob=0.7)
    C = qaoa.cut_values(n, e, w, integer=integer)
    scale = max(1.0, float(np.sum(np.abs(w))))
    for s in range(4):
        g, b = synth.angles(1, 10 * seed + s)
        dg, db = dense.dense_gradient(n, C, g, b)
        cg, cb = closed_form.gradient_p1_exact(n, e, w, g[0], b[0])
        assert abs(dg[0] - cg) < 1e-12 * scale and abs(db[0] - cb) < 1e-12 * scale


@pytest.mark.parametrize("n,fam,kind", [(12, "reg3", "int"), (13, "gnp", "u01")])
def test_p1_gradient_closed_form_against_adjoint(n, fam, kind):
    e, w, integer = synth.graph(fam, n, 7, weights=kind, prob=0.3)
    C = qaoa.cut_values(n, e, w, integer=integer)
    g, b = synth.angles(1, 9)
    _, dg, db, _ = qaoa.adjoint_gradient(n, C, g, b)
    cg, cb = closed_form.gradient_p1_exact(n, e, w, g[0], b[0])
    scale = max(1.0, float(np.sum(np.abs(w))))
    assert abs(dg[0] - cg) < 1e-11 * scale and abs(db[0] - cb) < 1e-11 * scale


def test_linear_ramp():
    g, b = qaoa.linear_ramp(4)
    assert np.allclose(g, [0.25, 0.5, 0.75, 1.0]) and np.allclose(b, [0.75, 0.5, 0.25, 0.0])


# ------------------------------------------------------------------ planted mistakes

def test_pins_detect_planted_mixer_sign(monkeypatch):
    n = 5
    e, w, integer = synth.graph("gnp", n, 1, weights="u01", prob=0.7)
    C = qaoa.cut_values(n, e, w, integer=False)
    g, b = synth.angles(2, 3)
    bad = qaoa.qaoa_state(n, C, g, b, mixer_sign=-1)
    assert np.max(np.abs(bad - dense.dense_state(n, C, g, b))) > 1e-3


def test_pins_detect_planted_dropped_edge():
    name, n, val, edges = load_known_maxcuts()[-2]  # Petersen
    C = qaoa.cut_values(n, edges[:-1])
    assert C.sum() != len(edges) * (1 << (n - 1))


def test_pins_detect_planted_transposed_butterfly(monkeypatch):
    # a wrong operand in the butterfly: a -> cos a - i sin a (should be - i sin b).
    # (Swapping a and b in both outputs is X RX, which a flip-symmetric MaxCut
    # state cannot tell apart, so it is not a mistake the pins should catch.)
    def bad_rx(psi, n, beta, mixer_sign=1):
        c, s = np.cos(beta), np.sin(beta)
        out = psi.copy()
        for j in range(n):
            v = out.reshape(-1, 2, 1 << j)
            a, bb = v[:, 0, :].copy(), v[:, 1, :].copy()
            v[:, 0, :] = c * a - 1j * s * a
            v[:, 1, :] = c * bb - 1j * s * a
        return out
    monkeypatch.setattr(qaoa, "apply_rx_all", bad_rx)
    n = 5
    e, w, integer = synth.graph("gnp", n, 2, weights="int", prob=0.6)
    C = qaoa.cut_values(n, e, w)
    g, b = synth.angles(1, 1)
    assert np.max(np.abs(qaoa.qaoa_state(n, C, g, b) - dense.dense_state(n, C, g, b))) > 1e-3


def test_pins_detect_planted_gradient_sign(monkeypatch):
    n = 6
    e, w, integer = synth.graph("gnp", n, 4, weights="u01", prob=0.6)
    C = qaoa.cut_values(n, e, w, integer=False)
    g, b = synth.angles(2, 5)
    E, dg, db, _ = qaoa.adjoint_gradient(n, C, g, b)
    fg, fb = qaoa.finite_difference_gradient(n, C, g, b)
    # a real-part (instead of imaginary-part) gradient would not match
    assert np.max(np.abs(-dg - fg)) > 1e-3 or np.max(np.abs(-db - fb)) > 1e-3


def test_pins_detect_planted_p1_gradient_sign(monkeypatch):
    # a wrong sign in the derivative of the cosine products must fail the dense pin
    def bad(gamma, c):
        cs = np.cos(gamma * c)
        deriv = sum(c[j] * np.sin(gamma * c[j]) * np.prod(np.delete(cs, j)) for j in range(len(c)))
        return float(np.prod(cs)), float(deriv)
    monkeypatch.setattr(closed_form, "_cos_product_and_derivative", bad)
    n = 6
    e, w, integer = synth.graph("gnp", n, 4, weights="u01", prob=0.7)
    C = qaoa.cut_values(n, e, w, integer=False)
    g, b = synth.angles(1, 3)
    dg, _ = dense.dense_gradient(n, C, g, b)
    cg, _ = closed_form.gradient_p1_exact(n, e, w, g[0], b[0])
    assert abs(dg[0] - cg) > 1e-3
