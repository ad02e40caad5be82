"""General PUBO cost vectors (Eq. 3) on the device against the oracle, and QAOA runs on
a higher-degree objective.

Integer weights are bit-exact.  Float weights: the device quantises every weight to one
common fixed point 2^-s with sum|w| + 1 < 2^(62 - s) and rounds once per 2048 terms, the
oracle sums in float64 term by term; both are within (T + 2) 2^-52 (sum|w| + 1) of the
exact sum for T terms, which is the tolerance.
"""
import numpy as np
import pytest

import synth
from oracle import qaoa

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2407_13012_gb300 as q  # noqa: E402


def random_terms(n, nterms, seed, integer=True, maxdeg=4):
    u = synth.uniforms(seed, "weights", 6 * nterms).reshape(nterms, 6)
    terms = []
    for r in u:
        deg = int(r[0] * (maxdeg + 1))
        vars_ = sorted({int(x * n) for x in r[1:1 + deg]})
        wk = float(int(r[5] * 11) - 5) if integer else 2.0 * r[5] - 1.0
        terms.append((wk, vars_))
    return terms


def masks_of(terms):
    return np.array([sum(1 << i for i in t) for _, t in terms], dtype=np.uint32), \
        np.array([w for w, _ in terms], dtype=np.float64)


@pytest.mark.parametrize("n", [1, 5, 9, 13, 17])
@pytest.mark.parametrize("cdt", ["i32", "f64"])
def test_pubo_integer_bit_exact(n, cdt):
    terms = random_terms(n, 40, 3 * n)
    m, w = masks_of(terms)
    cv = q.cost_vector_pubo(n, m, w, integer=True, dtype=cdt)
    ref = qaoa.pubo_values(n, terms, integer=True)
    got = cv.C.cpu().numpy()
    assert np.array_equal(got.astype(np.int64) if cdt == "i32" else got, ref if cdt == "i32" else ref.astype(float))
    assert cv.cmin <= ref.min() and ref.max() <= cv.cmax


def test_pubo_many_chunks_and_constant_terms():
    n = 10
    terms = random_terms(n, 5000, 17) + [(7.0, []), (-2.0, [])]
    m, w = masks_of(terms)
    cv = q.cost_vector_pubo(n, m, w, integer=True)
    assert np.array_equal(cv.C.cpu().numpy().astype(np.int64), qaoa.pubo_values(n, terms, integer=True))
    empty = q.cost_vector_pubo(n, np.zeros(0), np.zeros(0), integer=True)
    assert np.all(empty.C.cpu().numpy() == 0)


@pytest.mark.parametrize("nterms", [30, 4500])
def test_pubo_float_weights(nterms):
    n = 11
    terms = random_terms(n, nterms, 5, integer=False)
    m, w = masks_of(terms)
    cv = q.cost_vector_pubo(n, m, w, integer=False, dtype="f64")
    ref = qaoa.pubo_values(n, terms, integer=False)
    tol = (nterms + 2) * 2.0 ** -52 * (np.sum(np.abs(w)) + 1.0)
    assert np.max(np.abs(cv.C.cpu().numpy() - ref)) <= tol


def test_maxcut_as_pubo_equals_cut_vector():
    for seed in range(3):
        e, w, _ = synth.graph("gnp", 14, seed, weights="int", prob=0.4)
        m, wt = masks_of(qaoa.maxcut_pubo_terms(e, w))
        a = q.cost_vector_pubo(14, m, wt, integer=True).C.cpu().numpy()
        b = q.cost_vector(q.Graph(14, e, w, True), "i32").C.cpu().numpy()
        assert np.array_equal(a, b)


def test_pubo_sampled_at_n24():
    n = 24
    terms = random_terms(n, 60, 99)
    m, w = masks_of(terms)
    C = q.cost_vector_pubo(n, m, w, integer=True).C
    z = synth.draws_u64(5, "state", 4096) & np.uint64((1 << n) - 1)
    got = C[torch.as_tensor(z.astype(np.int64), device=C.device)].cpu().numpy()
    for zi, ci in zip(z.tolist(), got.tolist()):
        assert ci == sum(int(wk) for wk, t in terms if all((zi >> i) & 1 for i in t))


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_qaoa_on_degree3_objective(dtype):
    """Layers, <C>, gradient and sampling on a cubic objective: the downstream path takes a
    PUBO cost vector like a MaxCut one."""
    n, p = 10, 2
    terms = random_terms(n, 30, 4, maxdeg=3)
    m, w = masks_of(terms)
    cv = q.cost_vector_pubo(n, m, w, integer=True)
    C = qaoa.pubo_values(n, terms, integer=True)
    gam, bet = synth.angles(p, 12)
    s = max(1.0, float(np.sum(np.abs(w))))
    psi = q.new_state(n, dtype)
    E = q.apply_layers(psi, cv, gam, bet, expect=True).cpu().numpy()
    ref = qaoa.qaoa_state(n, C, gam, bet)
    tol = 1e-10 * s if dtype == "c128" else 1e-4 * s
    assert abs(E[0] - qaoa.expectation(ref, C)) <= tol
    lam = q.new_state(n, dtype)
    out = q.gradient(psi, lam, cv, gam, bet).cpu().numpy()
    E0, dg, db, _ = qaoa.adjoint_gradient(n, C, gam, bet)
    assert abs(out[0] - E0) <= tol
    assert np.max(np.abs(out[2:] - np.concatenate([dg, db]))) <= tol
    if dtype == "c128":
        psi2 = torch.as_tensor(ref, device="cuda")
        zs, cz = q.sample(psi2, cv, 2000, 3)
        zr, cr = qaoa.sample(ref, C, synth.sample_uniforms(3, 2000))
        assert np.mean(zs.cpu().numpy() != zr) <= 1e-3
        assert np.array_equal(cz.cpu().numpy(), C[zs.cpu().numpy()].astype(float))
