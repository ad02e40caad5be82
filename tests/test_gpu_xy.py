"""Parity of the Hamming-weight-subspace QAOA with the ring XY mixer (CUDA path through
the C ABI) against the FP64 oracle ``oracle/xy.py``."""
from __future__ import annotations

from math import comb

import numpy as np
import pytest

from oracle import qaoa as oq
from oracle import xy as ox

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _q():
    import paper_2407_13012_gb300 as q
    return q


def random_graph(rng, n, prob, integer=True):
    edges = [(u, v) for u in range(n) for v in range(u + 1, n) if rng.random() < prob]
    if not edges and n >= 2:
        edges = [(0, n - 1)]
    w = rng.integers(1, 11, len(edges)).astype(np.float64) if integer else rng.uniform(0.05, 1.0, len(edges))
    return edges, w


def make(n, k, prob, seed, integer=True, cost_dtype="i32"):
    q = _q()
    rng = np.random.default_rng(seed)
    edges, w = random_graph(rng, n, prob, integer)
    g = q.Graph(n, np.array(edges, dtype=np.int32).reshape(-1, 2), w, integer=integer)
    cv = q.xy_cost_vector(g, k, cost_dtype if integer else "f64")
    C = oq.cut_values(n, edges, w, integer=integer) if edges else np.zeros(1 << n)
    return q, g, cv, C, rng


CASES = [(1, 0), (1, 1), (2, 1), (3, 1), (3, 2), (6, 3), (7, 3), (9, 4), (10, 2), (12, 6), (13, 5), (14, 7)]
# three mixer windows ([0, 8), [7, 16), [15, n)) with ragged edge classes
WIDE = [(17, 8), (18, 5), (18, 13)]


@pytest.mark.parametrize("n,k", CASES + [(16, 8), (12, 0), (12, 12), (15, 14)])
def test_xy_cost_vector_bit_exact(n, k):
    q, g, cv, C, _ = make(n, k, 0.5, seed=n * 41 + k)
    got = cv.C.cpu().numpy()
    assert got.shape == (comb(n, k),)
    assert np.array_equal(got.astype(np.int64), ox.subspace_costs(C, n, k).astype(np.int64))
    # float64 costs of the integer graph are the same integers
    cf = q.xy_cost_vector(g, k, "f64").C.cpu().numpy()
    assert np.array_equal(cf, got.astype(np.float64))


@pytest.mark.parametrize("n,k", [(9, 4), (13, 6)])
def test_xy_cost_vector_float_weights(n, k):
    q, g, cv, C, _ = make(n, k, 0.6, seed=7 * n + k, integer=False)
    got = cv.C.cpu().numpy()
    want = ox.subspace_costs(C, n, k)
    # one rounding of an exact fixed-point sum vs the oracle's edge-order float sum
    bound = (g.m + 1) * 2.0 ** -52 * max(1.0, float(np.abs(g.weights).sum()))
    assert np.max(np.abs(got - want)) <= bound


@pytest.mark.parametrize("scale", [1e-12, 1e-300, 1e12])
def test_xy_cost_vector_float_weights_any_scale(scale):
    """The common fixed point follows sum|w|, so tiny or huge weights keep their relative precision."""
    q = _q()
    n, k = 12, 6
    rng = np.random.default_rng(5)
    edges, w = random_graph(rng, n, 0.5, integer=False)
    w = w * scale
    g = q.Graph(n, np.array(edges, dtype=np.int32).reshape(-1, 2), w, integer=False)
    got = q.xy_cost_vector(g, k, "f64").C.cpu().numpy()
    want = ox.subspace_costs(oq.cut_values(n, edges, w, integer=False), n, k)
    bound = (g.m + 1) * 2.0 ** -52 * float(np.abs(w).sum())
    assert np.max(np.abs(got - want)) <= bound


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n,k", CASES + WIDE)
@pytest.mark.parametrize("integer", [True, False])
def test_xy_layers_match_oracle(n, k, dtype, integer):
    q, g, cv, C, rng = make(n, k, 0.5, seed=1000 + 37 * n + k + (0 if integer else 5), integer=integer)
    p = 3
    gammas, betas = rng.uniform(-1.2, 1.2, p), rng.uniform(-1.2, 1.2, p)
    psi = q.xy_new_state(n, k, dtype)
    out = q.xy_apply_layers(psi, n, k, cv, gammas, betas, init=True, expect=True).cpu().numpy()
    want = ox.restrict(ox.xy_state(n, k, C, gammas, betas), n, k)
    E, nrm = ox.xy_expectation(want, ox.subspace_costs(C, n, k))
    got = psi.cpu().numpy()
    if dtype == "c128":
        assert np.max(np.abs(got - want)) < 1e-12
        assert abs(out[0] - E) <= 1e-10 * max(1.0, abs(E))
        assert abs(out[1] - nrm) < 1e-12
    else:
        assert np.max(np.abs(got - want)) < 2e-5
        assert abs(out[0] - E) <= 1e-4 * max(1.0, abs(E))
        assert abs(out[1] - nrm) < 1e-5
    # the stand-alone expectation runs the same reduction
    again = q.xy_expectation(psi, n, k, cv).cpu().numpy()
    assert np.array_equal(again, out)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n,k", CASES + WIDE)
@pytest.mark.parametrize("integer", [True, False])
def test_xy_gradient_matches_oracle(n, k, dtype, integer):
    """The subspace adjoint gradient against oracle/xy.py's (one 2 Im <lambda|H_g|psi_g> term
    per gate, pinned to central differences); complex128 within 1e-10 max(1, sum|w|),
    complex64 within 1e-4 max(1, |value|) per entry."""
    q, g, cv, C, rng = make(n, k, 0.5, seed=2000 + 37 * n + k + (0 if integer else 5), integer=integer)
    p = 3
    gammas, betas = rng.uniform(-1.2, 1.2, p), rng.uniform(-1.2, 1.2, p)
    psi, lam = q.xy_new_state(n, k, dtype), q.xy_new_state(n, k, dtype)
    out = q.xy_gradient(psi, lam, n, k, cv, gammas, betas).cpu().numpy()
    E, dg, db = ox.xy_adjoint_gradient(n, k, C, gammas, betas)
    ref = np.concatenate([[E], dg, db])
    got = np.concatenate([out[:1], out[2:]])
    if dtype == "c128":
        scale = max(1.0, float(np.abs(g.weights).sum())) if g.m else 1.0
        assert np.max(np.abs(got - ref)) <= 1e-10 * scale
        assert abs(out[1] - 1.0) < 1e-12
        dicke = np.full(comb(n, k), 1.0 / np.sqrt(comb(n, k)))
        assert np.max(np.abs(psi.cpu().numpy() - dicke)) < 1e-12  # the pass undoes every gate
    else:
        assert np.all(np.abs(got - ref) <= 1e-4 * np.maximum(1.0, np.abs(ref)))
        assert abs(out[1] - 1.0) < 1e-5


def test_xy_gradient_at_bench_size_is_consistent():
    """n = 24, k = 12 (2.7e6 amplitudes): no full-space oracle, so the complex128 gradient
    is checked against the complex64 one and against the device's own central differences
    of <C> (h = 1e-5) for one angle of each kind."""
    q = _q()
    n, k = 24, 12
    rng = np.random.default_rng(7)
    edges = [(j, (j + 1) % n) for j in range(n)] + [(j, (j + n // 2) % n) for j in range(n // 2)]
    w = rng.integers(1, 11, len(edges)).astype(np.float64)
    g = q.Graph(n, np.array(edges, dtype=np.int32), w, integer=True)
    cv = q.xy_cost_vector(g, k, "i32")
    gammas, betas = rng.uniform(0, np.pi, 2), rng.uniform(0, np.pi, 2)
    psi, lam = q.xy_new_state(n, k, "c128"), q.xy_new_state(n, k, "c128")
    out = q.xy_gradient(psi, lam, n, k, cv, gammas, betas).cpu().numpy()
    p32, l32 = q.xy_new_state(n, k, "c64"), q.xy_new_state(n, k, "c64")
    out32 = q.xy_gradient(p32, l32, n, k, cv, gammas, betas).cpu().numpy()
    assert np.all(np.abs(out32 - out) <= 1e-4 * np.maximum(1.0, np.abs(out)))
    h = 1e-5

    def energy(gm, bt):
        st = q.xy_new_state(n, k, "c128")
        return q.xy_apply_layers(st, n, k, cv, gm, bt, init=True, expect=True).cpu().numpy()[0]

    fd_g = (energy(gammas + [h, 0], betas) - energy(gammas - [h, 0], betas)) / (2 * h)
    fd_b = (energy(gammas, betas + [0, h]) - energy(gammas, betas - [0, h])) / (2 * h)
    scale = float(w.sum())
    assert abs(out[2] - fd_g) <= 1e-6 * scale and abs(out[2 + 2 + 1] - fd_b) <= 1e-6 * scale


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n,k", CASES)
def test_xy_sample_matches_oracle(n, k, dtype):
    """Sampling on F_k (Sec. IV-D over the subspace) against oracle/xy.py's xy_sample under
    the same uniforms: mismatches only where a target lies within rounding of a CDF step
    (<= 1e-5 of the shots), every bitstring has k ones and its cost is C(z) exactly."""
    import synth
    q, g, cv, C, rng = make(n, k, 0.5, seed=3000 + 37 * n + k)
    gammas, betas = rng.uniform(-1.2, 1.2, 2), rng.uniform(-1.2, 1.2, 2)
    psi = q.xy_new_state(n, k, dtype)
    q.xy_apply_layers(psi, n, k, cv, gammas, betas)
    ref_in = psi.cpu().numpy().astype(np.complex128)  # exactly the values the sampler reads
    shots, seed = 20000, 77 + n
    z, cz = q.xy_sample(psi, n, k, cv, shots, seed)
    z, cz = z.cpu().numpy().astype(np.uint64), cz.cpu().numpy()
    zr, cr = ox.xy_sample(ref_in, n, k, ox.subspace_costs(C, n, k), synth.sample_uniforms(seed, shots))
    assert np.mean(z != zr) <= 1e-5
    assert all(bin(int(x)).count("1") == k for x in z[:2000])
    assert np.array_equal(cz, C[z.astype(np.int64)].astype(np.float64))


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_xy_sample_ragged_multichunk(dtype):
    """n = 26, k = 13: binom(26, 13) = 10,400,600 amplitudes, a ragged last leaf and three
    scan chunks (4096 leaves of 1024 each); mass in the last entries of the last leaf too."""
    import synth
    q = _q()
    n, k = 26, 13
    D = comb(n, k)
    rng = np.random.default_rng(11)
    edges, w = random_graph(rng, n, 0.15, integer=True)
    g = q.Graph(n, np.array(edges, dtype=np.int32).reshape(-1, 2), w, integer=True)
    cv = q.xy_cost_vector(g, k, "i32")
    Csub = cv.C.cpu().numpy().astype(np.int64)
    u = synth.uniforms(5, "state", 2 * D).reshape(-1, 2) - 0.5
    amp = u[:, 0] + 1j * u[:, 1]
    amp[-40:] *= 30.0  # weight on the ragged end
    amp /= np.linalg.norm(amp)
    tdt = torch.complex128 if dtype == "c128" else torch.complex64
    psi = torch.as_tensor(amp).to(tdt).cuda()
    ref_in = psi.cpu().numpy().astype(np.complex128)
    shots, seed = 100000, 123
    z, cz = q.xy_sample(psi, n, k, cv, shots, seed)
    z, cz = z.cpu().numpy().astype(np.uint64), cz.cpu().numpy()
    zr, cr = ox.xy_sample(ref_in, n, k, Csub, synth.sample_uniforms(seed, shots))
    assert np.mean(z != zr) <= 1e-5
    assert np.array_equal(cz, cr)
    states = ox.feasible_states(n, k)
    assert np.sum(z >= np.uint64(states[-40])) > 0  # the ragged end is reached
    del psi
    torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_xy_layers_continue_from_a_given_state(dtype):
    n, k = 11, 4
    q, g, cv, C, rng = make(n, k, 0.4, seed=99)
    gammas, betas = rng.uniform(-1, 1, 4), rng.uniform(-1, 1, 4)
    psi = q.xy_new_state(n, k, dtype)
    q.xy_apply_layers(psi, n, k, cv, gammas[:2], betas[:2], init=True)
    q.xy_apply_layers(psi, n, k, cv, gammas[2:], betas[2:], init=False)
    want = ox.restrict(ox.xy_state(n, k, C, gammas, betas), n, k)
    tol = 1e-12 if dtype == "c128" else 2e-5
    assert np.max(np.abs(psi.cpu().numpy() - want)) < tol


def test_xy_layers_with_wide_cost_range_use_direct_phases():
    # integer costs whose span exceeds the phase-table limit take exp(-i gamma C) directly
    n, k = 10, 5
    q = _q()
    rng = np.random.default_rng(5)
    edges = [(u, v) for u in range(n) for v in range(u + 1, n) if rng.random() < 0.5]
    w = rng.integers(1000, 5000, len(edges)).astype(np.float64)
    g = q.Graph(n, np.array(edges, dtype=np.int32), w, integer=True)
    cv = q.xy_cost_vector(g, k)
    assert cv.span == 0 or cv.span > q.MAX_TABLE_SPAN
    C = oq.cut_values(n, edges, w)
    gammas, betas = rng.uniform(-0.01, 0.01, 2), rng.uniform(-1, 1, 2)
    psi = q.xy_new_state(n, k, "c128")
    q.xy_apply_layers(psi, n, k, cv, gammas, betas)
    want = ox.restrict(ox.xy_state(n, k, C, gammas, betas), n, k)
    assert np.max(np.abs(psi.cpu().numpy() - want)) < 1e-12


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_xy_bench_size_invariants(dtype):
    """Balanced cut of a random 3-regular graph, n = 32, k = 16 (601,080,390 amplitudes):
    properties that hold at any size.  A phase-only evolution keeps the Dicke expectation
    W 2k(n-k) / (n(n-1)); every layer keeps the norm."""
    import synth
    q = _q()
    n, k = 32, 16
    edges, w, _ = synth.graph("reg3", n, seed=3, weights="int")
    g = q.Graph(n, edges, w, integer=True)
    cv = q.xy_cost_vector(g, k)
    assert cv.C.numel() == comb(n, k)
    W = float(np.sum(w))
    psi = q.xy_new_state(n, k, dtype)
    out = q.xy_apply_layers(psi, n, k, cv, [0.3, -0.7], [0.0, 0.0], expect=True).cpu().numpy()
    dicke = W * 2 * k * (n - k) / (n * (n - 1))
    tol = 1e-9 if dtype == "c128" else 1e-4
    assert abs(out[0] - dicke) <= tol * dicke and abs(out[1] - 1) <= tol
    out = q.xy_apply_layers(psi, n, k, cv, [0.2], [0.45], init=True, expect=True).cpu().numpy()
    assert abs(out[1] - 1) <= tol
    assert 0 < out[0] < W
    # sampled entries of the cost vector against the cut of their unranked state
    C = cv.C[:: 10_000_019].cpu().numpy()
    ranks = np.arange(0, comb(n, k), 10_000_019)
    for r, c in zip(ranks, C):
        z = ox.state_of_rank(n, k, int(r))
        assert bin(z).count("1") == k
        cut = sum(int(wi) for (u, v), wi in zip(edges, w) if ((z >> int(u)) ^ (z >> int(v))) & 1)
        assert cut == c
