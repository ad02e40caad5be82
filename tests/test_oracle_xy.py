"""Pins of the Hamming-weight-subspace XY-mixer oracle (``oracle/xy.py``) against
what the mathematics fixes: dense matrix exponentials of the Pauli-built
Hamiltonians, the combinatorial number system, a closed form for the Dicke
state, and the conservation laws of the mixer."""
from __future__ import annotations

import itertools
from math import comb

import numpy as np
import pytest
from scipy.linalg import expm

from oracle import qaoa as oq
from oracle import xy as ox

import synth

_I = np.eye(2, dtype=np.complex128)
_X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)


def pauli_on(n, ops):
    """Dense tensor product with ops[j] on qubit j (bit j of the index)."""
    out = np.ones((1, 1), dtype=np.complex128)
    for q in range(n - 1, -1, -1):
        out = np.kron(out, ops.get(q, _I))
    return out


def xy_term(n, a, b):
    return 0.5 * (pauli_on(n, {a: _X, b: _X}) + pauli_on(n, {a: _Y, b: _Y}))


def random_state(rng, n):
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    return v / np.linalg.norm(v)


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_pair_gate_is_the_exponential_of_the_xy_term(n):
    rng = np.random.default_rng(11 + n)
    psi = random_state(rng, n)
    for a, b in itertools.permutations(range(n), 2):
        beta = rng.uniform(-2, 2)
        want = expm(-1j * beta * xy_term(n, a, b)) @ psi
        got = ox.apply_pair_gate(psi, n, min(a, b), max(a, b), beta) if a < b else ox.apply_pair_gate(psi, n, a, b, beta)
        np.testing.assert_allclose(got, want, atol=1e-13)


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_ring_mixer_is_the_product_of_the_parity_set_exponentials(n):
    # the sets of the parity ring mixer, written out from the ring (j, j+1 mod n)
    pairs = [(j, (j + 1) % n) for j in range(n)] if n > 2 else [(0, 1)]
    even = [p for p in pairs if p[0] % 2 == 0 and p[0] < n - 1]
    odd = [p for p in pairs if p[0] % 2 == 1 and p[0] < n - 1]
    close = [p for p in pairs if p[0] == n - 1]
    sets = [even, odd + close] if n % 2 == 0 else [even, odd, close]
    rng = np.random.default_rng(5 + n)
    psi = random_state(rng, n)
    beta = 0.37
    want = psi
    for s in sets:
        if s:
            want = expm(-1j * beta * sum(xy_term(n, a, b) for a, b in s)) @ want
    np.testing.assert_allclose(ox.apply_xy_mixer(psi, n, beta), want, atol=1e-12)
    # every ring pair appears exactly once
    got_pairs = sorted(tuple(sorted(p)) for s in ox.ring_pair_sets(n) for p in s)
    assert got_pairs == sorted({tuple(sorted(p)) for p in pairs})


@pytest.mark.parametrize("n", [1, 2, 5, 8])
def test_rank_order_is_the_combinatorial_number_system(n):
    for k in range(n + 1):
        fk = ox.feasible_states(n, k)
        assert len(fk) == comb(n, k) == ox.subspace_dim(n, k)
        for r, z in enumerate(fk):
            bits = [j for j in range(n) if (int(z) >> j) & 1]
            assert sum(comb(c, i + 1) for i, c in enumerate(bits)) == r
        subsets = sorted(sum(1 << j for j in c) for c in itertools.combinations(range(n), k))
        assert list(fk) == subsets
        assert [ox.state_of_rank(n, k, r) for r in range(len(fk))] == subsets


@pytest.mark.parametrize("n,k", [(4, 2), (5, 2), (6, 3), (7, 1)])
def test_mixer_keeps_the_hamming_weight_and_the_norm(n, k):
    rng = np.random.default_rng(n * 10 + k)
    fk = ox.feasible_states(n, k)
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[fk] = rng.standard_normal(len(fk)) + 1j * rng.standard_normal(len(fk))
    psi /= np.linalg.norm(psi)
    out = ox.apply_xy_mixer(psi, n, 0.81)
    outside = np.ones(1 << n, dtype=bool)
    outside[fk] = False
    assert np.all(out[outside] == 0)
    assert abs(np.linalg.norm(out) - 1) < 1e-14


@pytest.mark.parametrize("n,k", [(4, 2), (6, 3), (7, 2), (9, 4)])
def test_dicke_expectation_closed_form(n, k):
    # every edge is cut by a fraction 2 k (n - k) / (n (n - 1)) of F_k
    rng = np.random.default_rng(n + 100 * k)
    edges = [(u, v) for u in range(n) for v in range(u + 1, n) if rng.random() < 0.6]
    w = rng.integers(1, 10, len(edges)).astype(np.float64)
    C = oq.cut_values(n, edges, w)
    E, nrm = ox.xy_expectation(ox.restrict(ox.dicke_state(n, k), n, k), ox.subspace_costs(C, n, k))
    assert abs(nrm - 1) < 1e-14
    assert abs(E - w.sum() * 2 * k * (n - k) / (n * (n - 1))) < 1e-12


@pytest.mark.parametrize("n,k", [(4, 2), (5, 3)])
def test_layers_match_dense_exponentials(n, k):
    rng = np.random.default_rng(3 * n + k)
    edges = [(u, v) for u in range(n) for v in range(u + 1, n) if rng.random() < 0.7]
    w = rng.uniform(0.2, 1.5, len(edges))
    C = oq.cut_values(n, edges, w, integer=False)
    gammas, betas = rng.uniform(-1, 1, 3), rng.uniform(-1, 1, 3)
    psi = ox.dicke_state(n, k)
    HC = np.diag(C.astype(np.complex128))
    for g, b in zip(gammas, betas):
        psi = expm(-1j * g * HC) @ psi
        for s in ox.ring_pair_sets(n):
            psi = expm(-1j * b * sum(xy_term(n, a, c) for a, c in s)) @ psi
    np.testing.assert_allclose(ox.xy_state(n, k, C, gammas, betas), psi, atol=1e-12)


@pytest.mark.parametrize("n", [3, 6])
def test_extreme_weights_are_one_dimensional_and_fixed(n):
    C = oq.cut_values(n, [(0, 1), (1, 2)], [2.0, 3.0])
    for k in (0, n):
        assert ox.subspace_dim(n, k) == 1
        out = ox.restrict(ox.xy_state(n, k, C, [0.4, -0.2], [0.9, 1.3]), n, k)
        assert out.shape == (1,) and abs(abs(out[0]) - 1) < 1e-15
        assert ox.xy_expectation(out, ox.subspace_costs(C, n, k))[0] == 0.0


def test_phase_only_layer_keeps_the_expectation():
    n, k = 6, 3
    C = oq.cut_values(n, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (5, 0), (0, 3)])
    psi = ox.xy_state(n, k, C, [0.3, 0.7], [0.2, 0.0])
    before = ox.xy_state(n, k, C, [0.3], [0.2])
    Cs = ox.subspace_costs(C, n, k)
    e1 = ox.xy_expectation(ox.restrict(psi, n, k), Cs)[0]
    e0 = ox.xy_expectation(ox.restrict(before, n, k), Cs)[0]
    assert abs(e1 - e0) < 1e-13


@pytest.mark.parametrize("n,k", [(2, 1), (5, 2), (8, 4), (9, 1)])
def test_moved_amplitudes_per_pair_gate(n, k):
    # the algorithmic bytes of a pair-gate pass count the states of F_k with z_a != z_b:
    # 2 binom(n - 2, k - 1) for every pair, the states the gate actually changes
    fk = ox.feasible_states(n, k)
    rng = np.random.default_rng(n + k)
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[fk] = rng.standard_normal(len(fk)) + 1j * rng.standard_normal(len(fk))
    for s in ox.ring_pair_sets(n):
        for a, b in s:
            moved = np.count_nonzero(ox.apply_pair_gate(psi, n, a, b, 0.7) != psi)
            assert moved == 2 * comb(n - 2, k - 1)


@pytest.mark.parametrize("n,k", [(4, 2), (5, 2), (6, 3), (7, 3)])
def test_adjoint_gradient_matches_central_differences(n, k):
    rng = np.random.default_rng(17 * n + k)
    edges = [(u, v) for u in range(n) for v in range(u + 1, n) if rng.random() < 0.6]
    w = rng.uniform(0.2, 1.5, len(edges))
    C = oq.cut_values(n, edges, w, integer=False)
    p = 3
    gammas, betas = rng.uniform(-1, 1, p), rng.uniform(-1, 1, p)

    def energy(g, b):
        psi = ox.xy_state(n, k, C, g, b)
        return float(np.real(np.vdot(psi, C * psi)))

    E, dg, db = ox.xy_adjoint_gradient(n, k, C, gammas, betas)
    assert abs(E - energy(gammas, betas)) < 1e-12
    h = 1e-6
    for l in range(p):
        e = np.zeros(p)
        e[l] = h
        fd_g = (energy(gammas + e, betas) - energy(gammas - e, betas)) / (2 * h)
        fd_b = (energy(gammas, betas + e) - energy(gammas, betas - e)) / (2 * h)
        assert abs(dg[l] - fd_g) < 1e-7 * max(1.0, abs(fd_g))
        assert abs(db[l] - fd_b) < 1e-7 * max(1.0, abs(fd_b))


def test_adjoint_gradient_vanishes_where_the_mixer_cannot_act():
    # k = 0: a one-dimensional subspace, E = 0 and every derivative is 0
    n = 5
    C = oq.cut_values(n, [(0, 1), (1, 2), (2, 4)], [1.0, 2.0, 3.0])
    E, dg, db = ox.xy_adjoint_gradient(n, 0, C, [0.3, 0.5], [0.2, -0.4])
    assert E == 0.0 and np.all(dg == 0) and np.all(db == 0)


@pytest.mark.parametrize("n,k", [(1, 0), (1, 1), (4, 2), (7, 3), (10, 5), (12, 4)])
def test_subspace_sampling_equals_full_space_sampling(n, k):
    """Rank order is increasing z, so sampling the subspace vector must give exactly the
    full-space sampler's bitstrings for the same state embedded in 2**n amplitudes."""
    rng = np.random.default_rng(31 * n + k)
    edges = [(u, v) for u in range(n) for v in range(u + 1, n) if rng.random() < 0.5]
    w = rng.integers(1, 11, len(edges)).astype(np.float64)
    C = oq.cut_values(n, edges, w) if edges else np.zeros(1 << n, dtype=np.int64)
    psi = ox.xy_state(n, k, C, rng.uniform(0, 1, 2), rng.uniform(0, 1, 2))
    u = synth.sample_uniforms(5 + n, 5000)
    z_full, c_full = oq.sample(psi, C, u)
    z_sub, c_sub = ox.xy_sample(ox.restrict(psi, n, k), n, k, ox.subspace_costs(C, n, k), u)
    assert np.array_equal(z_full, z_sub) and np.array_equal(c_full, c_sub)
    assert all(bin(int(z)).count("1") == k for z in z_sub[:200])


def test_subspace_sampling_chi_square():
    n, k = 10, 4
    rng = np.random.default_rng(3)
    psi = rng.normal(size=comb(n, k)) + 1j * rng.normal(size=comb(n, k))
    psi /= np.linalg.norm(psi)
    shots = 100000
    z, _ = ox.xy_sample(psi, n, k, np.zeros(comb(n, k)), synth.sample_uniforms(9, shots))
    states = ox.feasible_states(n, k)
    idx = np.searchsorted(states, z.astype(np.int64))
    assert np.array_equal(states[idx], z.astype(np.int64))
    obs = np.bincount(idx, minlength=len(states))
    prob = np.abs(psi) ** 2
    chi2 = np.sum((obs - shots * prob) ** 2 / (shots * prob))
    dof = len(states) - 1
    assert chi2 < dof + 6 * np.sqrt(2 * dof)
