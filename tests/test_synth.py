"""Seeded synthetic inputs: SplitMix64 reference values, determinism, graph families."""
import numpy as np
import pytest

import synth


def test_splitmix64_reference_outputs():
    # first three outputs of SplitMix64 from state 0 (published reference values)
    assert synth.mix64(1 * synth.GOLDEN) == 0xE220A8397B1DCDAF
    assert synth.mix64(2 * synth.GOLDEN) == 0x6E789E6AA1B965F4
    assert synth.mix64(3 * synth.GOLDEN) == 0x06C45D188009454F


def test_vectorised_draws_match_scalar():
    x = synth.draws_u64(12345, "sample", 20)
    st = synth.Stream(12345, "sample")
    assert [int(v) for v in x] == [st.next_u64() for _ in range(20)]
    u = synth.uniforms(9, "angles", 1000)
    assert u.min() >= 0.0 and u.max() < 1.0


def test_gnp_is_deterministic_and_simple():
    e1 = synth.gnp_edges(20, 0.3, 4)
    e2 = synth.gnp_edges(20, 0.3, 4)
    assert np.array_equal(e1, e2)
    assert np.all(e1[:, 0] < e1[:, 1])
    assert len({tuple(x) for x in e1}) == len(e1)
    m = np.mean([len(synth.gnp_edges(30, 0.2, s)) for s in range(20)])
    assert abs(m - 0.2 * 435) < 15


def test_regular3():
    for n in (4, 10, 24, 32):
        e = synth.regular3_edges(n, 1)
        deg = np.bincount(e.ravel(), minlength=n)
        assert np.all(deg == 3) and len(e) == 3 * n // 2
        assert len({tuple(x) for x in e}) == len(e) and np.all(e[:, 0] != e[:, 1])


def test_weights_and_angles():
    w = synth.edge_weights(1000, "int", 3, 1, 10)
    assert set(np.unique(w)) == set(range(1, 11))
    g, b = synth.angles(6, 2)
    assert len(g) == len(b) == 6 and np.all((g >= 0) & (g < np.pi))
    psi = synth.random_state(7, 1)
    assert abs(np.linalg.norm(psi) - 1) < 1e-14


def test_batch_instances_families_sizes_and_determinism():
    a = synth.batch_instances(200, 4, n_lo=8, n_hi=20, p=3)
    b = synth.batch_instances(200, 4, n_lo=8, n_hi=20, p=3)
    fams = {"reg3": 0, "gnp": 0}
    for (n, fam, e, w, gam, bet), y in zip(a, b):
        assert np.array_equal(e, y[2]) and np.array_equal(w, y[3]) and np.array_equal(gam, y[4])
        assert 8 <= n <= 20 and len(gam) == 3 and len(bet) == 3
        assert np.all((w >= 1) & (w <= 5)) and np.all(w == np.floor(w))
        assert np.all((0 <= e) & (e < n)) and np.all(e[:, 0] < e[:, 1])
        if fam == "reg3":
            assert n % 2 == 0 and np.all(np.bincount(e.ravel(), minlength=n) == 3)
        fams[fam] += 1
    assert 70 <= fams["reg3"] <= 130


def test_proposer_param_layout_round_trip():
    torch = pytest.importorskip("torch")
    from paper_2407_13012_gb300 import proposer
    import paper_2407_13012_gb300 as q
    for p in (1, 4):
        net = proposer.make_net(p)
        vec = proposer.pack(net)
        H = proposer.HIDDEN
        assert len(vec) == 3 * H + 3 * (2 * H * H + H) + 2 * H * H + H + 2 * p * H + 2 * p
        assert len(vec) == q.proposer_param_count(p)
        assert np.array_equal(proposer.pack(proposer.unpack(vec, p)), vec)
