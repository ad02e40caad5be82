"""Batched adjoint gradients (many small integer-weight graphs in one persistent launch)
against the oracle, per graph.

Tolerances as for every gradient: complex128 1e-10 max(1, sum|w|) on E and every
derivative, |norm - 1| <= 1e-12; complex64 1e-4 max(1, |value|) per entry.
"""
import numpy as np
import pytest

import synth
from oracle import qaoa

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2407_13012_gb300 as q  # noqa: E402


def scale_of(w):
    return max(1.0, float(np.sum(np.abs(w))))


def check_rows(out, insts, dtype, p, integer=True):
    for row, (n, fam, e, w, gam, bet) in zip(out, insts):
        C = qaoa.cut_values(n, e, w, integer=integer)
        E, dg, db, _ = qaoa.adjoint_gradient(n, C, gam, bet)
        s = scale_of(w)
        ref = np.concatenate([[E], dg, db])
        got = np.concatenate([row[:1], row[2:]])
        # complex128: 1e-10 max(1, sum|w|); complex64: 1e-4 relative to each value (absolute below 1)
        tol = 1e-10 * s if dtype == "c128" else 1e-4 * np.maximum(1.0, np.abs(ref))
        ctx = (n, fam, dtype)
        assert abs(row[1] - 1.0) <= (1e-12 if dtype == "c128" else 1e-5), ctx
        assert np.all(np.abs(got - ref) <= tol), ctx


def run(insts, dtype, tiles=None, integer=True):
    graphs = [q.Graph(n, e, w, integer) for (n, fam, e, w, gam, bet) in insts]
    ang = np.stack([np.concatenate([gam, bet]) for (*_, gam, bet) in insts])
    return q.batch_gradient(graphs, ang, dtype, tiles=tiles).cpu().numpy()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("tile", [None, 0, 1])
def test_batch_small_graphs_vs_oracle(dtype, tile):
    """48 graphs with n = 4..14 (both families, weights 1..5, p = 3), each tile size."""
    p = 3
    insts = synth.batch_instances(48, 11, n_lo=4, n_hi=14, p=p)
    tiles = None if tile is None else np.full(q.MAX_N + 1, tile)
    check_rows(run(insts, dtype, tiles), insts, dtype, p)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_batch_large_graphs_vs_oracle(dtype):
    """Graphs that need two and three tile groups (n = 16..20) mixed with small ones."""
    p = 3
    insts = [x for x in synth.batch_instances(40, 5, n_lo=16, n_hi=20, p=p)][:3]
    insts += synth.batch_instances(5, 6, n_lo=5, n_hi=9, p=p)
    check_rows(run(insts, dtype), insts, dtype, p)
    # the small tiles on the large graphs (three groups at n = 20)
    check_rows(run(insts, dtype, np.zeros(q.MAX_N + 1)), insts, dtype, p)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_batch_grouped_buckets_vs_oracle(dtype):
    """Several graphs per size at n = 16..19 (the sizes whose sweeps run grouped, one launch
    for all graphs of a size, each graph with its own weights, cost range and angles), mixed
    with small graphs for the persistent kernel; every row against the oracle."""
    p = 3
    insts = []
    for n_lo, count, seed in ((16, 24, 31), (18, 12, 32)):
        insts += [x for x in synth.batch_instances(count, seed, n_lo=n_lo, n_hi=n_lo + 1, p=p)]
    insts += synth.batch_instances(6, 33, n_lo=5, n_hi=12, p=p)
    sizes = [x[0] for x in insts]
    assert min(sizes.count(n) for n in (16, 17, 18, 19)) >= 2
    check_rows(run(insts, dtype), insts, dtype, p)


def test_batch_degenerate_graphs_and_depths():
    """n = 1 and edgeless graphs (C = 0: E = 0, zero gradient), and p = 1 and 6."""
    for p in (1, 6):
        insts = []
        for i, n in enumerate([1, 2, 3, 5]):
            e = np.zeros((0, 2), dtype=np.int32)
            gam, bet = synth.angles(p, 40 + i)
            insts.append((n, "empty", e, np.zeros(0), gam, bet))
        insts += synth.batch_instances(6, 7, n_lo=4, n_hi=12, p=p)
        out = run(insts, "c128")
        check_rows(out, insts, "c128", p)
        assert np.all(out[:4, 0] == 0.0) and np.all(out[:4, 2:] == 0.0)


def test_batch_matches_one_graph_path():
    """Each batched row equals the one-graph gradient of the same instance (consistency)."""
    p = 3
    insts = synth.batch_instances(12, 21, n_lo=8, n_hi=20, p=p)
    out = run(insts, "c128")
    for row, (n, fam, e, w, gam, bet) in zip(out, insts):
        g = q.Graph(n, e, w, True)
        cv = q.cost_vector(g, "i32")
        psi, lam = q.new_state(n, "c128"), q.new_state(n, "c128")
        one = q.gradient(psi, lam, cv, gam, bet).cpu().numpy()
        assert np.max(np.abs(row - one)) <= 2e-10 * scale_of(w)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_batch_workload_4096_graphs(dtype):
    """The batched workload at full size: 4096 graphs, n ~ 8..20, p = 3.  Every row has norm 1
    and 0 <= E <= sum w; a sample of rows (one per qubit count) matches the oracle."""
    p = 3
    insts = synth.batch_instances(4096, 1, p=p)
    out = run(insts, dtype)
    W = np.array([np.sum(x[3]) for x in insts])
    assert np.all(np.isfinite(out))
    assert np.max(np.abs(out[:, 1] - 1.0)) <= (1e-12 if dtype == "c128" else 1e-4)
    assert np.all(out[:, 0] >= -1e-6) and np.all(out[:, 0] <= W * (1 + 1e-6))
    pick, seen = [], set()
    for i, x in enumerate(insts):
        if x[0] not in seen and x[0] <= 16:
            seen.add(x[0])
            pick.append(i)
    check_rows(out[pick], [insts[i] for i in pick], dtype, p)


def test_batch_autotune():
    tiles, ms = q.batch_autotune("c128", 3, 8, 14, graphs_per_n=152)
    assert set(np.unique(tiles[8:15])) <= {0, 1}
    assert np.all(ms[8:15] > 0)
    insts = synth.batch_instances(20, 3, n_lo=8, n_hi=14, p=3)
    check_rows(run(insts, "c128", tiles), insts, "c128", 3)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_batch_float_weights_vs_oracle(dtype):
    """U(0,1) weights (float64 costs, directly computed phases), n = 4..18, p = 4."""
    p = 4
    insts = []
    for i, x in enumerate(synth.batch_instances(30, 8, n_lo=4, n_hi=18, p=p)):
        n, fam, e, w, gam, bet = x
        insts.append((n, fam, e, synth.edge_weights(len(e), "u01", 1000 + i), gam, bet))
    check_rows(run(insts, dtype, integer=False), insts, dtype, p, integer=False)
