"""The learned angle proposer's fused inference kernel against the same network in plain
PyTorch float32, and the trained proposer against random starting angles.

Tolerance: float32 with different summation orders over <= 2H + 32 terms per output, so
|kernel - reference| <= 1e-4 (1 + |reference|).
"""
from pathlib import Path

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2407_13012_gb300 as q  # noqa: E402
from paper_2407_13012_gb300 import proposer  # noqa: E402


def graphs_for_test():
    insts = []
    for i, n in enumerate([2, 3, 7, 12, 15, 18, 24, 32]):
        e = synth.gnp_edges(n, 0.3, 50 + i)
        insts.append((n, e, synth.edge_weights(len(e), "u01", 50 + i)))
    e = synth.gnp_edges(10, 0.5, 3)
    insts.append((10, e, synth.edge_weights(len(e), "int", 3, 1, 5)))
    insts.append((6, np.zeros((0, 2), dtype=np.int32), np.zeros(0)))
    return insts


@pytest.mark.parametrize("p", [1, 4, 8])
def test_kernel_matches_torch_reference(p):
    torch.manual_seed(p)
    net = proposer.make_net(p)
    with torch.no_grad():  # larger than default weights, so every layer matters
        for prm in net.parameters():
            prm.mul_(2.0)
    vec = proposer.pack(net)
    assert len(vec) == q.proposer_param_count(p)
    insts = graphs_for_test()
    graphs = [q.Graph(n, e, w, False) for n, e, w in insts]
    got = q.propose_angles(graphs, torch.as_tensor(vec, device="cuda"), p).cpu().numpy()
    ref = proposer.reference_forward(net, insts, "cuda").cpu().numpy()
    assert got.shape == (len(insts), 2 * p)
    assert np.all(np.abs(got - ref) <= 1e-4 * (1.0 + np.abs(ref)))


@pytest.mark.skipif(not proposer.DEFAULT_WEIGHTS.exists(), reason="no trained proposer weights")
def test_trained_proposer_beats_random_starts():
    params, p, meta = proposer.load_weights()
    insts = synth.proposer_instances(48, 4321)
    graphs = [q.Graph(n, e, w, False) for n, e, w in insts]
    prop = q.propose_angles(graphs, torch.as_tensor(params, device="cuda"), p).cpu().numpy()
    rnd = np.random.default_rng(0).uniform(0, np.pi, prop.shape)
    e_prop = q.batch_gradient(graphs, prop, "c128").cpu().numpy()[:, 0]
    e_rnd = q.batch_gradient(graphs, rnd, "c128").cpu().numpy()[:, 0]
    W = np.array([w.sum() for _, _, w in insts])
    # the proposer's start is well above the uniform-superposition value W/2 and above random
    assert np.mean(e_prop / W) > np.mean(e_rnd / W) + 0.02
    assert np.mean(e_prop / W) > 0.55
