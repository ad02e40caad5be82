"""Learned angle proposer: a message-passing network that maps a weighted graph to 2p
starting angles for the on-device optimisers.

Inference runs in the library's fused CUDA kernel (``propose_angles``); this module holds
the same network in plain PyTorch float32 (for training, and as the kernel's numerics
reference), the generation of training targets with the batched adjoint gradient, the
training loop and the evaluation.  Network (H = 64, 3 message-passing layers), for a graph
with weighted adjacency A, degrees d and weighted degrees s = A 1:

    h = relu([d / 4, s / 2] W_in + b_in)
    3 x: h = relu(h W_s + ((A h) / max(1, d)) W_m + b)
    angles = relu([mean h, max h] W_1 + b_1) W_2 + b_2

Command line (on a GPU)::

    python -m paper_2407_13012_gb300.proposer train --count 50000 --out proposer_p4.npz
    python -m paper_2407_13012_gb300.proposer eval --weights proposer_p4.npz
"""
from __future__ import annotations

import argparse
import json
import time
from pathlib import Path

import numpy as np

HIDDEN, LAYERS, NMAX = 64, 3, 32
DEFAULT_WEIGHTS = Path(__file__).resolve().parent / "proposer_p4.npz"


def _torch():
    import torch
    return torch


def make_net(p: int):
    """The network as a torch module (float32)."""
    torch = _torch()
    nn = torch.nn

    class ProposerNet(nn.Module):
        def __init__(self):
            super().__init__()
            self.p = p
            self.inp = nn.Linear(2, HIDDEN)
            self.ws = nn.ModuleList([nn.Linear(HIDDEN, HIDDEN) for _ in range(LAYERS)])
            self.wm = nn.ModuleList([nn.Linear(HIDDEN, HIDDEN, bias=False) for _ in range(LAYERS)])
            self.l1 = nn.Linear(2 * HIDDEN, HIDDEN)
            self.l2 = nn.Linear(HIDDEN, 2 * p)

        def forward(self, A, mask, deg):
            """A: (B, N, N) weighted adjacency (0 off the graph), mask: (B, N) 1 on vertices,
            deg: (B, N) vertex degrees."""
            s = A.sum(-1)
            x = torch.stack([deg * 0.25, s * 0.5], -1)
            m3 = mask.unsqueeze(-1)
            h = torch.relu(self.inp(x)) * m3
            for l in range(LAYERS):
                agg = torch.bmm(A, h) / torch.clamp(deg, min=1.0).unsqueeze(-1)
                h = torch.relu(self.ws[l](h) + self.wm[l](agg)) * m3
            n = mask.sum(-1, keepdim=True)
            g = torch.cat([h.sum(1) / n, h.max(1).values], -1)  # h >= 0 and 0 off the graph
            return self.l2(torch.relu(self.l1(g)))

    return ProposerNet()


def pack(net) -> np.ndarray:
    """The kernel's parameter vector: row-major (in x out) W_in, b_in, (W_s, W_m, b) x 3,
    W_1, b_1, W_2, b_2 (torch Linear stores out x in, hence the transposes)."""
    parts = [net.inp.weight.T, net.inp.bias]
    for l in range(LAYERS):
        parts += [net.ws[l].weight.T, net.wm[l].weight.T, net.ws[l].bias]
    parts += [net.l1.weight.T, net.l1.bias, net.l2.weight.T, net.l2.bias]
    return np.concatenate([t.detach().float().cpu().numpy().reshape(-1) for t in parts]).astype(np.float32)


def unpack(vec: np.ndarray, p: int):
    """A torch module holding the parameters of a packed vector."""
    torch = _torch()
    net = make_net(p)
    k = 0

    def take(shape):
        nonlocal k
        size = int(np.prod(shape))
        out = torch.as_tensor(np.asarray(vec[k:k + size], dtype=np.float32).reshape(shape))
        k += size
        return out

    with torch.no_grad():
        net.inp.weight.copy_(take((2, HIDDEN)).T)
        net.inp.bias.copy_(take((HIDDEN,)))
        for l in range(LAYERS):
            net.ws[l].weight.copy_(take((HIDDEN, HIDDEN)).T)
            net.wm[l].weight.copy_(take((HIDDEN, HIDDEN)).T)
            net.ws[l].bias.copy_(take((HIDDEN,)))
        net.l1.weight.copy_(take((2 * HIDDEN, HIDDEN)).T)
        net.l1.bias.copy_(take((HIDDEN,)))
        net.l2.weight.copy_(take((HIDDEN, 2 * p)).T)
        net.l2.bias.copy_(take((2 * p,)))
    assert k == len(vec), (k, len(vec))
    return net


def graph_tensors(insts, device, nmax: int | None = None):
    """Padded adjacency (B, N, N), vertex mask (B, N) and degrees (B, N) of (n, edges, w)."""
    torch = _torch()
    N = nmax or max(n for n, _, _ in insts)
    A = np.zeros((len(insts), N, N), dtype=np.float32)
    D = np.zeros((len(insts), N), dtype=np.float32)
    M = np.zeros((len(insts), N), dtype=np.float32)
    for b, (n, e, w) in enumerate(insts):
        M[b, :n] = 1.0
        if len(e):
            A[b, e[:, 0], e[:, 1]] = w
            A[b, e[:, 1], e[:, 0]] = w
            np.add.at(D[b], e[:, 0], 1.0)
            np.add.at(D[b], e[:, 1], 1.0)
    return (torch.as_tensor(A, device=device), torch.as_tensor(M, device=device),
            torch.as_tensor(D, device=device))


def reference_forward(net, insts, device):
    """The network on (n, edges, w) graphs with degrees counted from the edge lists (as the
    kernel counts them), float32."""
    torch = _torch()
    A, M, D = graph_tensors(insts, device)
    with torch.no_grad():
        return net.to(device)(A, M, D).double()


# ---------------------------------------------------------------- training targets

def ramp_init(count: int, p: int, scale: float = 2.0) -> np.ndarray:
    """The linear-ramp schedule gamma_i = scale i / p, beta_i = 1 - i / p (Sec. II-A) for
    every graph; the optimiser's common starting point."""
    i = np.arange(1, p + 1, dtype=np.float64)
    return np.tile(np.concatenate([scale * i / p, 1.0 - i / p]), (count, 1))


def optimise_batch(insts, p: int, steps: int = 150, lr: float = 0.03, dtype: str = "c64", init=None,
                   chunk: int = 8192, device="cuda", log=None):
    """Adam ascent on <C> for every graph at once (batched adjoint gradients on the device,
    `chunk` graphs per launch).  Returns (angles (G, 2p), E (G,)) at the last step."""
    from . import Graph, batch_gradient
    ang = ramp_init(len(insts), p) if init is None else np.array(init, dtype=np.float64)
    E = np.zeros(len(insts))
    for c0 in range(0, len(insts), chunk):
        sub = insts[c0:c0 + chunk]
        graphs = [Graph(n, e, w, False) for n, e, w in sub]
        a = ang[c0:c0 + chunk]
        m, v = np.zeros_like(a), np.zeros_like(a)
        for t in range(1, steps + 1):
            out = batch_gradient(graphs, a, dtype, device=device).cpu().numpy()
            g = out[:, 2:]
            E[c0:c0 + len(sub)] = out[:, 0]
            m = 0.9 * m + 0.1 * g
            v = 0.999 * v + 0.001 * g * g
            a = a + lr * (m / (1 - 0.9 ** t)) / (np.sqrt(v / (1 - 0.999 ** t)) + 1e-8)
        ang[c0:c0 + chunk] = a
        if log:
            log(f"optimised graphs {c0}..{c0 + len(sub)}: mean E {E[c0:c0 + len(sub)].mean():.4f}")
    return ang, E


def train(insts, targets, p: int, epochs: int = 60, batch: int = 512, lr: float = 2e-3, seed: int = 0,
          device="cuda", log=None):
    """Fit the network to optimised angles (mean squared error), 10% held out for validation."""
    torch = _torch()
    torch.manual_seed(seed)
    net = make_net(p).to(device)
    A, M, D = graph_tensors(insts, device, nmax=max(n for n, _, _ in insts))
    Y = torch.as_tensor(targets, dtype=torch.float32, device=device)
    nval = max(1, len(insts) // 10)
    perm = torch.randperm(len(insts), generator=torch.Generator().manual_seed(seed)).to(device)
    val, tr = perm[:nval], perm[nval:]
    opt = torch.optim.Adam(net.parameters(), lr=lr)
    sched = torch.optim.lr_scheduler.CosineAnnealingLR(opt, T_max=epochs)
    for ep in range(epochs):
        net.train()
        order = tr[torch.randperm(len(tr), device=device)]
        for b0 in range(0, len(order), batch):
            idx = order[b0:b0 + batch]
            loss = torch.mean((net(A[idx], M[idx], D[idx]) - Y[idx]) ** 2)
            opt.zero_grad()
            loss.backward()
            opt.step()
        sched.step()
        if log and (ep % 10 == 0 or ep == epochs - 1):
            net.eval()
            with torch.no_grad():
                vl = torch.mean((net(A[val], M[val], D[val]) - Y[val]) ** 2).item()
            log(f"epoch {ep}: train mse {loss.item():.5f} val mse {vl:.5f}")
    net.eval()
    return net


def save_weights(path, net, p: int, meta: dict):
    np.savez_compressed(path, params=pack(net), p=np.int32(p), meta=json.dumps(meta))


def load_weights(path=DEFAULT_WEIGHTS):
    d = np.load(path)
    return d["params"].astype(np.float32), int(d["p"]), json.loads(str(d["meta"]))


# ---------------------------------------------------------------- evaluation

def evaluate(params: np.ndarray, p: int, insts, max_evals: int = 100, dtype: str = "c128", seed: int = 0,
             tol: float = 1e-3, device="cuda", log=None):
    """Approximation ratio and time to a near-optimal value, per graph, for three starting
    points of the on-device L-BFGS: the proposer, the linear ramp and random angles U(0, pi).

    The target of a graph is (1 - tol) times the best final <C> over the three runs; the time
    to it is the device time of the evaluations until the best value so far reaches it (plus
    the proposer's own inference for its start).  maxcut is max_z C(z) of the cost vector."""
    torch = _torch()
    from . import Graph, cost_vector, optimize_lbfgs, propose_angles
    graphs = [Graph(n, e, w, False) for n, e, w in insts]
    pt = torch.as_tensor(params, device=device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    propose_angles(graphs, pt, p, device=device)  # warm-up
    e0.record()
    prop = propose_angles(graphs, pt, p, device=device)
    e1.record()
    torch.cuda.synchronize()
    prop_ms = e0.elapsed_time(e1) / len(graphs)
    rng = np.random.default_rng(seed)
    rows = []
    for gi, (g, (n, e, w)) in enumerate(zip(graphs, insts)):
        cv = cost_vector(g, "f64", device=device)
        maxcut = float(cv.C.max().item())
        starts = {"proposer": prop[gi].clone(), "ramp": torch.as_tensor(ramp_init(1, p)[0], device=device),
                  "random": torch.as_tensor(rng.uniform(0.0, np.pi, 2 * p), device=device)}
        runs = {}
        for name, ang in starts.items():
            e0.record()
            hist, info = optimize_lbfgs(cv, ang, max_evals=max_evals, m=10, gtol=1e-6, dtype=dtype)
            e1.record()
            torch.cuda.synchronize()
            h = hist.cpu().numpy()
            runs[name] = (np.maximum.accumulate(h[:, 0]), e0.elapsed_time(e1) / max(1, len(h)), info)
        best = max(r[2]["E"] for r in runs.values())
        target = best - tol * abs(best)
        row = {"n": n, "maxcut": maxcut}
        for name, (run_best, ms_eval, info) in runs.items():
            hit = np.nonzero(run_best >= target)[0]
            k = int(hit[0]) + 1 if len(hit) else None
            row[name] = {"ratio_start": float(run_best[0] / maxcut), "ratio_final": info["E"] / maxcut,
                         "evals_to_target": k, "ms_to_target": None if k is None else
                         k * ms_eval + (prop_ms if name == "proposer" else 0.0)}
        rows.append(row)
        if log and gi % 16 == 0:
            log(f"graph {gi} n={n}: " + ", ".join(f"{k}: {row[k]['ratio_start']:.3f}->{row[k]['evals_to_target']}"
                                                  for k in starts))
    summary = {"graphs": len(rows), "p": p, "dtype": dtype, "proposer_ms_per_graph": prop_ms, "tol": tol}
    for name in ("proposer", "ramp", "random"):
        rs = [r[name] for r in rows]
        reached = [r for r in rs if r["evals_to_target"] is not None]
        summary[name] = {
            "mean_ratio_start": float(np.mean([r["ratio_start"] for r in rs])),
            "mean_ratio_final": float(np.mean([r["ratio_final"] for r in rs])),
            "reached_target": len(reached) / len(rs),
            "mean_evals_to_target": float(np.mean([r["evals_to_target"] for r in reached])) if reached else None,
            "mean_ms_to_target": float(np.mean([r["ms_to_target"] for r in reached])) if reached else None,
        }
    return summary, rows


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("cmd", choices=["train", "eval"])
    ap.add_argument("--p", type=int, default=4)
    ap.add_argument("--count", type=int, default=50000)
    ap.add_argument("--steps", type=int, default=150)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--out", default=str(DEFAULT_WEIGHTS))
    ap.add_argument("--weights", default=str(DEFAULT_WEIGHTS))
    ap.add_argument("--eval-count", type=int, default=128)
    ap.add_argument("--eval-n28", type=int, default=3)
    ap.add_argument("--max-evals", type=int, default=100)
    ap.add_argument("--json", default=None)
    a = ap.parse_args(argv)
    import synth  # the repository's seeded input generators (run from the repository root)

    def log(msg):
        print(f"[{time.strftime('%H:%M:%S')}] {msg}", flush=True)

    if a.cmd == "train":
        insts = synth.proposer_instances(a.count, a.seed)
        log(f"{len(insts)} instances, n 12..18, G(n, 0.3), U(0,1) weights")
        t0 = time.time()
        ang, E = optimise_batch(insts, a.p, steps=a.steps, log=log)
        log(f"targets in {time.time() - t0:.1f} s, mean E {E.mean():.4f}")
        net = train(insts, ang, a.p, epochs=a.epochs, log=log)
        meta = {"instances": a.count, "seed": a.seed, "family": "G(n,0.3) U(0,1), n 12..18",
                "targets": f"{a.steps} Adam steps (lr 0.03) from the linear ramp, batched adjoint gradients, c64",
                "epochs": a.epochs}
        save_weights(a.out, net, a.p, meta)
        log(f"saved {a.out}")
        return 0
    params, p, meta = load_weights(a.weights)
    res = {"weights": meta}
    held = synth.proposer_instances(a.eval_count, a.seed + 1000)
    res["held_out"], _ = evaluate(params, p, held, max_evals=a.max_evals, log=log)
    log(json.dumps(res["held_out"]))
    if a.eval_n28 > 0:
        big = synth.proposer_instances(a.eval_n28, a.seed + 2000, n_lo=28, n_hi=28)
        res["n28"], _ = evaluate(params, p, big, max_evals=a.max_evals, log=log)
        log(json.dumps(res["n28"]))
    if a.json:
        Path(a.json).write_text(json.dumps(res, indent=1))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
