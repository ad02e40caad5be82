"""Seeded synthetic inputs for MaxCut QAOA: graphs, edge weights, angles, sampling uniforms.

This module holds no QAOA arithmetic. It is the one piece shared by the CPU
oracle (``oracle/``) and the CUDA path (tests and ``bench.py``): both receive
the same graphs, weights and angles from here.

Every random number comes from SplitMix64 (Steele, Lea, Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014), used as a
counter-based generator: the i-th draw (i = 0, 1, ...) of a stream with base
state ``s`` is ``mix64(s + (i + 1) * GOLDEN)``.  A stream is keyed by
``(seed, purpose)`` with ``base = mix64(mix64(seed) ^ purpose_tag)``.  The
53-bit uniform of a 64-bit draw ``x`` is ``(x >> 11) * 2**-53`` in [0, 1).

The paper's instances (Sec. V: Erdos-Renyi G(n, p), random 3-regular and
complete graphs, n = 6..29) are not distributed with it; these generators
produce graphs of the same families.
"""
from __future__ import annotations

import numpy as np

MASK64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB

# Purpose tags: ASCII of a short name, so each consumer draws from its own stream.
PURPOSE = {
    "gnp": int.from_bytes(b"gnp-edge", "little"),
    "reg3": int.from_bytes(b"reg3-pai", "little"),
    "weights": int.from_bytes(b"weights_", "little"),
    "angles": int.from_bytes(b"angles__", "little"),
    "sample": int.from_bytes(b"sample__", "little"),
    "state": int.from_bytes(b"state___", "little"),
    "batch": int.from_bytes(b"batch-gr", "little"),
}


def mix64(z: int) -> int:
    """SplitMix64 output function (finaliser) on a 64-bit integer."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * _M1) & MASK64
    z = ((z ^ (z >> 27)) * _M2) & MASK64
    return z ^ (z >> 31)


def stream_base(seed: int, purpose: str) -> int:
    return mix64(mix64(seed & MASK64) ^ PURPOSE[purpose])


def draws_u64(seed: int, purpose: str, count: int, start: int = 0) -> np.ndarray:
    """Draws ``start .. start+count-1`` of stream (seed, purpose) as uint64 (vectorised mix64)."""
    base = np.uint64(stream_base(seed, purpose))
    i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = base + i * np.uint64(GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
        z = z ^ (z >> np.uint64(31))
    return z


def uniforms(seed: int, purpose: str, count: int, start: int = 0) -> np.ndarray:
    """53-bit uniforms in [0, 1) from stream (seed, purpose)."""
    return (draws_u64(seed, purpose, count, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


class Stream:
    """Sequential reader over one counter-based stream."""

    def __init__(self, seed: int, purpose: str):
        self.seed, self.purpose, self.i = seed, purpose, 0

    def next_u64(self) -> int:
        self.i += 1
        return mix64(stream_base(self.seed, self.purpose) + self.i * GOLDEN)

    def next_uniform(self) -> float:
        return (self.next_u64() >> 11) * (2.0 ** -53)

    def next_below(self, k: int) -> int:
        """Integer uniform in [0, k) by floor(u * k) of a 53-bit uniform."""
        return min(int(self.next_uniform() * k), k - 1)


# ---------------------------------------------------------------- graphs


def gnp_edges(n: int, prob: float, seed: int) -> np.ndarray:
    """Erdos-Renyi G(n, prob): for u < v in lexicographic order keep (u, v) if U < prob.

    Returns int32 array of shape (m, 2) with u < v in that order.
    """
    u_idx, v_idx = np.triu_indices(n, k=1)  # row-major: (0,1),(0,2),...,(1,2),...
    keep = uniforms(seed, "gnp", len(u_idx)) < prob
    return np.stack([u_idx[keep], v_idx[keep]], axis=1).astype(np.int32)


def regular3_edges(n: int, seed: int, max_restarts: int = 100000) -> np.ndarray:
    """Random 3-regular graph by the pairing (configuration) model, restarting until simple.

    n must be even and >= 4.  Points 3v, 3v+1, 3v+2 belong to vertex v; a
    Fisher-Yates shuffle of the 3n points (drawn from the stream) is paired
    off two by two.  A pairing with a loop or a repeated edge is rejected and
    the stream continues.  Edges are returned as (min, max) in pairing order.
    """
    if n < 4 or n % 2:
        raise ValueError("random 3-regular graphs need an even n >= 4")
    st = Stream(seed, "reg3")
    for _ in range(max_restarts):
        pts = list(range(3 * n))
        for i in range(3 * n - 1, 0, -1):
            j = st.next_below(i + 1)
            pts[i], pts[j] = pts[j], pts[i]
        seen, edges, ok = set(), [], True
        for k in range(0, 3 * n, 2):
            a, b = pts[k] // 3, pts[k + 1] // 3
            if a == b:
                ok = False
                break
            e = (min(a, b), max(a, b))
            if e in seen:
                ok = False
                break
            seen.add(e)
            edges.append(e)
        if ok:
            return np.asarray(edges, dtype=np.int32).reshape(-1, 2)
    raise RuntimeError("pairing model did not produce a simple graph")


def complete_edges(n: int) -> np.ndarray:
    u_idx, v_idx = np.triu_indices(n, k=1)
    return np.stack([u_idx, v_idx], axis=1).astype(np.int32)


def edge_weights(m: int, kind: str, seed: int, lo: int = 1, hi: int = 10) -> np.ndarray:
    """Edge weights as float64.

    kind: "unit" (all 1), "u01" (53-bit uniforms in [0, 1)), or "int" (integers
    uniform in {lo..hi}, stored exactly as float64).
    """
    if kind == "unit":
        return np.ones(m, dtype=np.float64)
    u = uniforms(seed, "weights", m)
    if kind == "u01":
        return u
    if kind == "int":
        k = hi - lo + 1
        return (lo + np.minimum(np.floor(u * k), k - 1)).astype(np.float64)
    raise ValueError(kind)


def angles(p: int, seed: int, lo: float = 0.0, hi: float = np.pi) -> tuple[np.ndarray, np.ndarray]:
    """Angles gamma_l, beta_l ~ U(lo, hi), drawn in the order gamma_1, beta_1, gamma_2, ..."""
    u = uniforms(seed, "angles", 2 * p)
    a = lo + (hi - lo) * u
    return a[0::2].copy(), a[1::2].copy()


def sample_uniforms(seed: int, shots: int) -> np.ndarray:
    """The uniforms u_0 .. u_{shots-1} a sampler keyed by ``seed`` consumes (stream "sample")."""
    return uniforms(seed, "sample", shots)


def random_state(n: int, seed: int) -> np.ndarray:
    """A normalised random complex128 statevector (for tests that start from a general state)."""
    u = uniforms(seed, "state", 2 << n).reshape(-1, 2) - 0.5
    psi = u[:, 0] + 1j * u[:, 1]
    return psi / np.linalg.norm(psi)


def graph(family: str, n: int, seed: int, weights: str = "unit", prob: float = 0.5,
          lo: int = 1, hi: int = 10):
    """Convenience: (edges int32 (m, 2), weights float64 (m,), weight_is_int bool)."""
    if family == "gnp":
        e = gnp_edges(n, prob, seed)
    elif family == "reg3":
        e = regular3_edges(n, seed)
    elif family == "complete":
        e = complete_edges(n)
    else:
        raise ValueError(family)
    w = edge_weights(len(e), weights, seed, lo, hi)
    return e, w, weights in ("unit", "int")


def batch_instances(count: int, seed: int, n_lo: int = 8, n_hi: int = 20, prob: float = 0.3, lo: int = 1,
                    hi: int = 5, p: int = 3):
    """The batched workload: ``count`` graphs, each a fair coin between a random 3-regular
    graph (n uniform over the even values in [n_lo, n_hi]) and G(n, prob) (n uniform in
    [n_lo, n_hi]), integer weights uniform in {lo..hi}, and its own angles U(0, pi).

    Returns a list of (n, family, edges, weights, gammas, betas); graph i draws its edges,
    weights and angles from the streams of seed ``seed * 2^20 + i``.
    """
    st = Stream(seed, "batch")
    evens = [n for n in range(max(n_lo, 4), n_hi + 1) if n % 2 == 0]
    out = []
    for i in range(count):
        reg3 = st.next_below(2) == 0 and len(evens) > 0
        n = evens[st.next_below(len(evens))] if reg3 else n_lo + st.next_below(n_hi - n_lo + 1)
        gseed = ((seed << 20) + i) & MASK64
        e = regular3_edges(n, gseed) if reg3 else gnp_edges(n, prob, gseed)
        w = edge_weights(len(e), "int", gseed, lo, hi)
        gam, bet = angles(p, gseed)
        out.append((n, "reg3" if reg3 else "gnp", e, w, gam, bet))
    return out


def proposer_instances(count: int, seed: int, n_lo: int = 12, n_hi: int = 18, prob: float = 0.3):
    """Graphs for the learned angle proposer: G(n, prob) with n uniform in [n_lo, n_hi] and
    U(0,1) weights.  Returns a list of (n, edges, weights); graph i draws its edges and
    weights from the streams of seed ``seed * 2^20 + i``."""
    st = Stream(seed, "batch")
    out = []
    for i in range(count):
        n = n_lo + st.next_below(n_hi - n_lo + 1)
        gseed = ((seed << 20) + i) & MASK64
        e = gnp_edges(n, prob, gseed)
        out.append((n, e, edge_weights(len(e), "u01", gseed)))
    return out
