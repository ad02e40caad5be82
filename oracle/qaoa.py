"""Plain FP64 CPU oracle for MaxCut QAOA (test infrastructure, not the product).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path.
Every routine is the plain definition from the paper (arXiv 2407.13012),
written for a reader to check by eye; none of it is blocked, fused or
reordered for speed.

Conventions
-----------
* Amplitude index z in [0, 2**n); qubit j is bit j of z.  This is the one-hot
  encoding of Eq. 3 (variable i carries weight 2**i).
* Cost (cut value) C(z) = sum over edges (u, v) of w_uv * [bit u of z != bit v of z]
  (MaxCut, Sec. V; diagonal cost Hamiltonian H_C = sum_x f(x)|x><x|, Sec. II-A).
* Cost unitary U_C(gamma) = exp(-i gamma H_C): psi_z *= exp(-i gamma C(z))
  (Eq. 1 and Sec. IV-B).
* Mixer U_M(beta) = exp(-i beta sum_j X_j) = prod_j RX_j(2 beta).  The paper's
  H_M = -sum_j X_j gives R_x(-2 beta) (Sec. II-A, Sec. IV-B); the two differ by
  beta -> -beta only.  This oracle uses RX(2 beta); ``mixer_sign=-1`` selects
  the paper's sign.
* State after p layers (Eq. 1): U_M(b_p) U_C(g_p) ... U_M(b_1) U_C(g_1) |+>^n.
"""
from __future__ import annotations

import numpy as np

# --------------------------------------------------------------------- costs


def cut_values(n: int, edges, weights=None, integer: bool = True) -> np.ndarray:
    """C(z) for all z in [0, 2**n): the weighted cut, summed edge by edge in edge-list order.

    MaxCut objective (Sec. V) as the diagonal of H_C (Sec. II-A), bit order of
    Eq. 3.  Integer weights give int64 values (exact).  Float weights give
    float64 values accumulated as acc = acc + w_e * cut_e(z) in edge order,
    where cut_e is 0 or 1 so every product is exact.
    """
    edges = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    m = len(edges)
    w = np.ones(m) if weights is None else np.asarray(weights, dtype=np.float64)
    z = np.arange(1 << n, dtype=np.int64)
    if integer:
        wi = w.astype(np.int64)
        if not np.array_equal(wi.astype(np.float64), w):
            raise ValueError("integer cut values need integral weights")
        acc = np.zeros(1 << n, dtype=np.int64)
        for e in range(m):
            u, v = edges[e]
            acc = acc + wi[e] * (((z >> u) ^ (z >> v)) & 1)
        return acc
    acc = np.zeros(1 << n, dtype=np.float64)
    for e in range(m):
        u, v = edges[e]
        acc = acc + w[e] * (((z >> u) ^ (z >> v)) & 1).astype(np.float64)
    return acc


def maxcut_pubo_terms(edges, weights=None):
    """MaxCut as a 0-1 polynomial: w_uv (x_u + x_v - 2 x_u x_v) per edge.

    Returns a list of (weight, [variable indices]) terms, the input form of
    Eq. 3 (terms t_k with weights w_k).
    """
    edges = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    w = np.ones(len(edges)) if weights is None else np.asarray(weights, dtype=np.float64)
    terms = []
    for (u, v), we in zip(edges, w):
        terms += [(we, [int(u)]), (we, [int(v)]), (-2.0 * we, [int(u), int(v)])]
    return terms


def pubo_values(n: int, terms, integer: bool = True) -> np.ndarray:
    """f(x) for all x by Eq. 3: sum_k w_k [x AND mask_k == mask_k], mask_k = sum_{i in t_k} 2**i.

    The term counts when every variable of t_k is 1 in x (the product of the
    x_i).  Reading of Eq. 3: its "x <=> x AND mask" is taken as
    (x AND mask) == mask.
    """
    x = np.arange(1 << n, dtype=np.int64)
    acc = np.zeros(1 << n, dtype=np.int64 if integer else np.float64)
    for wk, tk in terms:
        mask = 0
        for i in tk:
            mask |= 1 << i
        hit = ((x & mask) == mask)
        if integer:
            acc = acc + int(wk) * hit.astype(np.int64)
        else:
            acc = acc + wk * hit.astype(np.float64)
    return acc


# -------------------------------------------------------------------- states


def plus_state(n: int) -> np.ndarray:
    """|+>^n: every amplitude 1/sqrt(2**n) (Sec. IV-B)."""
    return np.full(1 << n, 1.0 / np.sqrt(float(1 << n)), dtype=np.complex128)


def apply_cost_unitary(psi: np.ndarray, C: np.ndarray, gamma: float) -> np.ndarray:
    """psi_z -> exp(-i gamma C(z)) psi_z (Sec. IV-B, Euler's formula)."""
    th = -gamma * np.asarray(C, dtype=np.float64)
    return psi * (np.cos(th) + 1j * np.sin(th))


def apply_rx_all(psi: np.ndarray, n: int, beta: float, mixer_sign: int = 1) -> np.ndarray:
    """prod_j RX_j(2 s beta) with s = mixer_sign; one qubit at a time (Sec. IV-B).

    RX(2b) = cos(b) I - i sin(b) X; on a pair (a, b') = (psi[z], psi[z | 2**j])
    with bit j of z clear: a -> cos a - i sin b', b' -> cos b' - i sin a.
    """
    c, s = np.cos(mixer_sign * beta), np.sin(mixer_sign * beta)
    out = psi.copy()
    for j in range(n):
        v = out.reshape(-1, 2, 1 << j)
        a, b = v[:, 0, :].copy(), v[:, 1, :].copy()
        v[:, 0, :] = c * a - 1j * s * b
        v[:, 1, :] = c * b - 1j * s * a
    return out


def apply_b(psi: np.ndarray, n: int) -> np.ndarray:
    """B psi with B = sum_j X_j (the generator of the mixer, Sec. IV-C)."""
    out = np.zeros_like(psi)
    for j in range(n):
        v = psi.reshape(-1, 2, 1 << j)
        o = out.reshape(-1, 2, 1 << j)
        o[:, 0, :] += v[:, 1, :]
        o[:, 1, :] += v[:, 0, :]
    return out


def qaoa_state(n: int, C: np.ndarray, gammas, betas, psi0: np.ndarray | None = None,
               mixer_sign: int = 1) -> np.ndarray:
    """Eq. 1: U_M(b_p) U_C(g_p) ... U_M(b_1) U_C(g_1) applied to |+>^n (or psi0)."""
    psi = plus_state(n) if psi0 is None else np.asarray(psi0, dtype=np.complex128).copy()
    for g, b in zip(gammas, betas):
        psi = apply_cost_unitary(psi, C, g)
        psi = apply_rx_all(psi, n, b, mixer_sign)
    return psi


# --------------------------------------------------------------- observables


def expectation(psi: np.ndarray, C: np.ndarray) -> float:
    """<psi|H_C|psi> = sum_i f(x_i) |psi_i|**2 (Sec. IV-D); numpy's pairwise sum."""
    return float(np.sum(np.asarray(C, dtype=np.float64) * (psi.real ** 2 + psi.imag ** 2)))


def norm2(psi: np.ndarray) -> float:
    return float(np.sum(psi.real ** 2 + psi.imag ** 2))


def sample(psi: np.ndarray, C: np.ndarray, u: np.ndarray):
    """Inverse-CDF sampling (Sec. IV-D): z_i = min{z : P(z) > u_i * P_total}.

    P is the inclusive running sum of |psi_z|**2 in index order.  If rounding
    puts the target at or past the end, z_i is the last index with nonzero
    probability.  Returns (z uint64, C[z] float64): the sampled bitstrings
    with their objective values.
    """
    prob = psi.real ** 2 + psi.imag ** 2
    P = np.cumsum(prob)
    total = P[-1]
    z = np.searchsorted(P, np.asarray(u, dtype=np.float64) * total, side="right")
    nz = np.nonzero(prob > 0)[0]
    last = nz[-1] if len(nz) else len(prob) - 1
    z = np.minimum(z, last)
    return z.astype(np.uint64), np.asarray(C, dtype=np.float64)[z]


# ------------------------------------------------------------------ gradient


def adjoint_gradient(n: int, C: np.ndarray, gammas, betas):
    """Adjoint differentiation of E = <C> in all 2p angles (Sec. II-B, Sec. IV-C).

    Forward to psi_p, set lam = C psi_p (so E = Re<psi|lam>).  Then for
    l = p..1: dE/dbeta_l = 2 Im <lam|B|psi>; uncompute both states with
    U_M(beta_l)^dagger; dE/dgamma_l = 2 Im <lam|C|psi>; uncompute both with
    U_C(gamma_l)^dagger.  The -i of each generator is absorbed by taking the
    imaginary part instead of the real part (Sec. IV-C).

    Returns (E, dE/dgamma (p,), dE/dbeta (p,), psi after the uncompute).
    """
    Cf = np.asarray(C, dtype=np.float64)
    p = len(gammas)
    psi = qaoa_state(n, Cf, gammas, betas)
    lam = Cf * psi
    E = float(np.vdot(psi, lam).real)
    dg, db = np.zeros(p), np.zeros(p)
    for l in range(p - 1, -1, -1):
        db[l] = 2.0 * np.vdot(lam, apply_b(psi, n)).imag
        psi = apply_rx_all(psi, n, -betas[l])
        lam = apply_rx_all(lam, n, -betas[l])
        dg[l] = 2.0 * np.vdot(lam, Cf * psi).imag
        psi = apply_cost_unitary(psi, Cf, -gammas[l])
        lam = apply_cost_unitary(lam, Cf, -gammas[l])
    return E, dg, db, psi


def finite_difference_gradient(n: int, C: np.ndarray, gammas, betas, h: float = 1e-6):
    """Central differences (E(t + h) - E(t - h)) / 2h in every angle."""
    gammas, betas = np.asarray(gammas, float), np.asarray(betas, float)

    def E(g, b):
        return expectation(qaoa_state(n, C, g, b), C)

    dg, db = np.zeros(len(gammas)), np.zeros(len(betas))
    for l in range(len(gammas)):
        e = np.zeros(len(gammas))
        e[l] = h
        dg[l] = (E(gammas + e, betas) - E(gammas - e, betas)) / (2 * h)
        db[l] = (E(gammas, betas + e) - E(gammas, betas - e)) / (2 * h)
    return dg, db


def linear_ramp(p: int):
    """Constant-speed schedule of Sec. II-A: beta_i = 1 - i/p, gamma_i = i/p, i = 1..p."""
    i = np.arange(1, p + 1, dtype=np.float64)
    return i / p, 1.0 - i / p
