"""Plain FP64 CPU oracle for QAOA inside a Hamming-weight subspace with a
constraint-preserving XY mixer (test infrastructure, not the product).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It shares no code with the CUDA path.

The paper names constraint-preserving mixers as future work: simulating only the
feasible states of a constrained problem shrinks the state the simulator carries
(Sec. VI).  It fixes no mixer, so this oracle takes the standard one for a
cardinality constraint, the XY mixer of the quantum alternating operator ansatz
(Hadfield et al., Algorithms 12(2):34, 2019):

* Feasible set F_k = {z in [0, 2**n) : popcount(z) = k} (qubit j = bit j of z, as
  everywhere else); for MaxCut this is the balanced cut (graph bisection) when
  k = n/2.  Its size is binom(n, k).
* Rank order: the states of F_k in increasing integer order.  The rank of z is
  its position in that order (the combinatorial number system), and a subspace
  state is the vector of amplitudes of F_k in rank order.
* Start state: the uniform superposition over F_k (the Dicke state).
* Cost unitary: psi_z *= exp(-i gamma C(z)) with the cut values C of the full
  problem, restricted to F_k.
* Pair gate on qubits (a, b): G_ab(beta) = exp(-i beta (X_a X_b + Y_a Y_b) / 2).
  (X_a X_b + Y_a Y_b) / 2 swaps |..0_a..1_b..> and |..1_a..0_b..> and annihilates
  the states with z_a = z_b, so G_ab keeps popcount(z).
* Ring XY mixer in parity order: the ring pairs (j, j+1 mod n) split into sets of
  disjoint pairs, applied set after set: even j (j < n - 1), then odd j (j < n - 1),
  then the closing pair (n-1, 0) alone when n is odd (for even n it belongs to the
  odd set).  n = 2 has the single pair (0, 1); n = 1 has none.

Everything below works on full 2**n vectors, so the restriction to F_k is a
check of the method, not an assumption of the code.
"""
from __future__ import annotations

from math import comb

import numpy as np


def feasible_states(n: int, k: int) -> np.ndarray:
    """F_k in rank order: every z in [0, 2**n) with popcount k, increasing."""
    z = np.arange(1 << n, dtype=np.int64)
    pop = np.zeros(1 << n, dtype=np.int64)
    for j in range(n):
        pop += (z >> j) & 1
    return z[pop == k]


def state_of_rank(n: int, k: int, r: int) -> int:
    """The state of F_k with rank r, one at a time (for sizes too large to enumerate):
    in the combinatorial number system r = sum_i binom(c_i, i), the top set bit c_k is the
    largest c with binom(c, k) <= r, and the rest is the state of rank r - binom(c_k, k)
    among k - 1 bits below it."""
    z, c = 0, n - 1
    for i in range(k, 0, -1):
        while comb(c, i) > r:
            c -= 1
        z |= 1 << c
        r -= comb(c, i)
        c -= 1
    return z


def subspace_dim(n: int, k: int) -> int:
    return comb(n, k) if 0 <= k <= n else 0


def ring_pair_sets(n: int):
    """The parity sets of the ring XY mixer, in application order."""
    if n < 2:
        return []
    if n == 2:
        return [[(0, 1)]]
    even = [(j, j + 1) for j in range(0, n - 1, 2)]
    odd = [(j, j + 1) for j in range(1, n - 1, 2)]
    if n % 2 == 0:
        return [even, odd + [(n - 1, 0)]]
    return [even, odd, [(n - 1, 0)]]


def apply_pair_gate(psi: np.ndarray, n: int, a: int, b: int, beta: float) -> np.ndarray:
    """G_ab(beta) on a full 2**n state: on the pair (z with z_a = 1, z_b = 0, and
    z' = z with both bits flipped) exp(-i beta K) = cos(beta) I - i sin(beta) K, K the
    swap of the two; states with z_a = z_b are unchanged."""
    out = psi.copy()
    c, s = np.cos(beta), np.sin(beta)
    z = np.arange(1 << n, dtype=np.int64)
    own = (((z >> a) & 1) == 1) & (((z >> b) & 1) == 0)
    zs = z[own]
    zp = zs ^ (1 << a) ^ (1 << b)
    out[zs] = c * psi[zs] - 1j * s * psi[zp]
    out[zp] = c * psi[zp] - 1j * s * psi[zs]
    return out


def apply_xy_mixer(psi: np.ndarray, n: int, beta: float) -> np.ndarray:
    for pair_set in ring_pair_sets(n):
        for a, b in pair_set:
            psi = apply_pair_gate(psi, n, a, b, beta)
    return psi


def dicke_state(n: int, k: int) -> np.ndarray:
    """Uniform superposition over F_k, as a full 2**n vector."""
    psi = np.zeros(1 << n, dtype=np.complex128)
    fk = feasible_states(n, k)
    psi[fk] = 1.0 / np.sqrt(len(fk))
    return psi


def xy_state(n: int, k: int, C: np.ndarray, gammas, betas, psi0: np.ndarray | None = None) -> np.ndarray:
    """Full 2**n state after p layers: U_XY(b_p) U_C(g_p) ... U_XY(b_1) U_C(g_1) psi0,
    psi0 the Dicke state over F_k unless given."""
    psi = dicke_state(n, k) if psi0 is None else np.asarray(psi0, dtype=np.complex128).copy()
    for g, b in zip(gammas, betas):
        psi = psi * np.exp(-1j * g * np.asarray(C, dtype=np.float64))
        psi = apply_xy_mixer(psi, n, b)
    return psi


def restrict(psi: np.ndarray, n: int, k: int) -> np.ndarray:
    """The amplitudes of F_k in rank order."""
    return psi[feasible_states(n, k)]


def subspace_costs(C: np.ndarray, n: int, k: int) -> np.ndarray:
    """C(z) for z in F_k, in rank order."""
    return np.asarray(C)[feasible_states(n, k)]


def xy_expectation(psi_sub: np.ndarray, C_sub: np.ndarray):
    """[<C>, <psi|psi>] of a subspace state (rank order)."""
    pr = np.abs(psi_sub) ** 2
    return float(np.sum(np.asarray(C_sub, dtype=np.float64) * pr)), float(np.sum(pr))


def xy_sample(psi_sub: np.ndarray, n: int, k: int, C_sub: np.ndarray, u: np.ndarray):
    """Inverse-CDF sampling (Sec. IV-D) of a subspace state: r_i = min{r : P(r) > u_i P_total}
    with P the inclusive running sum of |psi_r|**2 in rank order, the last rank with nonzero
    probability when rounding puts the target at or past the end.  Rank order is increasing
    z, so this is the full-space rule applied to the state embedded in 2**n amplitudes (the
    zeros off F_k add nothing to the running sum).  Returns (z uint64 of rank r_i, C_sub[r_i])."""
    prob = psi_sub.real ** 2 + psi_sub.imag ** 2
    P = np.cumsum(prob)
    total = P[-1]
    r = np.searchsorted(P, np.asarray(u, dtype=np.float64) * total, side="right")
    nz = np.nonzero(prob > 0)[0]
    last = nz[-1] if len(nz) else len(prob) - 1
    r = np.minimum(r, last)
    states = feasible_states(n, k)
    return states[r].astype(np.uint64), np.asarray(C_sub, dtype=np.float64)[r]


def xy_adjoint_gradient(n: int, k: int, C: np.ndarray, gammas, betas):
    """[E, dE/dgamma_1..p, dE/dbeta_1..p] of E = <psi|C|psi> for the subspace QAOA above.

    The circuit is a sequence of gates exp(-i theta H_g): per layer the cost unitary
    (H = diag(C), theta = gamma_l), then every ring pair gate in order (H = K_ab, the
    swap of z_a = 1, z_b = 0 with its partner, theta = beta_l).  For gate g with state
    psi_g right after it and lambda_g = (gates after g)^dagger C psi_final,
    dE/dtheta_g = 2 Im <lambda_g | H_g | psi_g>; a parameter's derivative sums over its
    gates.  psi_g is recovered by undoing the later gates (exp(+i theta H_g)).
    """
    Cf = np.asarray(C, dtype=np.float64)
    psi = xy_state(n, k, Cf, gammas, betas)
    E = float(np.real(np.vdot(psi, Cf * psi)))
    lam = Cf * psi
    p = len(gammas)
    dg, db = np.zeros(p), np.zeros(p)
    z = np.arange(1 << n, dtype=np.int64)
    for l in range(p - 1, -1, -1):
        for pair_set in reversed(ring_pair_sets(n)):
            for a, b in reversed(pair_set):
                own = (((z >> a) & 1) == 1) & (((z >> b) & 1) == 0)
                kpsi = np.zeros_like(psi)
                zs = z[own]
                zp = zs ^ (1 << a) ^ (1 << b)
                kpsi[zs], kpsi[zp] = psi[zp], psi[zs]
                db[l] += 2.0 * np.imag(np.vdot(lam, kpsi))
                psi = apply_pair_gate(psi, n, a, b, -betas[l])
                lam = apply_pair_gate(lam, n, a, b, -betas[l])
        dg[l] = 2.0 * np.imag(np.vdot(lam, Cf * psi))
        psi = psi * np.exp(1j * gammas[l] * Cf)
        lam = lam * np.exp(1j * gammas[l] * Cf)
    return E, dg, db
