"""Closed-form depth-1 weighted-MaxCut expectation (test infrastructure, not the product).

For p = 1 the QAOA expectation of C = sum_uv w_uv (1 - Z_u Z_v)/2 has a known
analytic form (the light-cone result for one layer; see e.g. Ozaeta, van Dam,
McMahon, "Expectation values from the single-layer quantum approximate
optimization algorithm on Ising problems", 2022).  With the conventions of
this repository (psi_z *= exp(-i g C(z)), mixer RX(2b) on every qubit, so the
paper's Eq. 1 with its mixer sign flipped), for an edge (u, v) and products
over the other vertices k (w_xk = 0 where there is no edge):

  <Z_u Z_v> = -1/2 sin(4b) sin(g w_uv) [prod_k cos(g w_uk) + prod_k cos(g w_vk)]
              -1/2 sin(2b)^2 [prod_k cos(g (w_uk + w_vk)) - prod_k cos(g (w_uk - w_vk))]

and <C> = sum_uv w_uv (1 - <Z_u Z_v>) / 2.  It needs O(n m) work, so it pins
the simulated <C> at any n, including sizes no CPU statevector reaches.
``gradient_p1_exact`` differentiates the same form analytically in (g, b), which
pins the adjoint gradient (Sec. II-B, IV-C) at any n as well.
"""
from __future__ import annotations

import numpy as np


def _adjacency(n: int, edges, weights) -> np.ndarray:
    A = np.zeros((n, n), dtype=np.float64)
    for (u, v), w in zip(np.asarray(edges).reshape(-1, 2), weights):
        A[u, v] += w
        A[v, u] += w
    return A


def zz_p1(n: int, edges, weights, gamma: float, beta: float) -> np.ndarray:
    """<Z_u Z_v> after one layer, one value per edge, in edge-list order."""
    edges = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    w = np.ones(len(edges)) if weights is None else np.asarray(weights, dtype=np.float64)
    A = _adjacency(n, edges, w)
    out = np.zeros(len(edges))
    for e, (u, v) in enumerate(edges):
        others = [k for k in range(n) if k != u and k != v]
        au, av = A[u, others], A[v, others]
        t1 = np.prod(np.cos(gamma * au)) + np.prod(np.cos(gamma * av))
        t2 = np.prod(np.cos(gamma * (au + av))) - np.prod(np.cos(gamma * (au - av)))
        out[e] = (-0.5 * np.sin(4 * beta) * np.sin(gamma * A[u, v]) * t1
                  - 0.5 * np.sin(2 * beta) ** 2 * t2)
    return out


def expectation_p1(n: int, edges, weights, gamma: float, beta: float) -> float:
    """<C> after one layer from the per-edge closed form."""
    edges = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    w = np.ones(len(edges)) if weights is None else np.asarray(weights, dtype=np.float64)
    zz = zz_p1(n, edges, w, gamma, beta)
    return float(np.sum(w * (1.0 - zz) / 2.0))


def gradient_p1(n: int, edges, weights, gamma: float, beta: float, h: float = 1e-5):
    """(d<C>/dgamma, d<C>/dbeta) of the closed form by central differences."""
    f = lambda g, b: expectation_p1(n, edges, weights, g, b)
    return ((f(gamma + h, beta) - f(gamma - h, beta)) / (2 * h),
            (f(gamma, beta + h) - f(gamma, beta - h)) / (2 * h))


def _cos_product_and_derivative(gamma: float, c: np.ndarray):
    """prod_k cos(gamma c_k) and its gamma-derivative sum_j -c_j sin(gamma c_j) prod_{k != j} cos(gamma c_k).

    The derivative is summed term by term (no division by a cosine, which may be 0).
    """
    cs = np.cos(gamma * c)
    prod = float(np.prod(cs))
    deriv = 0.0
    for j in range(len(c)):
        deriv += -c[j] * np.sin(gamma * c[j]) * float(np.prod(np.delete(cs, j)))
    return prod, deriv


def gradient_p1_exact(n: int, edges, weights, gamma: float, beta: float):
    """(d<C>/dgamma, d<C>/dbeta) after one layer, differentiated analytically.

    With s4 = sin(4b), q = sin(2b)^2, T1 = prod cos(g w_uk) + prod cos(g w_vk) and
    T2 = prod cos(g (w_uk + w_vk)) - prod cos(g (w_uk - w_vk)), the per-edge form is
    <Z_u Z_v> = -1/2 s4 sin(g w_uv) T1 - 1/2 q T2, so
      d<ZZ>/db = -2 cos(4b) sin(g w_uv) T1 - sin(4b) T2            (dq/db = 2 sin(4b))
      d<ZZ>/dg = -1/2 s4 (w_uv cos(g w_uv) T1 + sin(g w_uv) T1') - 1/2 q T2'
    with T1', T2' the derivatives of the cosine products, and
    d<C>/dt = sum_uv w_uv (-1/2) d<Z_u Z_v>/dt.  O(m n^2) work, any n.
    """
    edges = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    w = np.ones(len(edges)) if weights is None else np.asarray(weights, dtype=np.float64)
    A = _adjacency(n, edges, w)
    s4, c4 = np.sin(4 * beta), np.cos(4 * beta)
    q = np.sin(2 * beta) ** 2
    dE_dg = 0.0
    dE_db = 0.0
    for e, (u, v) in enumerate(edges):
        others = [k for k in range(n) if k != u and k != v]
        au, av = A[u, others], A[v, others]
        wuv = A[u, v]
        pu, dpu = _cos_product_and_derivative(gamma, au)
        pv, dpv = _cos_product_and_derivative(gamma, av)
        pp, dpp = _cos_product_and_derivative(gamma, au + av)
        pm, dpm = _cos_product_and_derivative(gamma, au - av)
        T1, dT1 = pu + pv, dpu + dpv
        T2, dT2 = pp - pm, dpp - dpm
        sg, cg = np.sin(gamma * wuv), np.cos(gamma * wuv)
        dzz_db = -2.0 * c4 * sg * T1 - s4 * T2
        dzz_dg = -0.5 * s4 * (wuv * cg * T1 + sg * dT1) - 0.5 * q * dT2
        dE_dg += w[e] * (-0.5) * dzz_dg
        dE_db += w[e] * (-0.5) * dzz_db
    return float(dE_dg), float(dE_db)
