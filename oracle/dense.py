"""Dense-matrix QAOA for n <= 6 (test infrastructure, not the product).

Builds the full 2**n x 2**n operators H_C = diag(C) (Sec. II-A) and
B = sum_j X_j (H_M = -B, Sec. II-A) and exponentiates them with
``scipy.linalg.expm``.  This is Eq. 1 taken literally, without the
one-qubit-at-a-time factorisation the simulators use, so it checks that
factorisation.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import expm

_X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_I = np.eye(2, dtype=np.complex128)


def x_on(n: int, j: int) -> np.ndarray:
    """X acting on qubit j (bit j of the index) as a dense 2**n x 2**n matrix."""
    out = np.ones((1, 1), dtype=np.complex128)
    for k in range(n - 1, -1, -1):  # kron puts the most significant factor first
        out = np.kron(out, _X if k == j else _I)
    return out


def b_matrix(n: int) -> np.ndarray:
    return sum(x_on(n, j) for j in range(n))


def dense_state(n: int, C, gammas, betas, mixer_sign: int = 1) -> np.ndarray:
    """Eq. 1 with U_C = expm(-i g H_C), U_M = expm(-i s b B), s = mixer_sign."""
    if n > 6:
        raise ValueError("dense check is for n <= 6")
    HC = np.diag(np.asarray(C, dtype=np.float64)).astype(np.complex128)
    B = b_matrix(n)
    psi = np.full(1 << n, 2.0 ** (-n / 2), dtype=np.complex128)
    for g, b in zip(gammas, betas):
        psi = expm(-1j * g * HC) @ psi
        psi = expm(-1j * mixer_sign * b * B) @ psi
    return psi


def dense_expectation(n: int, C, gammas, betas, mixer_sign: int = 1) -> float:
    psi = dense_state(n, C, gammas, betas, mixer_sign)
    HC = np.diag(np.asarray(C, dtype=np.float64))
    return float(np.real(np.conj(psi) @ HC @ psi))


def dense_gradient(n: int, C, gammas, betas, mixer_sign: int = 1):
    """Exact dE/dgamma_l and dE/dbeta_l of Eq. 1 from dense matrices (forward mode).

    Each factor is expm(-i t G) with a fixed generator G, so its t-derivative is
    (-i G) expm(-i t G).  The state with factor l differentiated is
    d psi / d t_l = U_p ... U_(l+1) (-i G_l) U_l ... U_1 |+>, and
    dE/dt_l = 2 Re <psi| H_C |d psi / d t_l>.  No adjoint recursion and no
    uncompute: an independent route to the gradient of Sec. II-B, IV-C.
    """
    if n > 6:
        raise ValueError("dense check is for n <= 6")
    HC = np.diag(np.asarray(C, dtype=np.float64)).astype(np.complex128)
    B = b_matrix(n)
    factors = []  # (generator, unitary) in application order
    for g, b in zip(gammas, betas):
        factors.append((HC, expm(-1j * g * HC)))
        factors.append((mixer_sign * B, expm(-1j * mixer_sign * b * B)))
    plus = np.full(1 << n, 2.0 ** (-n / 2), dtype=np.complex128)
    psi = plus.copy()
    for _, U in factors:
        psi = U @ psi
    grads = []
    for k in range(len(factors)):
        d = plus.copy()
        for j, (G, U) in enumerate(factors):
            d = U @ d
            if j == k:
                d = -1j * (G @ d)
        grads.append(2.0 * float(np.real(np.conj(psi) @ (HC @ d))))
    grads = np.array(grads)
    return grads[0::2], grads[1::2]
