"""FP64 CPU oracle for MaxCut QAOA — test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg (and its ``--impl reference`` arm) may import this package.  The CUDA path
never does; the two share no code.  Parity status of each function:

* ``qaoa.cut_values``: pinned (brute-force known max cuts, Eq. 3 PUBO form,
  complement symmetry, sum over z equals W 2**(n-1)).
* ``qaoa.qaoa_state`` / ``expectation`` / ``norm2``: pinned (dense expm for
  n <= 6, p = 1 closed form, uniform-state identities, norm, flip symmetry,
  beta + pi/2 invariance).
* ``qaoa.sample``: pinned (deterministic cases, chi-square against |psi|^2).
* ``qaoa.adjoint_gradient``: pinned (central finite differences, derivative
  of the p = 1 closed form, uncompute returns |+>).
* ``closed_form.expectation_p1``: pinned against ``dense.dense_expectation``.
* ``dense.dense_state``: pinned (unitarity, H_C = diag, B spectrum).
"""
from . import qaoa, dense, closed_form  # noqa: F401
