"""The combinatorial-number-system identities the subspace kernels rely on, checked
against the oracle's enumeration of F_k (no GPU): greedy unranking, Gosper's
next-equal-popcount rule walking F_k in rank order, and the rank offset binom(a, j)
between a state and its partner under an adjacent pair gate."""
from __future__ import annotations

from math import comb

import pytest

from oracle import xy as ox


def gosper_next(z: int) -> int:
    t = z | (z - 1)
    return (t + 1) | (((~t & (t + 1)) - 1) >> ((z & -z).bit_length()))


@pytest.mark.parametrize("n", [2, 5, 9, 12])
def test_gosper_walks_the_subspace_in_rank_order(n):
    for k in range(1, n + 1):
        fk = [int(z) for z in ox.feasible_states(n, k)]
        z = fk[0]
        for r in range(1, len(fk)):
            z = gosper_next(z)
            assert z == fk[r]


@pytest.mark.parametrize("n", [3, 6, 10, 13])
def test_adjacent_partner_rank_offset(n):
    # moving the set bit at a up to a + 1 raises the rank by binom(a, j), j = set bits below a
    for k in range(1, n):
        fk = [int(z) for z in ox.feasible_states(n, k)]
        rank = {z: r for r, z in enumerate(fk)}
        for a in range(n - 1):
            for r, z in enumerate(fk):
                if (z >> a) & 1 and not (z >> (a + 1)) & 1:
                    j = bin(z & ((1 << a) - 1)).count("1")
                    assert rank[z ^ (3 << a)] == r + comb(a, j)


@pytest.mark.parametrize("n,k", [(1, 0), (1, 1), (7, 3), (11, 5), (14, 13)])
def test_unrank_by_largest_binomial(n, k):
    fk = [int(z) for z in ox.feasible_states(n, k)]
    for r, z in enumerate(fk):
        # the top set bit of the state of rank r is the largest c with binom(c, k) <= r
        if k > 0:
            top = max(c for c in range(n) if comb(c, k) <= r)
            assert z.bit_length() - 1 == top
        assert ox.state_of_rank(n, k, r) == z
