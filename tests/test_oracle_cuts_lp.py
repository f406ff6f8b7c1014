"""Pins for the oracle's cut search (Algorithm 2) and LP construction
(Eqs. 10 and 16): brute force over every odd subset, Theorem 1, and the
equivalence of the augmented rows with the parity inequalities they encode.
"""

import itertools

import numpy as np
import pytest

from oracle import cuts, lp
from synth import named_code


def brute_min_odd(u):
    """Minimum of the left side of Eq. 6 over every odd V (plain loop)."""
    d = len(u)
    best, best_mask, all_lhs = np.inf, None, []
    for size in range(1, d + 1, 2):
        for V in itertools.combinations(range(d), size):
            s = sum((1 - u[e]) if e in V else u[e] for e in range(d))
            mask = sum(1 << e for e in V)
            all_lhs.append((s, mask))
            if s < best:
                best, best_mask = s, mask
    return best, best_mask, all_lhs


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5, 6, 7, 8])
def test_alg2_finds_minimum_odd_set(d):
    rng = np.random.default_rng(100 + d)
    for _ in range(300):
        u = rng.random(d)
        mask, lhs, violated = cuts.find_violated(u, 0.0)
        best, best_mask, all_lhs = brute_min_odd(u)
        assert abs(lhs - best) < 1e-12
        assert violated == (best < 1.0)
        if violated:
            assert mask == best_mask
            # Theorem 1: every other odd set is strictly satisfied
            others = [s for s, mk in all_lhs if mk != mask]
            assert all(s > 1.0 for s in others)
        assert cuts.popcount(mask) % 2 == 1


def test_alg2_integral_points():
    rng = np.random.default_rng(7)
    for _ in range(200):
        d = int(rng.integers(2, 9))
        u = rng.integers(0, 2, d).astype(float)
        mask, lhs, violated = cuts.find_violated(u, 1e-9)
        if int(u.sum()) % 2 == 0:
            # a satisfied check: the best odd set is tight, LHS exactly 1
            assert not violated and lhs == 1.0
        else:
            # odd parity: V = S gives LHS 0 (Section II-B equivalence)
            assert violated and lhs == 0.0
            assert mask == sum(1 << e for e in range(d) if u[e] == 1)


def test_alg2_tie_breaks_to_lowest_position():
    u = np.array([0.5, 0.5, 0.0, 0.0])
    mask, lhs, _ = cuts.find_violated(u, 0.0)
    assert mask == 0b0001 and lhs == 1.0


def test_augmented_rows_encode_parity_inequalities():
    code = named_code("gallager_120")
    rng = np.random.default_rng(3)
    for _ in range(20):
        gamma = rng.normal(size=code.n) * 3
        in_lp = rng.random(code.m) < 0.5
        masks = np.zeros(code.m, dtype=np.uint32)
        for j in range(code.m):
            d = code.row(j).size
            V = rng.random(d) < 0.5
            if V.sum() % 2 == 0:
                V[0] = ~V[0]
            masks[j] = sum(1 << e for e in range(d) if V[e])
        L = lp.build(code, gamma, in_lp, masks)
        u = rng.random(code.n)
        x = np.where(gamma < 0, 1 - u, u)
        for r, j in enumerate(L.rows):
            nbrs = code.row(j)
            inV = np.array([(int(masks[j]) >> e) & 1 for e in range(nbrs.size)], bool)
            # Eq. 5: sum_V u - sum_{N\V} u <= |V| - 1 ; slack = rhs - lhs
            slack = (inV.sum() - 1) - (u[nbrs[inV]].sum() - u[nbrs[~inV]].sum())
            assert abs(L.b[r] - L.A[r, :code.n] @ x - slack) < 1e-12
            assert L.A[r, code.n + r] == 1.0
        # cost: c'x = gamma'u - sum_{gamma<0} gamma
        assert abs(L.c[:code.n] @ x - (gamma @ u - gamma[gamma < 0].sum())) < 1e-9
        assert np.all(L.c >= 0)
