"""Parity inequalities and the per-check cut search (oracle).

Section II-B: for check j with neighbourhood N(j) and every odd-sized
V subset of N(j), the parity inequality in its second form (Eq. 6) reads

    sum_{i in V} (1 - u_i) + sum_{i in N(j) minus V} u_i  >=  1.

A set V is stored as a bit mask over the positions of N(j) in the row's
column order: bit e set <=> the e-th neighbour of j is in V.

Algorithm 2 (Section III) finds the only inequality of check j that can be
violated at u (Theorem 1): S = {i in N(j) : u_i > 1/2}; if |S| is odd V = S,
otherwise the neighbour i* closest to 1/2 is toggled in or out of S. The
paper does not say how to break a tie in the argmin; the oracle takes the
lowest neighbour position. The check is violated when the left side of Eq. 6
is below 1 - tau_cut.
"""

from __future__ import annotations

import numpy as np


def parity_lhs(u_nbrs: np.ndarray, mask: int) -> float:
    """Left side of Eq. 6 for the set V given by ``mask`` over the neighbour
    values ``u_nbrs`` (in row order), summed in row order."""
    s = 0.0
    for e, ue in enumerate(u_nbrs):
        if (mask >> e) & 1:
            s += 1.0 - float(ue)
        else:
            s += float(ue)
    return s


def find_violated(u_nbrs: np.ndarray, tau_cut: float):
    """Algorithm 2 for one check.

    Returns (mask, lhs, violated): the odd set V chosen by the algorithm, the
    left side of Eq. 6 at u for that V, and whether lhs < 1 - tau_cut.
    """
    u_nbrs = np.asarray(u_nbrs, dtype=np.float64)
    d = u_nbrs.size
    mask = 0
    count = 0
    for e in range(d):
        if u_nbrs[e] > 0.5:          # S = {i : u_i > 1/2}
            mask |= 1 << e
            count += 1
    if count % 2 == 0:               # |S| even: toggle i* = argmin |u_i - 1/2|
        best = 0
        best_dist = abs(u_nbrs[0] - 0.5)
        for e in range(1, d):
            dist = abs(u_nbrs[e] - 0.5)
            if dist < best_dist:     # strict: ties keep the lowest position
                best, best_dist = e, dist
        mask ^= 1 << best
    lhs = parity_lhs(u_nbrs, mask)
    return mask, lhs, lhs < 1.0 - tau_cut


def popcount(x: int) -> int:
    return bin(int(x)).count("1")
