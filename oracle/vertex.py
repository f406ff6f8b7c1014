"""Optimal vertex from the final interior-point iterate (oracle).

The decoder's decisions — is an inequality active (slack zero, Section
III-A), is a check violated (Algorithm 2), is the output integral (Section
II-B) — are statements about the exact LP solution, which Theorem 2 assumes
unique. A path-following iterate only approaches it: a nonbasic variable
still holds about mu / z_i, which is large when a reduced cost z_i is small,
and that error can exceed the margins the decisions need.

Section VI-A splits the columns at the optimum into the basic set
B = {i : x*_i > 0} and the nonbasic set N = {i : x*_i = 0}, and notes that
the unique solution is strictly complementary (x*_i > 0 = z*_i or
x*_i = 0 < z*_i). The final iterate (x, z) therefore reveals the partition:
i is basic iff x_i > z_i. Given the partition, the vertex is x*_N = 0 and
the solution of A_B x_B = b, which is unique because the basic columns of a
vertex are linearly independent. The oracle solves it as the minimum-norm
correction x_B + d with d = lstsq(A_B, b - A_B x_B).

The nonbasic entries are always set to zero. The corrected basic entries
replace the iterate's when the result is primal feasible (min x_B >= -tol
and ||A x - b||_inf <= tol) and its cost stays within cost_tol of the
iterate's; otherwise the iterate's basic entries are kept and the LP is
flagged.
"""

from __future__ import annotations

import numpy as np


def recover(A, b, c, x, z, tol: float = 1e-9, cost_tol: float = 1e-6):
    """Return (x_vertex, ok). ``ok`` is False when the partition x_i > z_i
    does not give a feasible vertex; ``x_vertex`` then holds the iterate's
    basic entries and zeros elsewhere."""
    A = np.asarray(A)
    basic = x > z
    AB = A[:, basic]
    r = b - AB @ x[basic]
    if AB.shape[1]:
        d = np.linalg.lstsq(AB, r, rcond=None)[0]
    else:
        d = np.zeros(0)
    xv = np.zeros_like(x)
    xv[basic] = x[basic] + d
    resid = float(np.max(np.abs(A @ xv - b))) if b.size else 0.0
    feasible = (AB.shape[1] == 0 or float(np.min(xv[basic])) >= -tol) and resid <= tol
    cost_ok = abs(float(c @ xv) - float(c @ x)) <= cost_tol * (1.0 + abs(float(c @ x)))
    if feasible and cost_ok:
        return xv, True
    xv[basic] = x[basic]
    return xv, False
