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
x*_i = 0 < z*_i). The final iterate (x, y, z) therefore reveals the
partition once it is close enough: i is basic iff x_i > z_i. Given the
partition:

  primal  x^_N = 0 and x^_B = x_B + d with d the minimum-norm solution of
          A_B d = b - A_B x_B (least squares);
  dual    y^ = y + e with e the minimum-norm solution of A_B' e = c_B - A_B' y,
          so that the reduced costs z^ = c - A' y^ vanish on B.

The pair is accepted as the LP's optimal vertex only with an optimality
certificate: x^ primal feasible (x^_B >= -tol, ||A x^ - b||_inf <= tol), z^
dual feasible on N (z^_N >= -tol (1 + max|c|)) and complementary
(|z^_B| <= tol (1 + max|c|)). Primal and dual feasibility with
complementarity prove x^ optimal, whatever the accuracy of the iterate.

When the certificate fails (the iterate has not separated the partition
yet), ``recover`` returns the iterate's basic entries with zeros elsewhere
and ok = False; the decoder then resumes the interior-point method with a
tighter gap tolerance.
"""

from __future__ import annotations

import numpy as np


def recover(A, b, c, x, z, y, tol: float = 1e-9):
    """Return (x_vertex, ok); ok means the vertex carries the optimality
    certificate above."""
    A = np.asarray(A)
    basic = x > z
    AB = A[:, basic]
    xv = np.zeros_like(x)
    if AB.shape[1]:
        d = np.linalg.lstsq(AB, b - AB @ x[basic], rcond=None)[0]
        e = np.linalg.lstsq(AB.T, c[basic] - AB.T @ y, rcond=None)[0]
        xv[basic] = x[basic] + d
        yh = y + e
    else:
        yh = y
    zh = c - A.T @ yh
    scale = 1.0 + float(np.max(np.abs(c))) if c.size else 1.0
    resid = float(np.max(np.abs(A @ xv - b))) if b.size else 0.0
    primal = (not AB.shape[1] or float(np.min(xv[basic])) >= -tol) and resid <= tol
    dual = (basic.all() or float(np.min(zh[~basic])) >= -tol * scale)
    compl = (not basic.any() or float(np.max(np.abs(zh[basic]))) <= tol * scale)
    if primal and dual and compl:
        return xv, True
    xv[basic] = x[basic]
    return xv, False
