"""Infeasible primal-dual path-following interior-point method (oracle).

Follows Section IV-B step by step on the augmented LP (Eq. 16) and its dual
(Eq. 17; the paper prints "minimize b'y", the dual of a minimisation is a
maximisation of b'y subject to A'y + z = c, z >= 0):

  residuals   r_b = b - A x,  r_c = c - A'y - z,  r_e = mu e - X Z e   (Eq. 23)
  scaling     D^2 = X Z^{-1}                                             (Eq. 27)
  Newton      (A D^2 A') dy = r_b + A D^2 r_c - A Z^{-1} r_e             (Eq. 24)
              dx = D^2 A' dy - D^2 r_c + Z^{-1} r_e                      (Eq. 25)
              dz = X^{-1} (r_e - Z dx)                                   (Eq. 26)
  update      x += beta_P dx, y += beta_D dy, z += beta_D dz, with the step
              lengths in [0, 1] keeping x, z >= 0
  centering   mu = sigma * x'z / q                                       (Eq. 28)
  stop        x'z small and ||r_b||, ||r_c|| small (end of Section IV-B)

Readings (``OracleParams``): sigma = 0.1 scales Eq. 28; each step length is
min(1, eta * largest step to the boundary of its own cone); the infeasible
variant may start anywhere with x, z > 0, and the oracle starts every LP
cold at x = e, y = 0, z = c + e; the stopping tests are relative:
x'z/(1+|c'x|) < tol_gap with ||r_b||/(1+||b||) and ||r_c||/(1+||c||) both
below tol_feas (or both below tol_feas_loose).

The normal equations are solved by a dense Cholesky factorisation of
A D^2 A' (Section IV-C names it as the direct method), so this oracle does not
depend on PCG.
"""

from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg

from .params import OracleParams, OK, NOT_CONVERGED


@dataclasses.dataclass
class IPMResult:
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    iters: int
    status: int
    gap: float
    feas_p: float
    feas_d: float


def step_to_boundary(v: np.ndarray, dv: np.ndarray) -> float:
    """Largest t with v + t dv >= 0 (inf if dv >= 0 everywhere)."""
    neg = dv < 0
    if not np.any(neg):
        return np.inf
    return float(np.min(-v[neg] / dv[neg]))


def newton_direction(A, x, y, z, b, c, mu, solve_normal):
    """Eqs. 23-27: residuals, D^2, the normal-equation right side and the
    Newton direction; ``solve_normal(d2, w)`` returns dy with
    (A D^2 A') dy = w."""
    rb = b - A @ x
    rc = c - A.T @ y - z
    re = mu - x * z
    d2 = x / z
    w = rb + A @ (d2 * rc) - A @ (re / z)
    dy = solve_normal(d2, w)
    dx = d2 * (A.T @ dy) - d2 * rc + re / z
    dz = (re - z * dx) / x
    return dx, dy, dz, w, d2


def cholesky_normal_solver(A):
    """Direct solve of (A D^2 A') dy = w.

    The Cholesky factor R (R'R = A D^2 A') is taken as the triangular factor
    of a Householder QR decomposition of D A' (q x p), so A D^2 A' is never
    formed: near the optimum D^2 spans more than 1/eps and the formed matrix
    is numerically singular, while D A' has only the square root of its
    condition number. Then R' t = w and R dy = t.
    """
    def solve(d2, w):
        DAt = np.sqrt(d2)[:, None] * A.T
        R = scipy.linalg.qr(DAt, mode="r", check_finite=False)[0][:A.shape[0]]
        t = scipy.linalg.solve_triangular(R, w, trans="T", check_finite=False)
        return scipy.linalg.solve_triangular(R, t, check_finite=False)
    return solve


def convergence_measures(A, b, c, x, y, z):
    rb = b - A @ x
    rc = c - A.T @ y - z
    gap = float(np.dot(x, z)) / (1.0 + abs(float(np.dot(c, x))))
    fp = float(np.linalg.norm(rb)) / (1.0 + float(np.linalg.norm(b)))
    fd = float(np.linalg.norm(rc)) / (1.0 + float(np.linalg.norm(c)))
    return gap, fp, fd


def solve(A, b, c, params: OracleParams | None = None, solve_normal=None,
          trace=None) -> IPMResult:
    """Solve min c'x s.t. Ax = b, x >= 0 by the path-following method.

    ``solve_normal`` defaults to dense Cholesky. ``trace`` (a list) receives
    one dict per iteration when given.
    """
    prm = params or OracleParams()
    p, q = A.shape
    if solve_normal is None:
        solve_normal = cholesky_normal_solver(A)
    x = np.ones(q)
    y = np.zeros(p)
    z = c + 1.0
    status = NOT_CONVERGED
    it = 0
    gap = fp = fd = np.inf
    for it in range(prm.max_ipm + 1):
        gap, fp, fd = convergence_measures(A, b, c, x, y, z)
        if gap < prm.tol_gap and ((fp < prm.tol_feas and fd < prm.tol_feas) or
                                  (fp < prm.tol_feas_loose and fd < prm.tol_feas_loose)):
            status = OK
            break
        if it == prm.max_ipm:
            break
        mu = prm.sigma * float(np.dot(x, z)) / q
        dx, dy, dz, w, d2 = newton_direction(A, x, y, z, b, c, mu, solve_normal)
        beta_p = min(1.0, prm.eta * step_to_boundary(x, dx))
        beta_d = min(1.0, prm.eta * step_to_boundary(z, dz))
        if trace is not None:
            trace.append(dict(it=it, gap=gap, feas_p=fp, feas_d=fd, mu=mu,
                              beta_p=beta_p, beta_d=beta_d, d2=d2.copy(),
                              w=w.copy(), dy=dy.copy(), x=x.copy(), z=z.copy()))
        x = x + beta_p * dx
        y = y + beta_d * dy
        z = z + beta_d * dz
    return IPMResult(x=x, y=y, z=z, iters=it, status=status, gap=gap,
                     feas_p=fp, feas_d=fd)
