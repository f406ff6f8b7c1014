"""Readings of the points the paper leaves open (oracle side).

Every field below is a rule or tolerance that the paper does not fix. The
CUDA library has its own copy of the same defaults (``lpdec_default_params``);
tests pass identical values to both sides explicitly.

  sigma     centering factor: mu = sigma * x'z / q. Eq. 28 states
            mu = x'z/q (sigma = 1), under which a feasible iterate's
            duality gap does not shrink; the path-following reading keeps
            the proportionality and scales it by sigma < 1.
  eta       fraction of the step to the boundary (Section IV-B asks only
            that x, z stay nonnegative): beta_P = min(1, eta * max step).
  tol_gap   stop when x'z / (1 + |c'x|) < tol_gap  (Section IV-B, end).
  tol_feas  ... and ||r_b||/(1+||b||) < tol_feas, ||r_c||/(1+||c||) < tol_feas;
            or, once the gap test holds, both below tol_feas_loose (the
            Newton solves lose accuracy as D^2 spreads near the optimum; the
            optimal vertex is recovered from the iterate either way).
  tol_pcg   PCG stops when ||w - Q dy||_2 / ||w||_2 < tol_pcg.
  tau_act   a cut is active iff its slack x_{n+j} <= tau_act (the paper's
            "slack variable is zero", Section III-A), read on the optimal
            vertex recovered from the final iterate (see ``vertex``).
  tau_cut   check j is violated iff the left side of Eq. 6 for the set V of
            Algorithm 2 is < 1 - tau_cut.
  tau_int   the output is integral iff max_i |u_i - round(u_i)| <= tau_int.
  tau_inc   Theorem 2(b): with unique LP optima the cost gamma'u^k rises
            strictly from one LP to the next, so no cut set repeats. When
            an LP's cost does not exceed the previous one by more than
            tau_inc * (1 + |previous cost|), that hypothesis has failed (a
            tie or a numerically non-unique optimum, where MALP can cycle
            between two cut sets without reaching the optimum) and the frame
            continues as ALP (Algorithm 1) from its current cut set.
  max_alp, max_ipm, max_pcg: iteration caps; reaching one ends the frame
            with status NOT_CONVERGED.
"""

from __future__ import annotations

import dataclasses

# frame status codes (same values as the C library's LPDEC_* codes)
OK = 0
NOT_CONVERGED = -3


@dataclasses.dataclass
class OracleParams:
    sigma: float = 0.1
    eta: float = 0.99
    tol_gap: float = 1e-8
    tol_feas: float = 1e-8
    tol_feas_loose: float = 1e-6
    tol_pcg: float = 1e-10
    tau_act: float = 1e-9
    tau_cut: float = 1e-9
    tau_int: float = 1e-9
    tau_inc: float = 1e-9
    max_alp: int = 200
    max_ipm: int = 60
    max_pcg: int = 1000
    variant: str = "malp_a"   # "malp_a" | "malp_b" | "alp"
