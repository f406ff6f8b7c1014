"""Adaptive LP decoding (oracle): MALP-A (Algorithm 3), MALP-B and ALP
(Algorithm 1).

MALP-A (Section III-A):
  1. The first LP holds only the one-sided box constraints of Eq. 8; its
     solution u^0 is the bitwise hard decision (u_i = 0 if gamma_i >= 0,
     else 1).
  2. Repeat: for every check j with no ACTIVE parity inequality in the
     current LP, run Algorithm 2 at u^{k-1}; if it finds a violated
     inequality, drop j's old (inactive) inequality, if any, and add the new
     one. If anything was added, solve the LP to get u^k. Stop when nothing
     was added; u^k is the LP decoding solution.
  Theorem 2(b) makes the cost gamma'u^k strictly increasing when every LP
  optimum is unique. When the cost does not rise (by more than tau_inc,
  relative), that hypothesis has failed: the optimum is not unique (or not
  numerically unique), and MALP's removal of inactive inequalities can then
  cycle between cut sets without reaching the LP decoding optimum. The frame
  then continues as ALP (Algorithm 1) from its current cut set: from there on
  nothing is removed and every check is searched. ALP only adds
  inequalities, so the cost cannot fall and no cut set repeats; it stops
  when no parity inequality is violated, i.e. at a point of the fundamental
  polytope that is optimal for a relaxation of it: the LP decoding optimum
  (Theorem 2(c) for ALP needs no uniqueness).
  MALP-B moves the removal to the start of the round: every inactive
  inequality is dropped before the search. ALP never removes anything and
  searches every check.

LP rows are the cut list ordered by check, and, within a check, by the
order in which its inequalities were added (a reordering of rows does not
change the LP).

An inequality is active when its slack x_{n+j} is zero (Section III-A). Each
LP is solved by ``ipm.solve`` on the augmented form of ``lp.build``; the
decisions are then taken on the optimal vertex recovered from the final
iterate (``vertex.recover``), where a nonbasic slack is exactly zero, so
"zero" is read as <= tau_act.

Outputs (Section II-B, ML certificate): the solution u, the certificate flag
(u is integral: max |u_i - round(u_i)| <= tau_int) and a hard decision. The
decoder declares failure on a fractional u and the paper defines no hard
decision for it; the oracle returns hard_i = [u_i > 1/2], except that an
entry within tau_int of 1/2 takes the channel's hard decision (so a 1/2 entry
does not turn on rounding noise).
"""

from __future__ import annotations

import dataclasses

import numpy as np

from . import cuts as _cuts
from . import ipm as _ipm
from . import lp as _lp
from . import vertex as _vertex
from .params import OracleParams, OK, NOT_CONVERGED


@dataclasses.dataclass
class LPRecord:
    p: int
    objective: float          # gamma'u^k
    ipm_iters: int
    u: np.ndarray
    in_lp: np.ndarray
    masks: np.ndarray
    slack: np.ndarray          # slack per LP row
    rows: np.ndarray


@dataclasses.dataclass
class DecodeResult:
    u: np.ndarray              # float64 [n]
    hard: np.ndarray           # uint8 [n]
    cert: int                  # 1 = integral (ML codeword), 0 = fractional
    in_lp: np.ndarray          # bool [m] final cut set
    masks: np.ndarray          # uint32 [m] (0 where not in the LP)
    alp_iters: int             # number of LPs solved
    ipm_iters_total: int
    lp_rows_final: int         # rows of the last LP solved (MALP-B drops
                               # inactive inequalities after it, Section III-A)
    objective: float           # gamma'u
    status: int
    history: list              # LPRecord per LP solved
    cuts: list                 # final cut list (ALP keeps several per check)
    vertex_failures: int = 0   # LPs whose vertex recovery was rejected
    alp_switch: int = 0        # LPs solved before a MALP frame continued as
                               # ALP (0: it never did)


def hard_decision(gamma: np.ndarray) -> np.ndarray:
    """u^0 of Eq. 8: 0 where gamma_i >= 0, 1 where gamma_i < 0."""
    return np.where(np.asarray(gamma) >= 0, 0.0, 1.0)


def outputs(u: np.ndarray, gamma: np.ndarray, tau_int: float):
    dist = np.abs(u - np.round(u))
    cert = int(np.max(dist) <= tau_int) if u.size else 1
    hard = (u > 0.5).astype(np.uint8)
    near_half = np.abs(u - 0.5) <= tau_int
    hard[near_half] = hard_decision(gamma)[near_half].astype(np.uint8)
    return hard, cert


def decode(code, gamma, params: OracleParams | None = None,
           solve_normal_factory=None) -> DecodeResult:
    """Decode one frame. ``solve_normal_factory(A)`` may replace the dense
    Cholesky Newton solve (e.g. by PCG) for experiments."""
    prm = params or OracleParams()
    gamma = np.asarray(gamma, dtype=np.float64)
    n, m = code.n, code.m
    u = hard_decision(gamma)
    cost = float(np.dot(gamma, u))      # gamma'u^0
    in_lp = np.zeros(m, dtype=bool)
    masks = np.zeros(m, dtype=np.uint32)   # V of check j's (latest) inequality
    slack = np.full(m, np.inf)         # least slack over check j's inequalities
    cuts = []                          # cut list (check, mask) in insertion order
    alp = prm.variant == "alp"         # ALP semantics (from the start, or after a stall)
    alp_switch = 0
    history = []
    status = OK
    ipm_total = 0
    lps = 0
    vfail = 0
    while True:
        flag = False
        if prm.variant == "malp_b" and not alp:
            drop = in_lp & (slack > prm.tau_act)
            in_lp[drop] = False
            masks[drop] = 0
        for j in range(m):
            if not alp and in_lp[j] and slack[j] <= prm.tau_act:
                continue                # j has an active inequality
            mask, lhs, violated = _cuts.find_violated(u[code.row(j)], prm.tau_cut)
            if violated:
                flag = True
                if alp:
                    cuts.append((j, mask))
                else:
                    cuts = [c for c in cuts if c[0] != j]   # replaces j's old inequality
                    cuts.append((j, mask))
                in_lp[j] = True
                masks[j] = mask
        if not alp:
            cuts = [c for c in cuts if in_lp[c[0]]]         # MALP-B drops
        if not flag:
            break
        if lps >= prm.max_alp:
            status = NOT_CONVERGED
            break
        order = sorted(range(len(cuts)), key=lambda t: (cuts[t][0], t))
        lp = _lp.build_from_cuts(code, gamma, [cuts[t] for t in order])
        solver = solve_normal_factory(lp.A) if solve_normal_factory else None
        res = _ipm.solve(lp.A, lp.b, lp.c, prm, solve_normal=solver)
        lps += 1
        ipm_total += res.iters
        xv, vok = _vertex.recover(lp.A, lp.b, lp.c, res.x, res.z, res.y)
        # an iterate that has not separated the optimal partition yet: resume
        # the method with a tighter gap until the vertex is certified optimal
        for scale in (1e-2, 1e-3):
            if vok or res.status != OK:
                break
            tight = dataclasses.replace(prm, tol_gap=prm.tol_gap * scale,
                                        max_ipm=2 * prm.max_ipm)
            res = _ipm.solve(lp.A, lp.b, lp.c, tight, solve_normal=solver)
            ipm_total += res.iters
            xv, vok = _vertex.recover(lp.A, lp.b, lp.c, res.x, res.z, res.y)
        vfail += int(not vok)
        u = lp.u_from_x(xv)
        s_rows = xv[n:]
        slack = np.full(m, np.inf)
        for r, j in enumerate(lp.rows):   # a check is active if any of its rows is
            slack[j] = min(slack[j], s_rows[r])
        history.append(LPRecord(p=lp.p, objective=float(np.dot(gamma, u)),
                                ipm_iters=res.iters, u=u.copy(),
                                in_lp=in_lp.copy(), masks=masks.copy(),
                                slack=s_rows.copy(), rows=lp.rows.copy()))
        if res.status != OK:
            status = NOT_CONVERGED
            break
        new_cost = history[-1].objective
        if not alp and new_cost - cost <= prm.tau_inc * (1.0 + abs(cost)):
            alp = True                  # Theorem 2(b) fails: continue as ALP
            alp_switch = lps
        cost = new_cost
    hard, cert = outputs(u, gamma, prm.tau_int)
    out_masks = np.where(in_lp, masks, 0).astype(np.uint32)
    order = sorted(range(len(cuts)), key=lambda t: (cuts[t][0], t))
    return DecodeResult(u=u, hard=hard, cert=cert, in_lp=in_lp.copy(),
                        masks=out_masks, alp_iters=lps,
                        ipm_iters_total=ipm_total,
                        lp_rows_final=history[-1].p if history else 0,
                        objective=float(np.dot(gamma, u)), status=status,
                        history=history, cuts=[cuts[t] for t in order],
                        vertex_failures=vfail, alp_switch=alp_switch)
