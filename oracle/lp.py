"""The LP solved at one iteration of adaptive LP decoding, in augmented form
(oracle).

Eq. 10 (Section III-A) states the LP as: minimize gamma'u subject to
A u <= b (one parity inequality per check in the cut set, by Theorem 3),
u_i >= 0 for gamma_i >= 0 and u_i <= 1 for gamma_i < 0.

Section IV-B converts it to the augmented primal form of Eq. 16
(minimize c'x subject to A x = b, x >= 0) in two steps:
  1. x_i = u_i, c_i = gamma_i where gamma_i >= 0; x_i = 1 - u_i,
     c_i = -gamma_i where gamma_i < 0 ("flipped" bits). Every box
     constraint becomes x_i >= 0 and the parity coefficients change sign on
     the flipped bits.
  2. Each parity inequality A_j x <= b_j gets a slack column n+j with
     coefficient +1 and cost 0: A_j x + x_{n+j} = b_j. q = n + p.

For the cut of check j with odd set V (Eq. 5 form):
    sum_{i in V} u_i - sum_{i in N(j) minus V} u_i <= |V| - 1.
With s_i = +1 for i in V and -1 otherwise, substituting u_i = 1 - x_i on the
flipped bits gives coefficient a_{j,i} = s_i (unflipped) or -s_i (flipped)
and right side b_j = |V| - 1 - sum_{flipped i in N(j)} s_i.

The LP rows are the checks of the cut set in increasing check order.
"""

from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class AugmentedLP:
    A: np.ndarray          # dense p x q (float64), slack block = identity
    b: np.ndarray          # [p]
    c: np.ndarray          # [q]
    rows: np.ndarray       # [p] check index of each LP row
    flip: np.ndarray       # [n] bool, gamma_i < 0
    n: int

    @property
    def p(self) -> int:
        return self.A.shape[0]

    @property
    def q(self) -> int:
        return self.A.shape[1]

    def u_from_x(self, x: np.ndarray) -> np.ndarray:
        xs = x[:self.n]
        return np.where(self.flip, 1.0 - xs, xs)

    def objective_u(self, x: np.ndarray, gamma: np.ndarray) -> float:
        return float(np.dot(gamma, self.u_from_x(x)))


def build(code, gamma: np.ndarray, in_lp: np.ndarray, masks: np.ndarray) -> AugmentedLP:
    """Augmented LP (Eq. 16) of the cut set {(j, masks[j]) : in_lp[j]}, one
    row per check in increasing check order (MALP-A / MALP-B)."""
    rows = np.flatnonzero(in_lp)
    return build_from_cuts(code, gamma, [(int(j), int(masks[j])) for j in rows])


def build_from_cuts(code, gamma: np.ndarray, cuts) -> AugmentedLP:
    """Augmented LP (Eq. 16) of an ordered list of cuts (check j, mask of V).
    A check may appear more than once (ALP, Algorithm 1)."""
    n = code.n
    gamma = np.asarray(gamma, dtype=np.float64)
    flip = gamma < 0
    p = len(cuts)
    q = n + p
    A = np.zeros((p, q))
    b = np.zeros(p)
    for r, (j, mask) in enumerate(cuts):
        nbrs = code.row(j)
        size_v = 0
        rhs_shift = 0.0
        for e, i in enumerate(nbrs):
            s = 1.0 if (mask >> e) & 1 else -1.0
            size_v += int(s > 0)
            if flip[i]:
                A[r, i] = -s
                rhs_shift += s
            else:
                A[r, i] = s
        A[r, n + r] = 1.0
        b[r] = size_v - 1 - rhs_shift
    c = np.concatenate([np.abs(gamma), np.zeros(p)])
    return AugmentedLP(A=A, b=b, c=c,
                       rows=np.asarray([j for j, _ in cuts], dtype=np.int64),
                       flip=flip, n=n)
