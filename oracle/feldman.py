"""Plain definitions the adaptive decoder must reproduce (oracle).

* LP decoding (Eq. 7, Section II-B): minimize gamma'u over the fundamental
  polytope P, described by every parity inequality of Eq. 5 (all odd-sized
  V subset of N(j), 2^(d_j - 1) per check) and the box 0 <= u <= 1. Solved
  with scipy's HiGHS dual simplex, a library LP solver that shares nothing
  with the interior-point oracle. Theorem 2(c) states that ALP, MALP-A and
  MALP-B all end at this solution.
* ML decoding (Eq. 3): minimize gamma'u over the codewords, by enumerating
  ker(H) over GF(2). The ML certificate property (Section II-B) says an
  integral LP decoding output is this codeword.
"""

from __future__ import annotations

import itertools

import numpy as np
from scipy.optimize import linprog


def parity_inequalities(code):
    """Rows (coefficients over u) and right sides of Eq. 5 for every check
    and every odd subset V of its neighbourhood."""
    rows, rhs = [], []
    for j in range(code.m):
        nbrs = code.row(j)
        d = nbrs.size
        for size in range(1, d + 1, 2):
            for V in itertools.combinations(range(d), size):
                a = np.zeros(code.n)
                a[nbrs] = -1.0
                a[nbrs[list(V)]] = 1.0
                rows.append(a)
                rhs.append(size - 1.0)
    return np.asarray(rows), np.asarray(rhs)


def parity_inequalities_sparse(code):
    """The rows of ``parity_inequalities`` as a scipy CSR matrix (codes whose
    dense inequality matrix would not fit memory, e.g. n = 16000)."""
    import scipy.sparse as sp
    indptr, indices, data, rhs = [0], [], [], []
    for j in range(code.m):
        nbrs = code.row(j)
        d = nbrs.size
        for size in range(1, d + 1, 2):
            for V in itertools.combinations(range(d), size):
                sgn = -np.ones(d)
                sgn[list(V)] = 1.0
                indices.extend(nbrs.tolist())
                data.extend(sgn.tolist())
                indptr.append(len(indices))
                rhs.append(size - 1.0)
    A = sp.csr_matrix((np.asarray(data), np.asarray(indices), np.asarray(indptr)),
                      shape=(len(rhs), code.n))
    return A, np.asarray(rhs)


def lp_decode_sparse(code, gamma):
    """Full LP decoding (Eq. 7) with a sparse constraint matrix. Returns
    (u, objective)."""
    A, b = parity_inequalities_sparse(code)
    res = linprog(np.asarray(gamma, dtype=np.float64), A_ub=A, b_ub=b,
                  bounds=(0.0, 1.0), method="highs-ds")
    if res.status != 0:
        raise RuntimeError(f"linprog failed: {res.message}")
    return res.x, float(res.fun)


def lp_decode(code, gamma):
    """Full LP decoding (Eq. 7). Returns (u, objective)."""
    A, b = parity_inequalities(code)
    res = linprog(np.asarray(gamma, dtype=np.float64), A_ub=A, b_ub=b,
                  bounds=(0.0, 1.0), method="highs-ds")
    if res.status != 0:
        raise RuntimeError(f"linprog failed: {res.message}")
    return res.x, float(res.fun)


def gf2_nullspace(H) -> np.ndarray:
    """Rows spanning {u : H u = 0 mod 2}, by Gauss-Jordan elimination."""
    A = (np.asarray(H) & 1).astype(np.uint8).copy()
    m, n = A.shape
    pivots = []
    r = 0
    for col in range(n):
        if r >= m:
            break
        nz = np.flatnonzero(A[r:, col])
        if nz.size == 0:
            continue
        piv = r + nz[0]
        A[[r, piv]] = A[[piv, r]]
        others = np.flatnonzero(A[:, col])
        others = others[others != r]
        A[others] ^= A[r]
        pivots.append(col)
        r += 1
    free = [col for col in range(n) if col not in set(pivots)]
    basis = np.zeros((len(free), n), dtype=np.uint8)
    for t, f in enumerate(free):
        basis[t, f] = 1
        for i, pc in enumerate(pivots):
            basis[t, pc] = A[i, f]
    return basis


def codewords(code, max_dim: int = 20) -> np.ndarray:
    B = gf2_nullspace(code.dense())
    k = B.shape[0]
    if k > max_dim:
        raise ValueError(f"code dimension {k} too large to enumerate")
    coef = ((np.arange(2 ** k)[:, None] >> np.arange(k)[None, :]) & 1).astype(np.uint8)
    return (coef @ B % 2).astype(np.uint8)


def ml_decode(code, gamma):
    """Exhaustive ML decoding (Eq. 3). Returns (codeword, cost)."""
    C = codewords(code)
    cost = C.astype(np.float64) @ np.asarray(gamma, dtype=np.float64)
    best = int(np.argmin(cost))
    return C[best], float(cost[best])
