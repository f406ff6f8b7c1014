"""Seeded LDPC parity-check matrix constructions (input generation only).

A code is stored as a parity-check matrix H (m x n over GF(2)) in CSR form:
``row_ptr`` (int32, m+1) and ``col_idx`` (int32, E), columns of each row in
increasing order. The paper (Section II-A) describes a code by H and its
Tanner graph; the simulations of Sections III-D and VI-B use random
(3,6)-regular codes from which all cycles of length four are removed.

Constructions:
  * ``gallager_regular``: Gallager's stacked-permutation (dv,dc) ensemble,
    with an edge-swap repair that removes every 4-cycle.
  * ``peg_code`` / ``peg_regular``: progressive edge growth. Each new edge of
    a variable node goes to an available check node (degree below its target)
    that is farthest from the node in the current graph; ties go to the lowest
    current degree, then to a seeded random choice. This yields girth >= 6 at
    the sizes used here.
  * ``irregular_degrees``: variable-degree sequence from an edge-perspective
    degree distribution lambda(x) with a fixed check degree.
  * ``hamming74``: the 3 x 7 Hamming parity-check matrix with a chosen column
    order.
"""

from __future__ import annotations

import dataclasses
import functools

import numpy as np


@dataclasses.dataclass(frozen=True)
class Code:
    """Parity-check matrix H in CSR form (rows = checks, columns = bits)."""

    m: int
    n: int
    row_ptr: np.ndarray  # int32 [m+1]
    col_idx: np.ndarray  # int32 [E], sorted within each row
    name: str = ""

    @property
    def E(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def design_rate(self) -> float:
        return 1.0 - self.m / self.n

    def row(self, j: int) -> np.ndarray:
        return self.col_idx[self.row_ptr[j]:self.row_ptr[j + 1]]

    def dense(self) -> np.ndarray:
        H = np.zeros((self.m, self.n), dtype=np.uint8)
        for j in range(self.m):
            H[j, self.row(j)] = 1
        return H

    def check_degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)

    def var_degrees(self) -> np.ndarray:
        return np.bincount(self.col_idx, minlength=self.n)


def from_rows(rows, n: int, name: str = "") -> Code:
    m = len(rows)
    row_ptr = np.zeros(m + 1, dtype=np.int32)
    cols = []
    for j, r in enumerate(rows):
        r = sorted(int(v) for v in r)
        if len(set(r)) != len(r):
            raise ValueError(f"row {j} has a repeated column")
        cols.extend(r)
        row_ptr[j + 1] = len(cols)
    return Code(m=m, n=n, row_ptr=row_ptr,
                col_idx=np.asarray(cols, dtype=np.int32), name=name)


def from_dense(H, name: str = "") -> Code:
    H = np.asarray(H)
    return from_rows([np.flatnonzero(H[j]) for j in range(H.shape[0])],
                     H.shape[1], name=name)


# ---------------------------------------------------------------------------
# Gallager construction with 4-cycle removal
# ---------------------------------------------------------------------------

def _first_conflict(j, rows, var_checks):
    """Return (other_check, shared_var_a, shared_var_b) if check j shares two
    variables with another check (a 4-cycle), else None."""
    seen = {}
    for v in dict.fromkeys(rows[j]):
        for c in dict.fromkeys(var_checks[v]):
            if c == j:
                continue
            if c in seen:
                return c, seen[c], v
            seen[c] = v
    return None


def _repair_4cycles(rows, n, group_of, rng, dc_of):
    """Remove every 4-cycle (two checks sharing two bits) and repeated bit of
    a row by swapping a shared bit of an offending row with a random bit of
    another row of the same swap group (rows of group -1 are never changed)."""
    m = len(rows)
    var_checks = [[] for _ in range(n)]
    for j, r in enumerate(rows):
        for v in r:
            var_checks[v].append(j)
    groups = {}
    for j, g in enumerate(group_of):
        groups.setdefault(g, []).append(j)
    work = list(range(m))
    budget = 200 * m + 10000
    while work:
        budget -= 1
        if budget < 0:
            raise RuntimeError("4-cycle removal did not converge")
        j = work.pop()
        dup = len(set(rows[j])) != len(rows[j])
        if dup:
            seen = set()
            for v in rows[j]:
                if v in seen:
                    va = vb = v
                    break
                seen.add(v)
            c = j
        else:
            hit = _first_conflict(j, rows, var_checks)
            if hit is None:
                continue
            c, va, vb = hit
        row = j if group_of[j] >= group_of[c] else c
        if group_of[row] < 0:
            row = c if row == j else j
        g = groups[group_of[row]]
        v = va if rng.integers(2) == 0 else vb
        r3 = row
        while r3 == row:
            r3 = g[int(rng.integers(len(g)))]
        v3 = rows[r3][int(rng.integers(dc_of[r3]))]
        if v3 in rows[row] or v in rows[r3]:
            work.append(j)
            continue
        rows[row][rows[row].index(v)] = v3
        rows[r3][rows[r3].index(v3)] = v
        var_checks[v][var_checks[v].index(row)] = r3
        var_checks[v3][var_checks[v3].index(r3)] = row
        work.extend([j, c, row, r3])
    return rows


def gallager_regular(n: int, dv: int = 3, dc: int = 6, seed: int = 0,
                     name: str | None = None, remove_4cycles: bool = True) -> Code:
    """(dv,dc)-regular H with all 4-cycles removed (seeded).

    When dc divides n this is Gallager's ensemble: H stacks dv blocks of n/dc
    rows; block 0 has row r covering columns r*dc..r*dc+dc-1 and block b>0
    applies a random column permutation to block 0. Otherwise the n*dv bit
    sockets are randomly permuted onto the m*dc check sockets (m = n*dv/dc).
    4-cycles (two checks sharing two bits) and repeated bits are then removed
    by swapping a shared bit of the offending row (in a permuted block) with a
    random bit of another row of the same block, until none remains.
    ``remove_4cycles=False`` skips the repair (tiny codes, where girth 6 is
    impossible).
    """
    if (n * dv) % dc:
        raise ValueError("n*dv must be a multiple of dc")
    rng = np.random.default_rng([0x9A11A6E5, seed, n, dv, dc])
    m = n * dv // dc
    rows = []
    if n % dc == 0:
        mb = n // dc
        group_of = []
        for b in range(dv):
            perm = np.arange(n) if b == 0 else rng.permutation(n)
            for r in range(mb):
                rows.append([int(v) for v in perm[r * dc:(r + 1) * dc]])
                group_of.append(b if b > 0 else -1)
    else:
        sockets = rng.permutation(np.repeat(np.arange(n), dv))
        rows = [[int(v) for v in sockets[j * dc:(j + 1) * dc]] for j in range(m)]
        group_of = [0] * m
    if remove_4cycles:
        rows = _repair_4cycles(rows, n, group_of, rng, [dc] * m)
    return from_rows(rows, n, name=name or f"gallager({dv},{dc}) n={n} seed={seed}")


# ---------------------------------------------------------------------------
# Progressive edge growth
# ---------------------------------------------------------------------------

def peg_code(var_degrees, check_degrees, seed: int = 0, name: str = "") -> Code:
    """PEG-style construction for given variable and check degree sequences.

    Variables are processed in order of increasing degree (ties by index).
    For each new edge of variable v, a breadth-first expansion of the current
    Tanner graph from v records the depth at which each check is first
    reached (checks never reached count as infinitely far). The edge goes to
    an available check (current degree below its target, not yet adjacent to
    v) of greatest depth; ties go to the lowest current degree, then to a
    seeded random pick.
    """
    var_degrees = np.asarray(var_degrees, dtype=np.int64)
    check_degrees = np.asarray(check_degrees, dtype=np.int64)
    n, m = len(var_degrees), len(check_degrees)
    if var_degrees.sum() != check_degrees.sum():
        raise ValueError("degree sequences do not have the same edge count")
    rng = np.random.default_rng([0x5E6, seed, n, m])
    dvmax, dcmax = int(var_degrees.max()), int(check_degrees.max())
    vc = np.full((n, dvmax), -1, dtype=np.int64)   # var -> checks
    cv = np.full((m, dcmax), -1, dtype=np.int64)   # check -> vars
    vdeg = np.zeros(n, dtype=np.int64)
    cdeg = np.zeros(m, dtype=np.int64)
    INF = np.iinfo(np.int64).max
    order = np.lexsort((np.arange(n), var_degrees))
    for v in order:
        for k in range(int(var_degrees[v])):
            depth = np.full(m, INF, dtype=np.int64)
            if vdeg[v] > 0:
                seen_v = np.zeros(n, dtype=bool)
                seen_v[v] = True
                fc = vc[v, :vdeg[v]]
                d = 0
                depth[fc] = d
                while True:
                    nv = cv[fc].ravel()
                    nv = nv[nv >= 0]
                    nv = np.unique(nv[~seen_v[nv]])
                    if nv.size == 0:
                        break
                    seen_v[nv] = True
                    nc = vc[nv].ravel()
                    nc = np.unique(nc[nc >= 0])
                    nc = nc[depth[nc] == INF]
                    if nc.size == 0:
                        break
                    d += 1
                    depth[nc] = d
                    fc = nc
            avail = cdeg < check_degrees
            avail[vc[v, :vdeg[v]]] = False
            cand = np.flatnonzero(avail)
            if cand.size == 0:
                raise RuntimeError("PEG ran out of available checks")
            dmax = depth[cand].max()
            cand = cand[depth[cand] == dmax]
            cand = cand[cdeg[cand] == cdeg[cand].min()]
            c = int(cand[rng.integers(cand.size)])
            vc[v, vdeg[v]] = c
            vdeg[v] += 1
            cv[c, cdeg[c]] = v
            cdeg[c] += 1
    rows = [cv[j, :cdeg[j]] for j in range(m)]
    return from_rows(rows, n, name=name)


def peg_regular(n: int, dv: int = 3, dc: int = 6, seed: int = 0) -> Code:
    if (n * dv) % dc:
        raise ValueError("n*dv must be a multiple of dc")
    m = n * dv // dc
    return peg_code(np.full(n, dv), np.full(m, dc), seed=seed,
                    name=f"peg({dv},{dc}) n={n} seed={seed}")


def irregular_degrees(n: int, lam: dict, dc: int):
    """Variable-degree sequence for an edge-perspective distribution
    lambda(x) = sum_i lam[i] x^(i-1) and constant check degree dc.

    Node fractions are proportional to lam[i]/i; counts are rounded and the
    largest class is adjusted so that the edge count is a multiple of dc.
    Returns (var_degrees, m).
    """
    degs = sorted(lam)
    w = np.array([lam[d] / d for d in degs])
    frac = w / w.sum()
    counts = np.floor(frac * n).astype(np.int64)
    counts[np.argmax(frac)] += n - counts.sum()
    # adjust pairs of classes (d_a -> d_b) until the edge count divides dc
    E = int(np.dot(counts, degs))
    i_lo = 0
    guard = 0
    while E % dc:
        guard += 1
        if guard > 10 * dc:
            raise RuntimeError("cannot match the edge count to dc")
        # move one node from the lowest degree class to the next one
        counts[i_lo] -= 1
        counts[i_lo + 1] += 1
        E = int(np.dot(counts, degs))
    var_degrees = np.repeat(np.array(degs), counts)
    return var_degrees, E // dc


def irregular_code(n: int, lam: dict, dc: int, seed: int = 0) -> Code:
    vd, m = irregular_degrees(n, lam, dc)
    return peg_code(vd, np.full(m, dc), seed=seed,
                    name=f"irregular n={n} dc={dc} seed={seed}")


def hamming74(col_order=None) -> Code:
    """3 x 7 Hamming parity-check matrix; column k holds the binary
    expansion of col_order[k] (a permutation of 1..7)."""
    if col_order is None:
        col_order = list(range(1, 8))
    H = np.zeros((3, 7), dtype=np.uint8)
    for k, v in enumerate(col_order):
        for b in range(3):
            H[b, k] = (v >> b) & 1
    return from_dense(H, name=f"hamming74 {list(col_order)}")


# ---------------------------------------------------------------------------
# Codewords (for symmetry tests)
# ---------------------------------------------------------------------------

def _gf2_nullspace(H: np.ndarray) -> np.ndarray:
    """Basis (rows) of {u : H u = 0 mod 2} by Gauss-Jordan elimination."""
    A = (np.asarray(H) & 1).astype(np.uint8).copy()
    m, n = A.shape
    pivots = []
    r = 0
    for c in range(n):
        if r >= m:
            break
        piv = np.flatnonzero(A[r:, c])
        if piv.size == 0:
            continue
        p = r + piv[0]
        if p != r:
            A[[r, p]] = A[[p, r]]
        rows = np.flatnonzero(A[:, c])
        rows = rows[rows != r]
        A[rows] ^= A[r]
        pivots.append(c)
        r += 1
    free = [c for c in range(n) if c not in set(pivots)]
    basis = np.zeros((len(free), n), dtype=np.uint8)
    for t, f in enumerate(free):
        basis[t, f] = 1
        for i, pc in enumerate(pivots):
            basis[t, pc] = A[i, f]
    return basis


def random_codeword(code: Code, seed: int) -> np.ndarray:
    """A uniformly random codeword of ker(H) (seeded)."""
    B = _gf2_nullspace(code.dense())
    rng = np.random.default_rng([0xC0DE, seed])
    coef = rng.integers(0, 2, size=B.shape[0]).astype(np.uint8)
    return (coef @ B % 2).astype(np.uint8) if B.shape[0] else np.zeros(code.n, np.uint8)


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

@functools.lru_cache(maxsize=None)
def named_code(name: str) -> Code:
    """The codes of the workloads:

    * ``gallager_120``: (3,6) Gallager, n=120, m=60, seed 0.
    * ``peg_1008``: (3,6) PEG-style, n=1008, m=504, seed 0.
    * ``gallager_16000``: (3,6) Gallager, n=16000, m=8000, seed 0.
    * ``gallager_<n>``: (3,6) Gallager of length n (n multiple of 6), seed 0.
    * ``gallager330_8000``: (3,30) Gallager, n=8000, m=800, seed 0.
    * ``irregular_4000``: lambda(x)=0.25x+0.3x^2+0.45x^7, dc=8, n=4000.
    """
    if name == "peg_1008":
        return peg_regular(1008, 3, 6, seed=0)
    if name == "gallager330_8000":
        return gallager_regular(8000, 3, 30, seed=0)
    if name == "irregular_4000":
        return irregular_code(4000, {2: 0.25, 3: 0.30, 8: 0.45}, 8, seed=0)
    if name.startswith("gallager_"):
        return gallager_regular(int(name.split("_")[1]), 3, 6, seed=0)
    if name.startswith("peg_"):
        return peg_regular(int(name.split("_")[1]), 3, 6, seed=0)
    raise KeyError(name)
