"""Maximum-weight triangular set (MTS) preconditioners and PCG (oracle).

Section V: the preconditioner for Q = A D^2 A' (p x p) is
M = A_M D_M^2 A_M' over a set M of p columns of A for which A_M can be
brought to triangular form by row and column permutations (a "triangular
set"); M z = r is then solved by A_M f1 = r, D_M^2 f2 = f1, A_M' z = f2,
each in linear time.

A triangular set is returned as two lists ``col`` and ``row`` of length p:
the k-th selected column col[k] is paired with row row[k]. The permuted
matrix T[k, l] = A[row[k], col[l]] is
  * upper triangular for the column-wise search (Algorithm 7), and
  * lower triangular for the triangulation step (Algorithm 5) and the
    incremental (Algorithm 6) and row-wise (Algorithm 8) searches.

Weights: the paper ranks columns by d_i (or alternatively x_i). The oracle
ranks by d_i^2 = x_i / z_i in double precision, which orders columns exactly
as d_i does. Ties go to the lower column index (standard columns 0..n-1
before slack columns n..n+p-1); the row-wise search picks the lowest-index
degree-1 row.
"""

from __future__ import annotations

import heapq

import numpy as np
import scipy.linalg


def _pattern(A):
    """Column -> rows and row -> columns lists of the nonzero pattern."""
    A = np.asarray(A)
    col_rows = [np.flatnonzero(A[:, i]) for i in range(A.shape[1])]
    row_cols = [np.flatnonzero(A[j, :]) for j in range(A.shape[0])]
    return col_rows, row_cols


# ---------------------------------------------------------------------------
# Algorithm 7: column-wise greedy search (upper-triangular A_M)
# ---------------------------------------------------------------------------

def colwise(A, w):
    """Algorithm 7. Repeatedly take the maximum-weight degree-1 column of
    the residual matrix, record it with the row of its only nonzero, and zero
    that row. DEG1 is kept in a binary heap (Section V-B) with lazy deletion
    of columns whose degree has dropped to zero."""
    p, q = A.shape
    col_rows, row_cols = _pattern(A)
    deg = np.array([len(r) for r in col_rows], dtype=np.int64)
    row_alive = np.ones(p, dtype=bool)
    taken = np.zeros(q, dtype=bool)
    heap = [(-float(w[i]), i) for i in range(q) if deg[i] == 1]
    heapq.heapify(heap)
    col, row = [], []
    for _ in range(p):
        while True:
            _, i = heapq.heappop(heap)
            if deg[i] == 1 and not taken[i]:
                break
        j = next(int(r) for r in col_rows[i] if row_alive[r])
        col.append(int(i))
        row.append(j)
        taken[i] = True
        row_alive[j] = False
        for i2 in row_cols[j]:
            if taken[i2]:
                continue
            deg[i2] -= 1
            if deg[i2] == 1:
                heapq.heappush(heap, (-float(w[i2]), int(i2)))
    return np.asarray(col), np.asarray(row)


# ---------------------------------------------------------------------------
# Algorithm 5: triangulation step; Algorithm 6: incremental greedy search
# ---------------------------------------------------------------------------

def triangulate(A, S):
    """Algorithm 5 on the columns S: peel degree-1 rows of A_S. Returns
    (col, row) of a lower-triangular form, or None. Rows that are already
    all zero are ignored when looking for the minimum row degree."""
    A = np.asarray(A)
    S = list(S)
    sub = A[:, S] != 0
    alive_c = np.ones(len(S), dtype=bool)
    alive_r = np.ones(A.shape[0], dtype=bool)
    col, row = [], []
    for _ in range(len(S)):
        deg = (sub[:, alive_c]).sum(axis=1)
        cand = np.flatnonzero(alive_r & (deg == 1))
        if cand.size == 0:
            return None
        j = int(cand[0])
        k = int(np.flatnonzero(sub[j] & alive_c)[0])
        col.append(S[k])
        row.append(j)
        alive_c[k] = False
        alive_r[j] = False
    return np.asarray(col), np.asarray(row)


def incremental(A, w):
    """Algorithm 6: scan columns by decreasing weight and keep each one
    whose addition leaves the set triangular (checked by Algorithm 5)."""
    p, q = A.shape
    order = sorted(range(q), key=lambda i: (-float(w[i]), i))
    M = []
    best = None
    for i in order:
        if len(M) >= p:
            break
        tri = triangulate(A, M + [i])
        if tri is not None:
            M.append(i)
            best = tri
    return best


# ---------------------------------------------------------------------------
# Algorithm 8: row-wise greedy search with diagonal expansion
# ---------------------------------------------------------------------------

def rowwise(A, w, n, expansion="diagonal"):
    """Algorithm 8: peel degree-1 rows (lowest index first); when none is
    left, zero the minimum-weight nonzero column (ties: lowest index).

    expansion = "diagonal" (Algorithm 8 as printed): rows never peeled are
    then paired with their own slack columns n + j, in increasing j.
    expansion = "triangular" (Section V-A's alternative): the same search is
    run again on the columns of A that have no nonzero in any row peeled so
    far (so the new pivots extend the lower-triangular set), and again,
    until every row is peeled; each such round peels at least one row,
    because every row not yet peeled keeps its own slack column."""
    A = np.asarray(A) != 0
    p, q = A.shape
    used_r = np.zeros(p, dtype=bool)
    col, row = [], []
    alive_c = A.any(axis=0)
    while True:
        while alive_c.any():
            deg = (A[:, alive_c]).sum(axis=1)
            cand = np.flatnonzero(deg == 1)
            if cand.size:
                j = int(cand[0])
                i = int(np.flatnonzero(A[j] & alive_c)[0])
                col.append(i)
                row.append(j)
                used_r[j] = True
                alive_c[i] = False
            else:
                live = np.flatnonzero(alive_c)
                i = int(min(live, key=lambda t: (float(w[t]), t)))
                alive_c[i] = False
        if expansion != "triangular" or used_r.all():
            break
        alive_c = A.any(axis=0) & ~A[used_r].any(axis=0)
    for j in range(p):
        if not used_r[j]:
            col.append(n + j)
            row.append(j)
    return np.asarray(col), np.asarray(row)


# ---------------------------------------------------------------------------
# M-solve and PCG (Algorithm 4)
# ---------------------------------------------------------------------------

def triangular_form(A, col, row):
    T = np.asarray(A)[np.ix_(row, col)]
    if np.allclose(np.tril(T, -1), 0):
        return T, False      # upper triangular
    if np.allclose(np.triu(T, 1), 0):
        return T, True       # lower triangular
    raise ValueError("selected set is not triangular under its order")


def msolve(A, d2, col, row, r):
    """z with A_M D_M^2 A_M' z = r: A_M f1 = r, f2 = f1 / d_M^2, A_M' z = f2
    (Section V), by triangular substitution on T = A[row, col]."""
    T, lower = triangular_form(A, col, row)
    f1 = scipy.linalg.solve_triangular(T, r[row], lower=lower)
    f2 = f1 / d2[col]
    zp = scipy.linalg.solve_triangular(T.T, f2, lower=not lower)
    z = np.empty_like(r)
    z[row] = zp
    return z


def pcg(A, d2, w, col, row, tol, max_iter, x0=None, residuals=None, coefficients=None):
    """Algorithm 4 on Q = A D^2 A' with the MTS preconditioner (col, row);
    col = None runs plain CG (M = I). Stops when ||r||_2 / ||w||_2 < tol (r
    the recurrence residual). ``coefficients`` (a list) receives (alpha,
    nu) per iteration."""
    Q = lambda v: A @ (d2 * (A.T @ v))  # noqa: E731
    if col is None:
        msolve_ = lambda r: r.copy()  # noqa: E731
    else:
        msolve_ = lambda r: msolve(A, d2, col, row, r)  # noqa: E731
    x = np.zeros_like(w) if x0 is None else x0.copy()
    r = w - Q(x)
    wn = float(np.linalg.norm(w))
    if wn == 0.0:
        return x, 0
    z = msolve_(r)
    h = z.copy()
    zr = float(np.dot(z, r))
    it = 0
    for it in range(max_iter + 1):
        rel = float(np.linalg.norm(r)) / wn
        if residuals is not None:
            residuals.append(rel)
        if rel < tol or it == max_iter:
            break
        l = Q(h)
        alpha = zr / float(np.dot(h, l))
        x = x + alpha * h
        r = r - alpha * l
        z = msolve_(r)
        zr_new = float(np.dot(z, r))
        nu = zr_new / zr
        if coefficients is not None:
            coefficients.append((alpha, nu))
        h = z + nu * h
        zr = zr_new
    return x, it


def pcg_normal_solver(A, n, select="colwise", tol=1e-10, max_iter=1000, log=None):
    """A ``solve_normal`` callback for ``ipm.solve`` that uses PCG with the
    chosen MTS selection, for experiments and iteration-count references."""
    def solve(d2, w):
        if select == "colwise":
            col, row = colwise(A, d2)
        elif select == "incremental":
            col, row = incremental(A, d2)
        elif select == "rowwise":
            col, row = rowwise(A, d2, n)
        else:
            col, row = np.arange(n, A.shape[1]), np.arange(A.shape[0])
        res = []
        dy, it = pcg(A, d2, w, col, row, tol, max_iter, residuals=res)
        if log is not None:
            log.append(dict(iters=it, final=res[-1] if res else 0.0))
        return dy
    return solve
