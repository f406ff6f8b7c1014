"""Pins for the oracle's MTS preconditioners (Algorithms 5-8), the M-solve
and PCG (Algorithm 4): structural triangularity, the greedy rule of
Algorithm 7 replayed step by step, dense-solve agreement, the exact
one-step case M = Q, Lemma 2 and Theorem 5.
"""

import numpy as np
import pytest

import oracle
from oracle import ipm, lp, mts
from oracle.params import OracleParams
from synth import awgn_llr_frames, named_code


def lps_of_frames(n_frames=6, ebn0=2.0, seed=0):
    code = named_code("gallager_120")
    G = awgn_llr_frames(code.n, code.design_rate, ebn0, seed, range(n_frames))
    out = []
    for g in G:
        res = oracle.decode(code, g)
        for h in res.history:
            out.append((code, g, lp.build(code, g, h.in_lp, h.masks), res.cert))
    return out


def test_colwise_is_upper_triangular_and_greedy():
    rng = np.random.default_rng(1)
    for code, g, L, _ in lps_of_frames()[:12]:
        p, q = L.A.shape
        w = np.exp(rng.normal(size=q) * 4)
        col, row = mts.colwise(L.A, w)
        assert len(set(col)) == p and sorted(row) == list(range(p))
        T = L.A[np.ix_(row, col)]
        assert np.allclose(np.tril(T, -1), 0)
        assert np.all(np.abs(np.diag(T)) == 1)
        # replay: at step k, col[k] is degree-1 in the residual matrix with
        # its only nonzero in row[k], and no degree-1 column outweighs it
        alive = np.ones(p, bool)
        taken = np.zeros(q, bool)
        for k in range(p):
            deg = (L.A[alive] != 0).sum(axis=0)
            deg1 = np.flatnonzero((deg == 1) & ~taken)
            i = col[k]
            assert i in deg1
            assert np.flatnonzero(L.A[:, i] * alive)[0] == row[k]
            best = max(deg1, key=lambda t: (w[t], -t))
            assert best == i
            alive[row[k]] = False
            taken[i] = True


def test_msolve_and_pcg_match_dense_solves():
    rng = np.random.default_rng(2)
    for code, g, L, _ in lps_of_frames()[:10]:
        p, q = L.A.shape
        d2 = np.exp(rng.normal(size=q) * 3)
        col, row = mts.colwise(L.A, d2)
        r = rng.normal(size=p)
        AM = L.A[:, col]
        M = AM @ np.diag(d2[col]) @ AM.T
        z = mts.msolve(L.A, d2, col, row, r)
        assert np.linalg.norm(M @ z - r) <= 1e-10 * np.linalg.norm(r) * max(1.0, np.linalg.norm(M))
        Q = L.A @ np.diag(d2) @ L.A.T
        x_ref = np.linalg.solve(Q, r)
        x, it = mts.pcg(L.A, d2, r, col, row, 1e-12, 5 * p)
        assert np.linalg.norm(x - x_ref) <= 1e-8 * np.linalg.norm(x_ref)


def test_pcg_converges_in_one_step_when_m_equals_q():
    """If d_i = 0 off the preconditioning set, M = A_M D_M^2 A_M' = Q and
    the first PCG step is exact."""
    rng = np.random.default_rng(3)
    for code, g, L, _ in lps_of_frames()[:8]:
        p, q = L.A.shape
        d2 = np.exp(rng.normal(size=q))
        col, row = mts.colwise(L.A, d2)
        d2z = np.zeros(q)
        d2z[col] = d2[col]
        w = rng.normal(size=p)
        res = []
        x, it = mts.pcg(L.A, d2z, w, col, row, 1e-12, 10, residuals=res)
        assert it <= 1 and res[-1] < 1e-12


def test_triangulation_and_rowwise_structure():
    rng = np.random.default_rng(4)
    for code, g, L, _ in lps_of_frames()[:6]:
        p, q = L.A.shape
        w = rng.random(q)
        col, row = mts.rowwise(L.A, w, code.n)
        assert len(col) == p and sorted(row) == list(range(p))
        T = L.A[np.ix_(row, col)]
        assert np.allclose(np.triu(T, 1), 0) and np.all(np.abs(np.diag(T)) == 1)
        tri = mts.triangulate(L.A, list(range(code.n, q)))     # slack set
        assert tri is not None


def test_rowwise_triangular_expansion_by_hand():
    """Section V-A's triangular expansion on a 2-row LP worked by hand:
    rows r0 = {c0, c1, s0}, r1 = {c0, c1, c2, s1}, weights c0 5, c1 0.3,
    c2 0.25, s0 0.1, s1 0.2. The search zeroes s0, s1, c2, c1 (least weight
    first, no row of degree one before), then r0 and r1 both hold only c0:
    r0 peels it and r1 is left empty. The diagonal expansion gives r1 its
    slack s1; the triangular expansion searches the columns without a
    nonzero in r0, {c2, s1}: it zeroes s1 (the lighter) and r1 peels c2."""
    A = np.array([[1, 1, 0, 1, 0], [1, 1, 1, 0, 1]])
    w = np.array([5.0, 0.3, 0.25, 0.1, 0.2])
    col, row = mts.rowwise(A, w, 3)
    assert list(col) == [0, 4] and list(row) == [0, 1]
    col, row = mts.rowwise(A, w, 3, "triangular")
    assert list(col) == [0, 2] and list(row) == [0, 1]


def test_rowwise_triangular_expansion_structure():
    """On LPs of decodes: the triangular expansion gives a full lower-
    triangular set with unit diagonal; it starts with the same pivots as
    the diagonal expansion (the first search is the same), keeps every
    column of a later round free of the rows peeled before it, and never
    needs more slack columns than the diagonal expansion adds."""
    rng = np.random.default_rng(9)
    differs = 0
    for code, g, L, _ in lps_of_frames()[:8]:
        p, q = L.A.shape
        for w in (rng.random(q), np.exp(rng.normal(size=q) * 4)):
            cd, rd = mts.rowwise(L.A, w, code.n)
            ct, rt = mts.rowwise(L.A, w, code.n, "triangular")
            assert len(ct) == p and sorted(rt) == list(range(p)) and len(set(ct)) == p
            T = L.A[np.ix_(rt, ct)]
            assert np.allclose(np.triu(T, 1), 0) and np.all(np.abs(np.diag(T)) == 1)
            # pivots of the first search: the diagonal result up to its tail of
            # slack columns in increasing rows (the expansion)
            k1 = 0
            while k1 < p and not (cd[k1] >= code.n and list(rd[k1:]) == sorted(rd[k1:])
                                  and all(cd[k1:] == code.n + rd[k1:])):
                k1 += 1
            assert list(ct[:k1]) == list(cd[:k1]) and list(rt[:k1]) == list(rd[:k1])
            assert np.sum(ct >= code.n) <= np.sum(cd >= code.n)
            differs += not np.array_equal(ct, cd)
    assert differs > 0


def test_lemma2_and_theorem5_on_integral_lps():
    """Lemma 2: the basic set of an integral LP has no stopping set
    (Algorithm 5 triangulates it). Theorem 5: near the optimum, the
    incremental (Algorithm 6) and row-wise (Algorithm 8) sets contain it."""
    prm = OracleParams()
    checked = 0
    for code, g, L, cert in lps_of_frames(10):
        tr = []
        r = ipm.solve(L.A, L.b, L.c, prm, trace=tr)
        u = L.u_from_x(r.x)
        if np.max(np.abs(u - np.round(u))) > 1e-6:
            continue
        basic = np.flatnonzero(r.x > r.z)
        assert mts.triangulate(L.A, basic) is not None
        d2 = r.x / r.z
        col_i, _ = mts.incremental(L.A, d2)
        col_r, _ = mts.rowwise(L.A, d2, code.n)
        assert set(basic) <= set(col_i)
        assert set(basic) <= set(col_r)
        checked += 1
        if checked >= 6:
            break
    assert checked >= 3


def test_pcg_newton_solver_reproduces_cholesky_ipm():
    """The IPM with PCG + column-wise MTS Newton solves ends at the same
    vertex as with the direct (Cholesky) solve."""
    prm = OracleParams()
    for code, g, L, _ in lps_of_frames(3):
        r1 = ipm.solve(L.A, L.b, L.c, prm)
        r2 = ipm.solve(L.A, L.b, L.c, prm,
                       solve_normal=mts.pcg_normal_solver(L.A, code.n, "colwise", 1e-10, 2000))
        assert r2.status == 0
        assert np.max(np.abs(L.u_from_x(r1.x) - L.u_from_x(r2.x))) < 1e-6


def _kappas(A, d2):
    """cond(Q) and cond(M^-1 Q) for Q = A D^2 A' and the column-wise MTS
    M = A_M D_M^2 A_M', from singular values of D-scaled factors (no
    product is formed: cond(Q) = cond(A D)^2, and M^-1 Q is similar to
    B B' with B = D_M^-1 A_M^-1 A D)."""
    d = np.sqrt(d2)
    AD = A * d
    s = np.linalg.svd(AD, compute_uv=False)
    col, row = mts.colwise(A, d2)
    B = np.linalg.solve(A[:, col], AD) / d[col][:, None]
    s2 = np.linalg.svd(B, compute_uv=False)
    return (s[0] / s[-1]) ** 2, (s2[0] / s2[-1]) ** 2, col, row


def test_mts_clusters_the_spectrum_near_an_integral_optimum():
    """Section VI: as the interior-point method approaches an integral
    optimum, Q = A D^2 A' becomes very ill-conditioned while the MTS
    preconditioner keeps M^-1 Q well conditioned, so PCG needs few
    iterations where plain CG would need many (Figs. 5-6)."""
    code = named_code("gallager_120")
    G = awgn_llr_frames(code.n, code.design_rate, 2.0, 0, range(12))
    prm = OracleParams()
    checked = 0
    for g in G:
        res = oracle.decode(code, g)
        if res.cert != 1 or not res.history:
            continue
        h = res.history[-1]
        L = lp.build(code, g, h.in_lp, h.masks)
        tr = []
        ipm.solve(L.A, L.b, L.c, prm, trace=tr)
        kq, kp, col, row = _kappas(L.A, tr[-1]["d2"])
        assert kq > 1e12 and kp < 1e3, (kq, kp)
        p = L.A.shape[0]
        w = np.random.default_rng(0).normal(size=p)
        rs = []
        mts.pcg(L.A, tr[-1]["d2"], w, col, row, 1e-8, 5 * p, residuals=rs)
        assert len(rs) - 1 <= p, len(rs)
        checked += 1
    assert checked >= 5


def _cg_iters(Q, w, tol, max_it):
    """Plain CG (no preconditioner) iterations to ||r|| < tol ||w||."""
    x = np.zeros_like(w)
    r = w.copy()
    h = r.copy()
    wn = np.linalg.norm(w)
    it = 0
    while np.linalg.norm(r) >= tol * wn and it < max_it:
        l = Q @ h
        a = (r @ r) / (h @ l)
        x += a * h
        rn = r - a * l
        h = rn + (rn @ rn) / (r @ r) * h
        r = rn
        it += 1
    return it


def test_preconditioners_against_plain_cg():
    """Section VI-B (Figs. 5-8): on the last LP of MALP-A decodings of a
    (3,6) n=480 code at 1.5 dB, plain CG stops converging as the interior
    point nears the optimum, while PCG with each MTS preconditioner
    (Algorithms 6, 7, 8) converges in far fewer iterations; in the
    ill-conditioned late iterations of fractional LPs the incremental search
    is the most effective and does at least as well as the row-wise one."""
    code = named_code("gallager_480")
    G = awgn_llr_frames(code.n, code.design_rate, 1.5, 0, range(4))
    prm = OracleParams()
    cap = 1000
    inc_late = row_late = 0
    n_int = 0
    for g in G:
        res = oracle.decode(code, g)
        h = res.history[-1]
        L = lp.build(code, g, h.in_lp, h.masks)
        tr = []
        ipm.solve(L.A, L.b, L.c, prm, trace=tr)
        p = L.A.shape[0]
        w = np.random.default_rng(0).normal(size=p)
        for t in (tr[(2 * len(tr)) // 3], tr[-1]):
            d2 = t["d2"]
            Q = (L.A * d2) @ L.A.T
            cg = _cg_iters(Q, w, 1e-4, cap)
            its = {}
            for name, (col, row) in (("col", mts.colwise(L.A, d2)),
                                     ("inc", mts.incremental(L.A, d2)),
                                     ("row", mts.rowwise(L.A, d2, code.n))):
                rs = []
                mts.pcg(L.A, d2, w, col, row, 1e-4, cap, residuals=rs)
                its[name] = len(rs) - 1
            if t is tr[-1]:
                assert min(its.values()) < cg, (its, cg)   # CG at the cap
            else:
                assert min(its.values()) * 3 <= cg, (its, cg)
            if res.cert == 1 and t is tr[-1]:
                n_int += 1
                assert cg == cap and max(its.values()) <= 60, (its, cg)
            if res.cert == 0 and t is tr[-1]:
                inc_late += its["inc"]
                row_late += its["row"]
                assert its["inc"] <= min(its["col"], its["row"]), its
    assert n_int >= 1 and inc_late <= row_late
