"""GPU parity of single hot-path steps against the oracle, through the C
ABI: the cut search (Algorithm 2 inside Algorithm 3), the column-wise MTS
selection (Algorithm 7), PCG (Algorithm 4) and one LP solve (Section IV-B
plus optimal-vertex recovery)."""

import numpy as np
import pytest

from oracle import cuts as ocuts
from oracle import ipm as oipm
from oracle import mts as omts
from oracle import vertex as overtex
from oracle.params import OracleParams
from paper_0902_0657_gb300 import lpdec as L
from synth import named_code

from .gpu_util import dev, host, lp_state_arrays, oracle_history, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dec120():
    torch_cuda()
    d = L.Decoder(named_code("gallager_120"))
    yield d
    d.close()


def oracle_search_round(code, u, in_lp, active, mask, tau):
    in_lp = in_lp.copy().astype(bool)
    mask = mask.copy()
    added = 0
    for j in range(code.m):
        if in_lp[j] and active[j]:
            continue
        mk, lhs, viol = ocuts.find_violated(u[code.row(j)], tau)
        if viol:
            in_lp[j] = True
            mask[j] = mk
            added = 1
    return in_lp.astype(np.uint8), mask, added


def test_cut_search_bit_exact(dec120):
    torch = torch_cuda()
    code = named_code("gallager_120")
    rng = np.random.default_rng(5)
    nf = 64
    U = rng.random((nf, code.n))
    # special values: exact halves, integral points, ties
    U[0] = 0.5
    U[1] = rng.integers(0, 2, code.n)
    U[2] = np.round(rng.random(code.n) * 4) / 4
    U[3, ::2] = 0.5
    in_lp = (rng.random((nf, code.m)) < 0.4).astype(np.uint8)
    active = ((rng.random((nf, code.m)) < 0.5) & (in_lp > 0)).astype(np.uint8)
    mask = np.where(in_lp > 0, rng.integers(1, 64, (nf, code.m)), 0).astype(np.uint32)
    d_u, d_act, d_in, d_mask = dev(U), dev(active), dev(in_lp), dev(mask)
    d_flag = torch.zeros(nf, dtype=torch.int32, device="cuda")
    rc = L.lpdec_cut_search_device(dec120.ctx, dec120.code, nf, d_u, d_act, d_in, d_mask, d_flag)
    assert rc == 0
    torch.cuda.synchronize()
    g_in, g_mask, g_flag = host(d_in), host(d_mask), host(d_flag)
    tau = dec120.params.tau_cut
    for f in range(nf):
        e_in, e_mask, e_add = oracle_search_round(code, U[f], in_lp[f], active[f], mask[f], tau)
        assert np.array_equal(g_in[f], e_in), f
        assert np.array_equal(g_mask[f], e_mask), f
        assert g_flag[f] == e_add


@pytest.mark.parametrize("kind", [L.LPDEC_MTS_COLUMN, L.LPDEC_MTS_INCREMENTAL,
                                  L.LPDEC_MTS_ROWWISE, L.LPDEC_MTS_ROWWISE_TRI])
def test_mts_selection_bit_exact(kind):
    """Algorithms 7 (column-wise), 6 with 5 (incremental) and 8 (row-wise
    with diagonal expansion, and with Section V-A's triangular expansion):
    the selected (column, row) pairs in selection
    order equal the oracle's, on LPs of oracle decodes with random weights,
    quantised weights (ties) and weights that differ below single
    precision."""
    torch = torch_cuda()
    code, recs = oracle_history("gallager_120", 2.0, 0, 12)
    g, in_lp, mask, lps = lp_state_arrays(code, recs)
    nf = len(lps)
    qm = code.n + code.m
    rng = np.random.default_rng(7)
    W = np.zeros((nf, qm))
    for f, lp in enumerate(lps):
        w = np.exp(rng.normal(size=lp.q) * 5)
        if f % 3 == 0:                       # ties: quantised weights
            w = np.round(rng.random(lp.q) * 4) + 1
        elif f % 3 == 1:                     # differences below single precision
            w = 1.0 + rng.integers(0, 4, size=lp.q) * 1e-12
        W[f, :lp.q] = w
    prm = L.lpdec_default_params()
    prm.precond = kind
    with L.Decoder(code, params=prm) as d:
        d_col = torch.empty((nf, code.m), dtype=torch.int32, device="cuda")
        d_row = torch.empty((nf, code.m), dtype=torch.int32, device="cuda")
        rc = L.lpdec_mts_select_device(d.ctx, d.code, nf, dev(g), dev(in_lp), dev(mask),
                                       dev(W), d_col, d_row)
        assert rc == 0
        col, row = host(d_col), host(d_row)
    for f, lp in enumerate(lps):
        w = W[f, :lp.q]
        if kind == L.LPDEC_MTS_COLUMN:
            ec, er = omts.colwise(lp.A, w)
        elif kind == L.LPDEC_MTS_INCREMENTAL:
            ec, er = omts.incremental(lp.A, w)
        elif kind == L.LPDEC_MTS_ROWWISE:
            ec, er = omts.rowwise(lp.A, w, code.n)
        else:
            ec, er = omts.rowwise(lp.A, w, code.n, "triangular")
        assert np.array_equal(col[f, :lp.p], ec), (kind, f)
        assert np.array_equal(row[f, :lp.p], er), (kind, f)
        assert np.all(col[f, lp.p:] == -1)


@pytest.mark.parametrize("kind", [L.LPDEC_MTS_INCREMENTAL, L.LPDEC_MTS_ROWWISE,
                                  L.LPDEC_MTS_ROWWISE_TRI])
def test_pcg_with_each_preconditioner_matches_dense_solve(kind):
    """PCG (Algorithm 4) preconditioned by the incremental and row-wise
    triangular sets (lower triangular: the level schedules run in the other
    directions) solves the Newton system as a dense solve does."""
    torch = torch_cuda()
    code, recs = oracle_history("gallager_120", 2.0, 0, 12)
    g, in_lp, mask, lps = lp_state_arrays(code, recs)
    nf = len(lps)
    qm = code.n + code.m
    rng = np.random.default_rng(13)
    D2 = np.zeros((nf, qm))
    Wv = np.zeros((nf, code.m))
    for f, lp in enumerate(lps):
        D2[f, :lp.q] = np.exp(rng.normal(size=lp.q) * 2)
        Wv[f, :lp.p] = rng.normal(size=lp.p)
    prm = L.lpdec_default_params()
    prm.precond = kind
    with L.Decoder(code, params=prm) as d:
        d_dy = torch.zeros((nf, code.m), dtype=torch.float64, device="cuda")
        d_it = torch.zeros(nf, dtype=torch.int32, device="cuda")
        rc = L.lpdec_pcg_device(d.ctx, d.code, nf, dev(g), dev(in_lp), dev(mask), dev(D2),
                                dev(Wv), d_dy, d_it)
        assert rc == 0
        dy, its = host(d_dy), host(d_it)
    for f, lp in enumerate(lps):
        Q = (lp.A * D2[f, :lp.q]) @ lp.A.T
        ref = np.linalg.solve(Q, Wv[f, :lp.p])
        rel = np.linalg.norm(dy[f, :lp.p] - ref) / np.linalg.norm(ref)
        kappa = np.linalg.cond(Q)
        assert rel <= max(1e-8, 1e-10 * kappa * 10), (kind, f, rel, kappa, its[f])
        assert its[f] <= lp.p + 5


def test_pcg_matches_dense_solve(dec120):
    torch = torch_cuda()
    code, recs = oracle_history("gallager_120", 2.0, 0, 12)
    g, in_lp, mask, lps = lp_state_arrays(code, recs)
    nf = len(lps)
    qm = code.n + code.m
    rng = np.random.default_rng(11)
    D2 = np.zeros((nf, qm))
    Wv = np.zeros((nf, code.m))
    for f, lp in enumerate(lps):
        D2[f, :lp.q] = np.exp(rng.normal(size=lp.q) * 2)
        Wv[f, :lp.p] = rng.normal(size=lp.p)
    d_dy = torch.zeros((nf, code.m), dtype=torch.float64, device="cuda")
    d_it = torch.zeros(nf, dtype=torch.int32, device="cuda")
    rc = L.lpdec_pcg_device(dec120.ctx, dec120.code, nf, dev(g), dev(in_lp), dev(mask),
                            dev(D2), dev(Wv), d_dy, d_it)
    assert rc == 0
    dy, its = host(d_dy), host(d_it)
    for f, lp in enumerate(lps):
        Q = (lp.A * D2[f, :lp.q]) @ lp.A.T
        ref = np.linalg.solve(Q, Wv[f, :lp.p])
        rel = np.linalg.norm(dy[f, :lp.p] - ref) / np.linalg.norm(ref)
        kappa = np.linalg.cond(Q)
        assert rel <= max(1e-8, 1e-10 * kappa * 10), (f, rel, kappa, its[f])
        assert its[f] <= lp.p + 5


def test_lp_solve_matches_oracle_vertex(dec120):
    torch = torch_cuda()
    code, recs = oracle_history("gallager_120", 2.0, 0, 12)
    g, in_lp, mask, lps = lp_state_arrays(code, recs)
    nf = len(lps)
    qm = code.n + code.m
    d_x = torch.zeros((nf, qm), dtype=torch.float64, device="cuda")
    d_st = torch.zeros(nf * L.STATS_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    rc = L.lpdec_lp_solve_device(dec120.ctx, dec120.code, nf, dev(g), dev(in_lp), dev(mask),
                                 d_x, d_st)
    assert rc == 0
    x = host(d_x)
    st = host(d_st).view(L.STATS_DTYPE)
    prm = OracleParams()
    for f, lp in enumerate(lps):
        r = oipm.solve(lp.A, lp.b, lp.c, prm)
        xv, ok = overtex.recover(lp.A, lp.b, lp.c, r.x, r.z, r.y)
        assert ok and st["status"][f] == 0 and st["vertex_failures"][f] == 0
        assert np.max(np.abs(x[f, :lp.q] - xv)) < 1e-9, f
        assert abs(st["objective"][f] - lp.objective_u(xv, g[f])) <= 1e-9 * (1 + abs(st["objective"][f]))
