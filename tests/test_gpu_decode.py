"""GPU parity of whole decodes against the oracle, through the C ABI.

Bar (decision outputs): hard decisions, certificates, final cut sets and
the number of LPs solved are bit-exact; u and the objective agree within
1e-6 (relative for the objective).
"""

import numpy as np
import pytest

import oracle
from paper_0902_0657_gb300 import lpdec as L
from synth import awgn_llr_frames, named_code
from synth.codes import from_rows

from .gpu_util import dev, host, torch_cuda

pytestmark = pytest.mark.gpu


def compare_frame(res, u, hard, cert, masks, st, ctx=""):
    assert st["status"] == res.status, ctx
    assert np.array_equal(hard, res.hard), ctx
    assert cert == res.cert, ctx
    assert np.array_equal(masks, res.masks), ctx
    assert st["alp_iters"] == res.alp_iters, ctx
    assert st["alp_switch"] == res.alp_switch, ctx
    assert st["lp_rows_final"] == res.lp_rows_final, ctx
    assert st["lp_rows_max"] == max([h.p for h in res.history] or [0]), ctx
    assert np.max(np.abs(u - res.u)) <= 1e-6, ctx
    assert abs(st["objective"] - res.objective) <= 1e-6 * (1 + abs(res.objective)), ctx


@pytest.mark.parametrize("precision,threads,precond", [
    (L.LPDEC_FP64, 128, L.LPDEC_MTS_COLUMN), (L.LPDEC_MIXED, 128, L.LPDEC_MTS_COLUMN),
    (L.LPDEC_M32, 128, L.LPDEC_MTS_COLUMN), (L.LPDEC_FP64, 32, L.LPDEC_MTS_COLUMN),
    (L.LPDEC_MIXED, 256, L.LPDEC_MTS_COLUMN), (L.LPDEC_M32, 64, L.LPDEC_MTS_COLUMN),
    (L.LPDEC_FP64, 128, L.LPDEC_MTS_INCREMENTAL), (L.LPDEC_FP64, 128, L.LPDEC_MTS_ROWWISE),
    (L.LPDEC_FP64, 128, L.LPDEC_MTS_ADAPTIVE), (L.LPDEC_FP64, 128, L.LPDEC_MTS_ROWWISE_TRI)])
def test_decode_gallager120_200_frames(precision, threads, precond):
    """(3,6) n=120, Eb/N0 2.0 dB, 200 frames from seed 0, in FP64, in mixed
    precision (FP32 PCG refined against FP64 residuals) and with the FP32
    preconditioner solve, at several CTA sizes, and with each of the
    triangular-set preconditioners of Section V (they change the PCG
    iterations, not the LP solutions), with PCG kept for every Newton system
    it solves (no early switch to the dense solve)."""
    torch_cuda()
    code = named_code("gallager_120")
    G = awgn_llr_frames(code.n, code.design_rate, 2.0, 0, range(200))
    prm = L.lpdec_default_params()
    prm.precision = precision
    prm.threads_per_block = threads
    prm.precond = precond
    prm.precond_switch = 20   # (n = 120: switch early enough to be exercised)
    prm.dense_switch = 0      # (PCG for every Newton solve that converges)
    with L.Decoder(code, params=prm) as d:
        u, hard, cert, masks, st = d.decode_batch(G)
    n_frac = 0
    for f in range(200):
        res = oracle.decode(code, G[f])
        compare_frame(res, u[f], hard[f], cert[f], masks[f], st[f], f"frame {f}")
        assert st["vertex_failures"][f] == 0
        n_frac += res.cert == 0
    assert 0 < n_frac < 200


def test_decode_alone_equals_in_batch():
    """Each frame's result does not depend on the other frames of the batch."""
    torch_cuda()
    code = named_code("gallager_120")
    G = awgn_llr_frames(code.n, code.design_rate, 1.5, 3, range(24))
    with L.Decoder(code) as d:
        ub, hb, cb, mb, sb = d.decode_batch(G)
        for f in (0, 7, 23):
            u1, h1, c1, m1, s1 = d.decode_batch(G[f:f + 1])
            assert np.array_equal(u1[0], ub[f]) and np.array_equal(h1[0], hb[f])
            assert c1[0] == cb[f] and np.array_equal(m1[0], mb[f])


def test_decode_edge_cases():
    torch = torch_cuda()
    code = named_code("gallager_120")
    with L.Decoder(code) as d:
        # empty batch
        e = np.zeros((0, code.n))
        rc = L.lpdec_decode_frames(d.ctx, d.code, 0, e, np.zeros((0, code.n)),
                                   np.zeros((0, code.n), np.uint8), np.zeros(0, np.int32))
        assert rc == 0
        # hard decision already a codeword: no LP is solved
        g = np.abs(awgn_llr_frames(code.n, code.design_rate, 2.0, 0, [0])) + 0.25
        u, hard, cert, masks, st = d.decode_batch(g)
        assert st["alp_iters"][0] == 0 and cert[0] == 1 and not hard.any() and not masks.any()
        # zero LLRs are accepted (treated as gamma >= 0). The LP optimum need
        # not be unique then (Theorem 2 assumes it is), so the decoder owes a
        # defined status, and the oracle's optimal cost whenever both converge.
        g0 = awgn_llr_frames(code.n, code.design_rate, 2.0, 0, [1])
        g0[0, ::7] = 0.0
        u, hard, cert, masks, st = d.decode_batch(g0)
        res = oracle.decode(code, g0[0])
        assert st["status"][0] in (L.LPDEC_OK, L.LPDEC_ERR_NOT_CONVERGED)
        if st["status"][0] == 0 and res.status == 0:
            assert abs(st["objective"][0] - res.objective) <= 1e-6 * (1 + abs(res.objective))
        # non-finite LLRs: host entry rejects the call
        bad = awgn_llr_frames(code.n, code.design_rate, 2.0, 0, [2])
        bad[0, 5] = np.nan
        rc = L.lpdec_decode_frames(d.ctx, d.code, 1, bad, np.zeros((1, code.n)),
                                   np.zeros((1, code.n), np.uint8), np.zeros(1, np.int32))
        assert rc == L.LPDEC_ERR_INVALID_ARG
        # ... and the device entry flags only that frame
        g2 = awgn_llr_frames(code.n, code.design_rate, 2.0, 0, [3, 4])
        g2[1, 0] = np.inf
        d_u = torch.zeros((2, code.n), dtype=torch.float64, device="cuda")
        d_h = torch.zeros((2, code.n), dtype=torch.uint8, device="cuda")
        d_c = torch.zeros(2, dtype=torch.int32, device="cuda")
        d_s = torch.zeros(2 * L.STATS_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        rc = L.lpdec_decode_batch_device(d.ctx, d.code, 2, dev(g2), d_u, d_h, d_c, None, d_s)
        torch.cuda.synchronize()
        st = host(d_s).view(L.STATS_DTYPE)
        assert rc == 0 and st["status"][0] == 0 and st["status"][1] == L.LPDEC_ERR_INVALID_ARG


def test_decode_ragged_degrees_up_to_32():
    """Irregular rows (degrees 1..32) exercise the warp-per-check search at
    its width limit and ragged CSR rows."""
    torch_cuda()
    rng = np.random.default_rng(2)
    n = 96
    rows = [sorted(rng.choice(n, size=d, replace=False)) for d in
            [32, 31, 17, 9, 6, 6, 5, 3, 2, 12, 8, 7, 6, 6, 6, 4, 1, 20]]
    code = from_rows(rows, n)
    G = awgn_llr_frames(n, 0.5, 1.0, 4, range(16))
    with L.Decoder(code) as d:
        u, hard, cert, masks, st = d.decode_batch(G)
    for f in range(16):
        res = oracle.decode(code, G[f])
        compare_frame(res, u[f], hard[f], cert[f], masks[f], st[f], f"frame {f}")


def test_code_create_validates_csr():
    torch_cuda()
    ctx = L.lpdec_ctx_create(0)
    try:
        rp = np.array([0, 2, 4], np.int32)
        for ci in (np.array([1, 0, 2, 3], np.int32),      # unsorted row
                   np.array([0, 1, 2, 9], np.int32)):     # column out of range
            with pytest.raises(L.LpdecError):
                L.lpdec_code_create(ctx, 2, 4, rp, ci)
        rp33 = np.array([0, 33], np.int32)                # degree 33 > 32
        with pytest.raises(L.LpdecError):
            L.lpdec_code_create(ctx, 1, 40, rp33, np.arange(33, dtype=np.int32))
    finally:
        L.lpdec_ctx_destroy(ctx)


def test_cost_stall_switches_to_alp_as_oracle():
    """Theorem 2(b) rule: with a required cost rise larger than any real one,
    every frame that needs an LP continues as ALP (Algorithm 1) after its
    first LP, and ends, as in the oracle, at the LP decoding optimum."""
    from oracle.params import OracleParams
    torch_cuda()
    code = named_code("gallager_120")
    G = awgn_llr_frames(code.n, code.design_rate, 2.0, 0, range(32))
    prm = L.lpdec_default_params()
    prm.tau_inc = 1e6
    with L.Decoder(code, params=prm) as d:
        u, hard, cert, masks, st = d.decode_batch(G)
    for f in range(32):
        res = oracle.decode(code, G[f], OracleParams(tau_inc=1e6))
        compare_frame(res, u[f], hard[f], cert[f], masks[f], st[f], f"frame {f}")
        assert res.alp_iters == 0 or res.alp_switch == 1


def test_alp_matches_oracle():
    """ALP (Algorithm 1: inequalities are only added, every check is searched
    in every round; several inequalities per check) against the oracle's
    ALP."""
    from oracle.params import OracleParams
    torch_cuda()
    code = named_code("gallager_120")
    G = awgn_llr_frames(code.n, code.design_rate, 2.0, 0, range(100))
    prm = L.lpdec_default_params()
    prm.variant = L.LPDEC_ALP
    with L.Decoder(code, params=prm) as d:
        u, hard, cert, masks, st = d.decode_batch(G)
    more_rows = 0
    for f in range(100):
        res = oracle.decode(code, G[f], OracleParams(variant="alp"))
        compare_frame(res, u[f], hard[f], cert[f], masks[f], st[f], f"frame {f}")
        more_rows += res.lp_rows_final > len(set(j for j, _ in res.cuts))
    assert more_rows > 0   # some LP held two inequalities of one check


def test_per_frame_failures_leave_the_rest_of_the_batch():
    """A cap that one frame hits ends only that frame. With max_ipm = 1 a
    frame that needs an LP ends LPDEC_ERR_NOT_CONVERGED (unless one
    interior-point step already certifies the optimal vertex, in which case
    it ends as in the oracle); with a row capacity of 4 every frame whose
    cut list outgrows it ends LPDEC_ERR_OUT_OF_BUDGET. In both batches the
    other frames, among them those whose hard decision is a codeword, end
    with the oracle's result."""
    torch_cuda()
    code = named_code("gallager_120")
    G = awgn_llr_frames(code.n, code.design_rate, 2.0, 0, range(16))
    G[::3] = np.abs(G[::3]) + 0.25          # every third frame: no LP needed
    ref = [oracle.decode(code, g) for g in G]
    assert sum(r.alp_iters == 0 for r in ref) >= 5 and sum(r.alp_iters > 0 for r in ref) >= 5
    for field, value, status in (("max_ipm", 1, L.LPDEC_ERR_NOT_CONVERGED),
                                 ("lp_rows_cap", 4, L.LPDEC_ERR_OUT_OF_BUDGET)):
        prm = L.lpdec_default_params()
        setattr(prm, field, value)
        with L.Decoder(code, params=prm) as d:
            u, hard, cert, masks, st = d.decode_batch(G)
        failed = 0
        for f in range(16):
            rows = max([h.p for h in ref[f].history] or [0])
            must_fail = (field == "lp_rows_cap" and rows > value)
            if must_fail or (field == "max_ipm" and st["status"][f] != L.LPDEC_OK):
                assert st["status"][f] == status, (field, f, st["status"][f])
                assert ref[f].alp_iters > 0
                failed += 1
            else:
                compare_frame(ref[f], u[f], hard[f], cert[f], masks[f], st[f], f"{field} {f}")
        assert failed >= 3, field


def test_mixed_code_lengths_share_one_launch():
    """Frames of three codes of different lengths (n = 504, 1008 and 2016)
    in one batch through lpdec_decode_batch (per-frame codes, one persistent
    launch over the ragged batch): each frame equals its single-code decode
    bit for bit, and the n=504 frames also equal the oracle."""
    torch_cuda()
    names = ["gallager_504", "peg_1008", "gallager_2016"]
    codes = [named_code(nm) for nm in names]
    frames = []
    for k, c in enumerate(codes):
        G = awgn_llr_frames(c.n, c.design_rate, 2.5, 40 + k, range(6))
        frames += [(k, g) for g in G]
    order = [0, 6, 12, 1, 7, 13, 2, 8, 14, 3, 9, 15, 4, 10, 16, 5, 11, 17]
    frames = [frames[t] for t in order]
    with L.Decoder(codes[0]) as d:
        handles = [d.code, d.add_code(codes[1]), d.add_code(codes[2])]
        u, hard, cert, masks, st = d.decode_mixed([handles[k] for k, _ in frames],
                                                  [g for _, g in frames])
        for k, c in enumerate(codes):
            idx = [t for t, (kk, _) in enumerate(frames) if kk == k]
            G = np.stack([frames[t][1] for t in idx])
            with L.Decoder(c) as d1:
                u1, h1, c1, m1, s1 = d1.decode_batch(G)
            for a, t in enumerate(idx):
                assert np.array_equal(u[t], u1[a]), (names[k], t)
                assert np.array_equal(hard[t], h1[a]) and cert[t] == c1[a]
                assert np.array_equal(masks[t], m1[a])
                for fld in ("status", "alp_iters", "ipm_iters_total", "pcg_iters_total",
                            "lp_rows_final", "alp_switch", "objective"):
                    assert st[fld][t] == s1[fld][a], (names[k], t, fld)
                if k == 0:
                    res = oracle.decode(c, G[a])
                    compare_frame(res, u[t], hard[t], cert[t], masks[t], st[t], f"frame {t}")


def test_malp_b_matches_oracle():
    """MALP-B (Section III-A: every inactive inequality is dropped before the
    search) against the oracle's MALP-B on the n=120 workload."""
    from oracle.params import OracleParams
    torch_cuda()
    code = named_code("gallager_120")
    G = awgn_llr_frames(code.n, code.design_rate, 2.0, 0, range(100))
    prm = L.lpdec_default_params()
    prm.variant = L.LPDEC_MALP_B
    with L.Decoder(code, params=prm) as d:
        u, hard, cert, masks, st = d.decode_batch(G)
    for f in range(100):
        res = oracle.decode(code, G[f], OracleParams(variant="malp_b"))
        compare_frame(res, u[f], hard[f], cert[f], masks[f], st[f], f"frame {f}")


@pytest.mark.parametrize("warm,reuse", [(1, 0), (0, 1), (1, 1)])
def test_warm_start_and_mts_reuse_match_oracle(warm, reuse):
    """The paper's future work (Sections V, VII): interior-point warm starts
    across the LPs of a frame and reuse of the triangular set across
    interior-point iterations change the path, not the certified LP
    solutions: decisions and values equal the oracle's (cold starts, direct
    Newton solves)."""
    torch_cuda()
    code = named_code("gallager_120")
    G = awgn_llr_frames(code.n, code.design_rate, 2.0, 0, range(200))
    prm = L.lpdec_default_params()
    prm.warm_start = warm
    prm.mts_reuse = reuse
    with L.Decoder(code, params=prm) as d:
        u, hard, cert, masks, st = d.decode_batch(G)
    for f in range(200):
        res = oracle.decode(code, G[f])
        compare_frame(res, u[f], hard[f], cert[f], masks[f], st[f], f"frame {f}")


def test_autotune_picks_a_schedule_and_decodes_exactly():
    """lpdec_autotune times every lanes-per-row schedule of the triangular
    solves on a sample and keeps the fastest in the context; decoding with
    it (and with each fixed schedule) still gives the oracle's results."""
    torch_cuda()
    code = named_code("gallager_120")
    sample = awgn_llr_frames(code.n, code.design_rate, 3.0, 1, range(64))
    G = awgn_llr_frames(code.n, code.design_rate, 2.0, 0, range(60))
    ref = [oracle.decode(code, g) for g in G]
    with L.Decoder(code) as d:
        rc, pol, secs = L.lpdec_autotune(d.ctx, d.code, sample)
        assert rc == 0 and pol in (0, 1, 2, 4, 8) and np.all(secs > 0)
        u, hard, cert, masks, st = d.decode_batch(G)
    for f in range(60):
        compare_frame(ref[f], u[f], hard[f], cert[f], masks[f], st[f], f"tuned {pol}, frame {f}")
    for pol in (1, 2, 4, 8):
        prm = L.lpdec_default_params()
        prm.lane_policy = pol
        with L.Decoder(code, params=prm) as d:
            u, hard, cert, masks, st = d.decode_batch(G)
        for f in range(60):
            compare_frame(ref[f], u[f], hard[f], cert[f], masks[f], st[f], f"policy {pol}, frame {f}")


def test_frame_order_changes_start_times_not_results():
    """order_frames = 2 hands out the frames with the largest sum of
    -gamma_i over gamma_i < 0 first (they tend to need the most LPs), 0 in
    the given order: the per-frame results are identical, and with many
    more frames than CTAs the highest-sum frames start earlier."""
    torch_cuda()
    code = named_code("gallager_120")
    G = awgn_llr_frames(code.n, code.design_rate, 1.5, 5, range(3000))
    out = {}
    for mode in (0, 1, 2):
        prm = L.lpdec_default_params()
        prm.order_frames = mode
        with L.Decoder(code, params=prm) as d:
            rc, grid, ordered = L.lpdec_batch_grid(d.ctx, d.code, len(G))
            assert rc == 0 and 0 < grid < len(G) and ordered == (mode > 0)
            assert L.lpdec_batch_grid(d.ctx, d.code, grid)[2] == (mode == 2)
            out[mode] = d.decode_batch(G)
    for mode in (1, 2):
        for a, b in zip(out[0][:4], out[mode][:4]):
            assert np.array_equal(a, b), mode
        for fld in ("status", "alp_iters", "ipm_iters_total", "pcg_iters_total", "lp_rows_final",
                    "alp_switch", "objective"):
            assert np.array_equal(out[0][4][fld], out[mode][4][fld]), (mode, fld)
    key = np.where(G < 0, -G, 0.0).sum(axis=1)
    rank = np.argsort(-key, kind="stable")
    t = out[2][4]["t_start"]
    assert np.mean(t[rank[:300]]) < np.mean(t[rank[-300:]])
    t0 = out[0][4]["t_start"]
    assert np.mean(t0[:300]) < np.mean(t0[-300:])
