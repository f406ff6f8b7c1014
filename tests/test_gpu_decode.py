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
    assert st["lp_rows_final"] == res.lp_rows_final, ctx
    assert np.max(np.abs(u - res.u)) <= 1e-6, ctx
    assert abs(st["objective"] - res.objective) <= 1e-6 * (1 + abs(res.objective)), ctx


@pytest.mark.parametrize("precision,threads", [(L.LPDEC_FP64, 128), (L.LPDEC_MIXED, 128),
                                               (L.LPDEC_M32, 128), (L.LPDEC_FP64, 32),
                                               (L.LPDEC_MIXED, 256), (L.LPDEC_M32, 64)])
def test_decode_gallager120_200_frames(precision, threads):
    """(3,6) n=120, Eb/N0 2.0 dB, 200 frames from seed 0, in FP64, in mixed
    precision (FP32 PCG refined against FP64 residuals) and with the FP32
    preconditioner solve, at several CTA sizes."""
    torch_cuda()
    code = named_code("gallager_120")
    G = awgn_llr_frames(code.n, code.design_rate, 2.0, 0, range(200))
    prm = L.lpdec_default_params()
    prm.precision = precision
    prm.threads_per_block = threads
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
        rc = L.lpdec_decode_batch(d.ctx, d.code, 0, e, np.zeros((0, code.n)),
                                  np.zeros((0, code.n), np.uint8), np.zeros(0, np.int32))
        assert rc == 0
        # hard decision already a codeword: no LP is solved
        g = np.abs(awgn_llr_frames(code.n, code.design_rate, 2.0, 0, [0])) + 0.25
        u, hard, cert, masks, st = d.decode_batch(g)
        assert st["alp_iters"][0] == 0 and cert[0] == 1 and not hard.any() and not masks.any()
        # zero LLRs are accepted (treated as gamma >= 0). The LP optimum need
        # not be unique then and Theorem 2 (strictly increasing cost, hence
        # termination) assumes it is, so the decoder only owes a defined
        # status, and the oracle's optimal cost whenever both converge.
        g0 = awgn_llr_frames(code.n, code.design_rate, 2.0, 0, [1])
        g0[0, ::7] = 0.0
        u, hard, cert, masks, st = d.decode_batch(g0)
        res = oracle.decode(code, g0[0])
        assert st["status"][0] in (L.LPDEC_OK, L.LPDEC_ERR_NOT_CONVERGED, L.LPDEC_ERR_STALLED)
        if st["status"][0] == 0 and res.status == 0:
            assert abs(st["objective"][0] - res.objective) <= 1e-6 * (1 + abs(res.objective))
        # non-finite LLRs: host entry rejects the call
        bad = awgn_llr_frames(code.n, code.design_rate, 2.0, 0, [2])
        bad[0, 5] = np.nan
        rc = L.lpdec_decode_batch(d.ctx, d.code, 1, bad, np.zeros((1, code.n)),
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


def test_stall_rule_matches_oracle():
    """Theorem 2(b) stop rule: with a required cost rise larger than any
    real one, every frame that needs an LP stops after its first LP with
    LPDEC_ERR_STALLED, and its outputs are that LP's, as in the oracle."""
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
        assert res.alp_iters == 0 or (res.status == L.LPDEC_ERR_STALLED and res.alp_iters == 1)


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
