"""Serving entry points (lpdec_server_create / lpdec_submit / lpdec_poll /
lpdec_cancel) through the C ABI: continuous batching of frames of several
code lengths. Frames submitted in waves while earlier ones run come back
identical to the same frames decoded alone by the batch entry point; a
frame submitted while a long batch runs is taken by a free CTA of the
running kernel and finishes first; admission counts device-memory bytes;
cancelled tickets are released, and cancelled running frames stop."""

import time

import numpy as np
import pytest

from paper_0902_0657_gb300 import lpdec as L
from synth import awgn_llr_frames, named_code

from .gpu_util import torch_cuda

pytestmark = pytest.mark.gpu

FIELDS = ("status", "alp_iters", "alp_switch", "ipm_iters_total", "pcg_iters_total",
          "lp_rows_final", "objective")


def _wait(srv, tickets, limit_s=300.0):
    out, t0 = {}, time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = srv.poll(t)
                if r is not None:
                    out[t] = (r, time.time())
        assert time.time() - t0 < limit_s, "serving results overdue"
        time.sleep(0.001)
    return out


def test_mixed_lengths_in_waves_equal_alone():
    torch_cuda()
    codes = [named_code(nm) for nm in ("gallager_504", "peg_1008", "gallager_2016")]
    frames = []
    for k, c in enumerate(codes):
        G = awgn_llr_frames(c.n, c.design_rate, 2.0, 60 + k, range(30))
        frames += [(k, f, G[f]) for f in range(30)]
    rng = np.random.default_rng(1)
    order = rng.permutation(len(frames))
    with L.Server(codes) as srv:
        tickets = []
        for w in range(3):                              # three arrival waves
            for t in order[30 * w:30 * w + 30]:
                k, f, g = frames[t]
                tickets.append((t, srv.submit(g, code=k)))
            time.sleep(0.02)
        res = _wait(srv, [tk for _, tk in tickets])
        with pytest.raises(L.LpdecError):               # already polled
            srv.poll(tickets[0][1])
    for k, c in enumerate(codes):
        G = awgn_llr_frames(c.n, c.design_rate, 2.0, 60 + k, range(30))
        with L.Decoder(c) as d:
            u, hard, cert, masks, st = d.decode_batch(G)
        for t, tk in tickets:
            kk, f, _ = frames[t]
            if kk != k:
                continue
            (ru, rh, rc, rm, rs), _ = res[tk]
            ctx = (c.n, f)
            assert np.array_equal(ru, u[f]), ctx
            assert np.array_equal(rh, hard[f]) and rc == cert[f], ctx
            assert np.array_equal(rm, masks[f]), ctx
            for fld in FIELDS:
                assert rs[fld] == st[fld][f], (ctx, fld)


def test_frame_submitted_during_a_long_batch_finishes_first():
    """64 slow frames (1.5 dB: many fractional, seconds each) occupy 64 CTAs
    of the running kernel; a frame submitted 50 ms later is taken by another
    CTA at once and its result is ready before the slow batch's last."""
    torch_cuda()
    c = named_code("peg_1008")
    slow = awgn_llr_frames(c.n, c.design_rate, 1.5, 0, range(64))
    easy = awgn_llr_frames(c.n, c.design_rate, 4.0, 9, [0])[0]
    with L.Server([c]) as srv:
        ts = [srv.submit(g) for g in slow]
        time.sleep(0.05)
        te = srv.submit(easy)
        res = _wait(srv, ts + [te])
    t_easy = res[te][1]
    t_last = max(res[t][1] for t in ts)
    assert t_easy < t_last
    assert sum(res[t][1] > t_easy for t in ts) >= 1


def test_admission_counts_device_bytes():
    """An arena of two n=1008 regions and one n=120 region: two n=1008
    frames are admitted, a third is refused while they run, an n=120 frame
    still fits; once results are polled, n=1008 frames fit again."""
    torch_cuda()
    big, small = named_code("peg_1008"), named_code("gallager_120")
    Rb, Rs = L.region_bytes(big.n, big.m), L.region_bytes(small.n, small.m)
    with L.Server([big, small], max_pending=1) as probe:
        hbm, arena, used, out = probe.stats()
    scratch = hbm - arena
    # slow frames (21-25 LPs each in the oracle) and a fast one
    Gb = awgn_llr_frames(big.n, big.design_rate, 1.5, 0, [39, 9, 56, 0])
    Gs = awgn_llr_frames(small.n, small.design_rate, 2.0, 0, range(2))
    with L.Server([big, small], hbm_budget_bytes=scratch + 2 * Rb + Rs) as srv:
        assert srv.stats()[1] == 2 * Rb + Rs
        t0 = srv.submit(Gb[0], code=0)
        t1 = srv.submit(Gb[1], code=0)
        rc, _ = srv.try_submit(Gb[2], code=0)
        assert rc == L.LPDEC_ERR_OUT_OF_BUDGET
        t2 = srv.submit(Gs[0], code=1)
        assert srv.stats()[2] >= 2 * Rb          # the two slow frames still hold theirs
        _wait(srv, [t0, t1, t2])
        assert srv.stats()[2] == 0
        t3 = srv.submit(Gb[3], code=0)
        _wait(srv, [t3])


def test_cancel_releases_tickets_and_bytes():
    torch_cuda()
    c = named_code("gallager_120")
    G = awgn_llr_frames(c.n, c.design_rate, 1.5, 2, range(40))
    with L.Server([c]) as srv:
        ts = [srv.submit(g) for g in G]
        for t in ts[::4]:
            srv.cancel(t)
        keep = [t for k, t in enumerate(ts) if k % 4]
        _wait(srv, keep)
        for t in ts[::4]:
            with pytest.raises(L.LpdecError):
                srv.poll(t)
        t0 = time.time()
        while srv.stats()[2] and time.time() - t0 < 60:   # cancelled frames still running
            time.sleep(0.01)
        hbm, arena, used, out = srv.stats()
        assert used == 0 and out == 0


def test_cancel_stops_running_frames():
    """A cancelled frame that is running stops at its next check of the
    cancel flag (between LPs, every fourth interior-point iteration): the
    slowest frames of a 1.5 dB pool, seconds each when decoded, release
    their CTAs and regions well within that time, and frames submitted
    afterwards decode exactly as in a batch."""
    torch_cuda()
    c = named_code("peg_1008")
    pool = awgn_llr_frames(c.n, c.design_rate, 1.5, 4, range(200))
    key = np.where(pool < 0, -pool, 0.0).sum(axis=1)
    hard = pool[np.argsort(-key)[:16]]
    easy = awgn_llr_frames(c.n, c.design_rate, 3.0, 9, range(4))
    with L.Decoder(c) as d:
        st = d.decode_batch(hard)[4]
        ue, he, ce, me, se = d.decode_batch(easy)
    longest = float(st["seconds"].max())
    assert longest > 2.0, longest   # (these frames do take seconds)
    with L.Server([c]) as srv:
        ts = [srv.submit(g) for g in hard]
        time.sleep(0.5)
        t0 = time.time()
        for t in ts:
            srv.cancel(t)
        while srv.stats()[2] and time.time() - t0 < 120:
            time.sleep(0.005)
        released = time.time() - t0
        hbm, arena, used, out = srv.stats()
        assert used == 0 and out == 0
        assert released < min(3.0, 0.5 * longest), (released, longest)
        te = [srv.submit(g) for g in easy]
        res = _wait(srv, te)
    for k, t in enumerate(te):
        u, h, cert, mask, s = res[t][0]
        assert np.array_equal(h, he[k]) and cert == ce[k] and np.array_equal(u, ue[k])
        assert np.array_equal(mask, me[k]) and s["status"] == se["status"][k]
