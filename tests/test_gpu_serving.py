"""Serving entry points (lpdec_server_create / lpdec_submit / lpdec_poll)
through the C ABI: frames submitted in waves while earlier ones are on the
GPU come back identical to the same frames decoded alone by the batch entry
point, and admission stops at max_pending outstanding frames."""

import time

import numpy as np
import pytest

from paper_0902_0657_gb300 import lpdec as L
from synth import awgn_llr_frames, named_code

from .gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def _wait(srv, tickets, limit_s=300.0):
    out, t0 = {}, time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = srv.poll(t)
                if r is not None:
                    out[t] = r
        assert time.time() - t0 < limit_s, "serving results overdue"
        time.sleep(0.002)
    return out


def test_waves_equal_alone():
    torch_cuda()
    code = named_code("gallager_120")
    G = awgn_llr_frames(code.n, code.design_rate, 1.5, 7, range(150))
    with L.Server(code, lanes=2, batch=32) as srv:
        tickets = []
        for w in range(3):                       # three arrival waves
            tickets += [srv.submit(G[f]) for f in range(50 * w, 50 * w + 50)]
            time.sleep(0.01)
        assert tickets == list(range(150))
        res = _wait(srv, tickets)
        for t in (tickets[0], 10 ** 6):           # already polled, never issued
            with pytest.raises(L.LpdecError):
                srv.poll(t)
    with L.Decoder(code) as d:
        u, hard, cert, masks, st = d.decode_batch(G)
    for f, t in enumerate(tickets):
        ru, rh, rc, rs = res[t]
        assert np.array_equal(ru, u[f]), f
        assert np.array_equal(rh, hard[f]), f
        assert rc == cert[f] and rs["status"] == st["status"][f]
        assert rs["alp_iters"] == st["alp_iters"][f]


def test_admission_budget():
    torch_cuda()
    code = named_code("gallager_120")
    G = awgn_llr_frames(code.n, code.design_rate, 2.0, 3, range(6))
    with L.Server(code, lanes=1, batch=4, max_pending=4) as srv:
        tickets = [srv.submit(G[f]) for f in range(4)]
        rc, _ = L.lpdec_submit(srv.handle, G[4])
        assert rc == L.LPDEC_ERR_OUT_OF_BUDGET
        _wait(srv, tickets)
        assert srv.submit(G[5]) == 4              # a slot is free again
        _wait(srv, [4])
