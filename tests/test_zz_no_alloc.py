"""The allocation-free batch decode (lpdec_decode_batch_device_noalloc) is
for callers that cannot allocate device memory at decode time. It keeps its
workspace in one fixed device array inside the library, shared by every
call, so this checks, through the C ABI, that two calls in a row both give
the results of the regular device entry point (which uses context-owned
scratch): identical decisions, and u and the cost within 1e-6."""

import numpy as np
import pytest

from paper_0902_0657_gb300 import lpdec as L
from synth import awgn_llr_frames, named_code

from .gpu_util import dev, host, torch_cuda

pytestmark = pytest.mark.gpu


def outputs(torch, nf, n, m):
    return (torch.zeros((nf, n), dtype=torch.float64, device="cuda"),
            torch.zeros((nf, n), dtype=torch.uint8, device="cuda"),
            torch.zeros(nf, dtype=torch.int32, device="cuda"),
            torch.zeros((nf, m), dtype=torch.int32, device="cuda"),
            torch.zeros(nf * L.STATS_DTYPE.itemsize, dtype=torch.uint8, device="cuda"))


def to_host(o):
    u, h, c, mk, st = o
    return host(u), host(h), host(c), host(mk), host(st).view(L.STATS_DTYPE)


@pytest.mark.parametrize("name,nf,ebn0,precision,smem_budget,seed", [
    ("gallager_120", 64, 2.0, L.LPDEC_FP64, 0, 21),
    ("gallager_120", 64, 2.0, L.LPDEC_MIXED, 0, 21),
    ("peg_1008", 8, 3.0, L.LPDEC_FP64, 0, 21),
    # frames whose Newton solves reach the dense fallback
    ("peg_1008", 24, 2.0, L.LPDEC_FP64, 0, 0),
    # most arrays in global scratch: more frames than the array has CTA
    # slots, so CTAs take several frames each from the queue
    ("gallager_120", 900, 2.0, L.LPDEC_FP64, 8192, 5),
])
def test_noalloc_matches_regular_entry_twice(name, nf, ebn0, precision, smem_budget, seed):
    torch = torch_cuda()
    code = named_code(name)
    G = dev(awgn_llr_frames(code.n, code.design_rate, ebn0, seed, range(nf)))
    prm = L.lpdec_default_params()
    prm.precision = precision
    prm.smem_budget = smem_budget
    with L.Decoder(code, params=prm) as d:
        ref = outputs(torch, nf, code.n, code.m)
        rc = L.lpdec_decode_batch_device(d.ctx, d.code, nf, G, *ref)
        assert rc == 0
        torch.cuda.synchronize()
        ru, rh, rc_, rm, rs = to_host(ref)
        if name == "peg_1008" and ebn0 == 2.0:
            assert rs["dense_solves"].sum() > 0
        for call in range(2):
            out = outputs(torch, nf, code.n, code.m)
            rc = L.lpdec_decode_batch_device_noalloc(d.code, prm, nf, G, *out)
            assert rc == 0, L.error_string(rc)
            torch.cuda.synchronize()
            u, h, c, mk, st = to_host(out)
            assert np.array_equal(h, rh), call
            assert np.array_equal(c, rc_), call
            assert np.array_equal(mk, rm), call
            assert np.array_equal(st["status"], rs["status"]), call
            assert np.array_equal(st["alp_iters"], rs["alp_iters"]), call
            assert np.array_equal(st["dense_solves"], rs["dense_solves"]), call
            assert np.max(np.abs(u - ru)) <= 1e-6, call
            assert np.all(np.abs(st["objective"] - rs["objective"])
                          <= 1e-6 * (1 + np.abs(rs["objective"]))), call
