"""Full-size parity against stored oracle decodes (tests/golden/
peg1008_oracle.json, written by tests/golden/make_peg1008.py, which calls
only the oracle): the benchmark's (3,6) PEG code n = 1008 at Eb/N0 1.5, 2.0,
2.5 and 3.0 dB, 64 frames each plus two 2.0 dB frames (6188, 8718) whose
MALP cost stopped rising when LP vertices were not certified. Each SNR's
frames are decoded in one
persistent launch of the device entry point with the library's default
layout, in each precision mode.

Bar (Section II-B certificate, Theorem 2(c)): status, hard decision,
certificate, final cut set, number of LPs and of LPs before a switch to
ALP, and the rows of the last LP bit-exact; u and gamma'u within 1e-6.
"""

import json
import os

import numpy as np
import pytest

from paper_0902_0657_gb300 import lpdec as L
from synth import awgn_llr_frames, named_code

from .gpu_util import dev, host, torch_cuda

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "peg1008_oracle.json")


def load():
    with open(GOLDEN) as f:
        doc = json.load(f)
    code = named_code(doc["code"])
    rows = doc["frames"]
    for r in rows:
        bits = np.frombuffer(bytes.fromhex(r["hard"]), np.uint8)
        r["hard_v"] = np.unpackbits(bits, bitorder="little")[:code.n]
        r["masks_v"] = np.array([int(r["masks"][2 * j:2 * j + 2], 16) for j in range(code.m)],
                                np.uint32)
        u = r["hard_v"].astype(np.float64)
        for i, v in r["u_dev"]:
            u[i] = v
        r["u_v"] = u
    return code, doc["seed"], rows


def test_golden_file_covers_the_workload():
    code, seed, rows = load()
    snrs = sorted({r["ebn0"] for r in rows})
    assert snrs == [1.5, 2.0, 2.5, 3.0]
    assert all(sum(r["ebn0"] == e for r in rows) >= 64 for e in snrs)
    assert sum(r["cert"] == 0 for r in rows) >= 20          # fractional outputs
    assert {6188, 8718} <= {r["frame"] for r in rows if r["ebn0"] == 2.0}


@pytest.mark.gpu
@pytest.mark.parametrize("precision,dense_switch", [
    (L.LPDEC_FP64, 64), (L.LPDEC_M32, 64), (L.LPDEC_MIXED, 64),
    (L.LPDEC_FP64, 0), (L.LPDEC_FP64, 1)])
def test_full_size_matches_oracle_goldens(precision, dense_switch):
    """Every precision mode with the default switch to the dense solve,
    and FP64 with PCG until it stalls (0) or the dense solve for almost
    every Newton system (1)."""
    torch = torch_cuda()
    code, seed, rows = load()
    prm = L.lpdec_default_params()
    prm.precision = precision
    prm.dense_switch = dense_switch
    worst_u = 0.0
    failures = []
    with L.Decoder(code, params=prm) as d:
        for eb in sorted({r["ebn0"] for r in rows}):
            grp = [r for r in rows if r["ebn0"] == eb]
            G = awgn_llr_frames(code.n, code.design_rate, eb, seed, [r["frame"] for r in grp])
            nf = len(grp)
            d_u = torch.zeros((nf, code.n), dtype=torch.float64, device="cuda")
            d_h = torch.zeros((nf, code.n), dtype=torch.uint8, device="cuda")
            d_c = torch.zeros(nf, dtype=torch.int32, device="cuda")
            d_m = torch.zeros((nf, code.m), dtype=torch.int32, device="cuda")
            d_s = torch.zeros(nf * L.STATS_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
            rc = L.lpdec_decode_batch_device(d.ctx, d.code, nf, dev(G), d_u, d_h, d_c, d_m, d_s)
            assert rc == 0, L.error_string(rc)
            torch.cuda.synchronize()
            u, h, c = host(d_u), host(d_h), host(d_c)
            mk, st = host(d_m).view(np.uint32), host(d_s).view(L.STATS_DTYPE)
            for k, r in enumerate(grp):
                ctx = (eb, r["frame"])
                bad = []
                if st["status"][k] != r["status"]:
                    bad.append(f"status {st['status'][k]} vs {r['status']}")
                if not np.array_equal(h[k], r["hard_v"]):
                    bad.append("hard")
                if c[k] != r["cert"]:
                    bad.append("cert")
                du = float(np.max(np.abs(u[k] - r["u_v"])))
                worst_u = max(worst_u, du)
                if du > 1e-6:
                    bad.append(f"u {du:.1e}")
                if abs(st["objective"][k] - r["objective"]) > 1e-6 * (1 + abs(r["objective"])):
                    bad.append("objective")
                if not np.array_equal(mk[k], r["masks_v"]):
                    bad.append(f"cut set ({int((mk[k] != r['masks_v']).sum())} checks)")
                for fld in ("alp_iters", "alp_switch", "lp_rows_final"):
                    if st[fld][k] != r[fld]:
                        bad.append(f"{fld} {st[fld][k]} vs {r[fld]}")
                if bad:
                    failures.append((ctx, bad))
    print(f"precision {precision}, dense_switch {dense_switch}: "
          f"max |u - u_oracle| = {worst_u:.3e}")
    assert not failures, failures
