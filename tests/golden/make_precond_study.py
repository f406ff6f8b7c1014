"""Writes tests/golden/precond_study_peg2000.json: Newton systems of late
interior-point iterations of fractional LPs, the inputs of the
preconditioner study of Section VI-B (Figs. 5-8: residual against PCG
iteration for plain CG and the three triangular-set preconditioners).

Workload: the (3,6) PEG-style code n = 2000, m = 1000 (seed 0), BPSK over
AWGN at Eb/N0 1.5 dB and 1.0 dB (seed-0 frame pool). For each SNR the
first frame whose LP decoding output is fractional is decoded by the
oracle; the last LP of its adaptive loop is solved by the oracle's
interior-point method with a trace, and the Newton systems (D^2, right side
w) of its iterations at one half, three quarters and the end of the run are
stored with the LP (cut set per check).

Every value comes from the oracle; nothing is read from the CUDA path. Run
from the repository root (a few minutes):
    python tests/golden/make_precond_study.py
"""

from __future__ import annotations

import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

OUT = os.path.join(ROOT, "tests", "golden", "precond_study_peg2000.json")


def main():
    import oracle
    from oracle import ipm
    from oracle import lp as olp
    from oracle.params import OracleParams
    from synth import awgn_llr_frames, named_code
    code = named_code("peg_2000")
    cases = []
    for eb in (1.5, 1.0):
        for f in range(64):
            g = awgn_llr_frames(code.n, code.design_rate, eb, 0, [f])[0]
            r = oracle.decode(code, g)
            if r.cert == 0 and r.history:
                break
        h = r.history[-1]
        L = olp.build(code, g, h.in_lp, h.masks)
        trace = []
        ipm.solve(L.A, L.b, L.c, OracleParams(), trace=trace)
        its = sorted({len(trace) // 2, (3 * len(trace)) // 4, len(trace) - 1})
        cases.append({
            "ebn0": eb, "frame": f, "p": int(L.p), "q": int(L.q), "ipm_iters": len(trace),
            "in_lp": [int(v) for v in h.in_lp], "masks": [int(v) for v in h.masks],
            "systems": [{"iteration": int(k), "gap": float(trace[k]["gap"]),
                         "d2": [float(v) for v in trace[k]["d2"]],
                         "w": [float(v) for v in trace[k]["w"]]} for k in its],
        })
        print(f"{eb} dB: frame {f}, p {L.p}, {len(trace)} iterations, systems at {its}", flush=True)
    with open(OUT, "w") as fh:
        json.dump({"code": "peg_2000", "seed": 0,
                   "written_by": "tests/golden/make_precond_study.py (oracle only)",
                   "cases": cases}, fh, separators=(",", ":"))
        fh.write("\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main()
