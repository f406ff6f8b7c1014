"""Writes tests/golden/peg1008_oracle.json: oracle decodes of the benchmark's
code at full size, the expected values of the full-size GPU parity test.

Workload (Sections III-D and VI-B: random (3,6) codes without 4-cycles,
all-zero codeword, BPSK over AWGN): the (3,6) PEG-style code n = 1008,
m = 504 (seed 0), frames 0..63 of the seed-0 pool at each Eb/N0 in
{1.5, 2.0, 2.5, 3.0} dB, plus frames 6188 and 8718 at 2.0 dB, two frames
whose MALP-A cost stopped rising when LP vertices were accepted without a
dual certificate (they reach the full-LP optimum with certified LPs).

Every value comes from oracle.decode (FP64, dense Newton solves) with the
default parameters; nothing is read from the CUDA path. Per frame it
stores the status, the certificate, the numbers of LPs and of LPs before a
switch to ALP, the rows of the last LP, the cost gamma'u, the hard decision
(hex, bit i of the little-endian bit string = hard_i), the final cut set
(two hex digits per check: mask[j], 0 = no inequality) and u as the hard
decision plus the entries that differ from it by more than 1e-12 (as
[index, value] pairs).

Run from the repository root (about 5 minutes on 8 cores):
    python tests/golden/make_peg1008.py
"""

from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

OUT = os.path.join(ROOT, "tests", "golden", "peg1008_oracle.json")
CODE = "peg_1008"
SEED = 0
SNRS = (1.5, 2.0, 2.5, 3.0)
FRAMES = 64
EXTRA = ((2.0, 6188), (2.0, 8718))


def cases():
    out = [(eb, f) for eb in SNRS for f in range(FRAMES)]
    return out + [c for c in EXTRA if c not in out]


def decode_one(case):
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    import numpy as np
    import oracle
    from synth import awgn_llr_frames, named_code
    eb, f = case
    code = named_code(CODE)
    g = awgn_llr_frames(code.n, code.design_rate, eb, SEED, [f])[0]
    r = oracle.decode(code, g)
    hard = r.hard.astype(np.uint8)
    dev = np.flatnonzero(np.abs(r.u - hard) > 1e-12)
    return {
        "ebn0": eb, "frame": f, "status": int(r.status), "cert": int(r.cert),
        "alp_iters": int(r.alp_iters), "alp_switch": int(r.alp_switch),
        "lp_rows_final": int(r.lp_rows_final), "objective": float(r.objective),
        "hard": np.packbits(hard, bitorder="little").tobytes().hex(),
        "masks": "".join(f"{int(x):02x}" for x in r.masks),
        "u_dev": [[int(i), float(r.u[i])] for i in dev],
    }


def main():
    cs = cases()
    workers = max(1, (os.cpu_count() or 2) - 1)
    with mp.get_context("spawn").Pool(workers) as pool:
        rows = pool.map(decode_one, cs, chunksize=1)
    doc = {
        "what": "oracle decodes of the (3,6) PEG n=1008 code (seed 0), seed-0 frame pool",
        "code": CODE, "seed": SEED, "n": 1008, "m": 504,
        "written_by": "tests/golden/make_peg1008.py (oracle only)",
        "frames": rows,
    }
    with open(OUT, "w") as fh:
        json.dump(doc, fh, separators=(",", ":"))
        fh.write("\n")
    print(f"wrote {OUT}: {len(rows)} frames")


if __name__ == "__main__":
    main()
