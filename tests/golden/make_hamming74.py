"""Writes tests/golden/hamming74_pseudocodeword.json.

Remark 1 (Section III-B) cites the pseudocodeword w = [1, 1/2, 0, 1/2, 0, 0,
1/2] of the (7,4,3) Hamming code, which has exactly m = 3 fractional entries.
The paper does not print the parity-check matrix it belongs to. This script
searches the column orders of the 3 x 7 Hamming matrix (columns = the binary
expansions of 1..7) for one under which w is a vertex of the fundamental
polytope P: w satisfies every parity inequality (Eq. 5) and the box, and the
inequalities tight at w have rank 7. It then takes gamma = -sum_k lambda_k
a_k over the normals a_k of all tight inequalities (box included) with
weights lambda_k = k + 1 > 0. This puts gamma strictly inside the normal cone
of P at w, so w is the unique LP decoding optimum (Section II-A: every vertex
is the unique solution for some cost); the first column order whose gamma has
no zero entry is kept.

It uses only the oracle (parity inequalities) and the synthetic Hamming
constructor. Run from the repository root:
    python tests/golden/make_hamming74.py
"""

from __future__ import annotations

import itertools
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.feldman import parity_inequalities  # noqa: E402
from synth.codes import hamming74  # noqa: E402

W = np.array([1.0, 0.5, 0.0, 0.5, 0.0, 0.0, 0.5])


def tight_normals(code, w):
    A, b = parity_inequalities(code)
    lhs = A @ w
    if np.any(lhs > b + 1e-12):
        return None
    normals = [A[k] for k in np.flatnonzero(np.abs(lhs - b) <= 1e-12)]
    for i in range(code.n):            # box: -u_i <= 0 and u_i <= 1
        if w[i] == 0.0:
            e = np.zeros(code.n)
            e[i] = -1.0
            normals.append(e)
        if w[i] == 1.0:
            e = np.zeros(code.n)
            e[i] = 1.0
            normals.append(e)
    return np.asarray(normals)


def main():
    for order in itertools.permutations(range(1, 8)):
        code = hamming74(order)
        N = tight_normals(code, W)
        if N is None or np.linalg.matrix_rank(N) < 7:
            continue
        lam = np.arange(1, N.shape[0] + 1, dtype=np.float64)
        gamma = -(lam[:, None] * N).sum(axis=0)
        if np.any(gamma == 0):
            continue
        out = {
            "citation": "Remark 1, Section III-B: pseudocodeword "
                        "[1, 1/2, 0, 1/2, 0, 0, 1/2] of the (7,4,3) code, "
                        "m = 3 fractional entries",
            "col_order": list(order),
            "H": code.dense().tolist(),
            "gamma": gamma.tolist(),
            "u_expected": W.tolist(),
            "cert_expected": 0,
            "tight_inequalities": int(N.shape[0]),
        }
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                            "hamming74_pseudocodeword.json")
        with open(path, "w") as f:
            json.dump(out, f, indent=1)
        print("wrote", path, "col_order", order, "gamma", gamma)
        return
    raise SystemExit("no column order makes w a vertex")


if __name__ == "__main__":
    main()
