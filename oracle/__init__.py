"""CPU FP64 oracle for adaptive LP decoding — TEST INFRASTRUCTURE ONLY.

This package is the plain, slow, obviously correct reference against which
the CUDA decoder is checked. Only the test suite, the smoke check and the
CPU-baseline leg of the benchmark may import or run it; the decoder library
never does, and the two share no code (the only common inputs come from the
``synth`` generators).

Contents, each following the paper (Taghavi, Shokrollahi, Siegel,
"Efficient Implementation of Linear Programming Decoding"):

* ``params``   — every tolerance and rule the paper leaves open.
* ``cuts``     — parity inequalities (Eqs. 5-6) and Algorithm 2, the O(d_j)
                 search for the violated inequality of one check.
* ``lp``       — the augmented primal LP of Section IV-B (flip to x >= 0,
                 slack columns), built from the current cut set.
* ``ipm``      — the infeasible primal-dual path-following method of
                 Section IV-B; the Newton step's normal equations (Eq. 24)
                 are solved by dense Cholesky, a direct method.
* ``malp``     — Algorithm 3 (MALP-A), its variant MALP-B and Algorithm 1
                 (ALP): the adaptive cutting-plane decoder.
* ``mts``      — the MTS preconditioners of Section V (Algorithms 5-8), the
                 M-solve by two triangular substitutions, and the PCG method
                 (Algorithm 4).
* ``feldman``  — the plain definitions the decoder must reproduce on small
                 codes: LP decoding over the full fundamental polytope
                 (Eq. 7, all parity inequalities) and exhaustive ML decoding
                 (Eq. 3).
"""

from .params import OracleParams  # noqa: F401
from .malp import decode, DecodeResult  # noqa: F401
