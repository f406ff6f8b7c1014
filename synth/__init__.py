"""Seeded synthetic inputs for LP decoding: LDPC parity-check matrices and
BPSK/AWGN channel LLRs.

This package holds only input generation. It contains none of the decoder's
arithmetic (no cut search, no LP, no interior-point or preconditioner step),
so both the CPU oracle and the CUDA path may draw their inputs from it.

Workloads follow the simulations of the paper (Sections III-D and VI-B):
random (3,6)-regular LDPC codes with 4-cycles removed, the all-zero codeword
sent over BPSK/AWGN, and LLR costs gamma_i = log P(r_i|0)/P(r_i|1) (Eq. 3),
which for BPSK over AWGN is 2*y_i/sigma^2.
"""

from .codes import (  # noqa: F401
    Code,
    gallager_regular,
    peg_code,
    peg_regular,
    irregular_degrees,
    hamming74,
    from_dense,
    random_codeword,
    named_code,
)
from .channel import (  # noqa: F401
    sigma2_for_ebn0,
    awgn_llr_frames,
)
