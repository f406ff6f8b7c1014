"""Seeded BPSK/AWGN channel LLRs (input generation only).

The all-zero codeword is sent (the paper's simulations assume it without
loss of generality, Section III-C). BPSK maps bit 0 to +1, so the channel
output is y_i = 1 + sigma * n_i with n_i standard normal, and the LLR cost of
Eq. 3, gamma_i = log P(y_i|0)/P(y_i|1), equals 2*y_i/sigma^2.

The paper quotes an SNR without defining it; the workloads read it as Eb/N0
in dB with the design rate R = 1 - m/n:  sigma^2 = 1 / (2 R 10^(EbN0/10)).

Each frame draws its noise from its own stream, numpy's PCG64 seeded with
the tuple (seed, frame index), so any subset of frames can be regenerated
independently and identically for the oracle and the GPU.
"""

from __future__ import annotations

import numpy as np


def sigma2_for_ebn0(ebn0_db: float, rate: float) -> float:
    return 1.0 / (2.0 * rate * 10.0 ** (ebn0_db / 10.0))


def awgn_llr_frames(n: int, rate: float, ebn0_db, seed: int, frames,
                    codeword=None) -> np.ndarray:
    """LLR vectors gamma (float64, shape [len(frames), n]).

    ``ebn0_db`` is a scalar or one value per frame. ``frames`` is an iterable
    of frame indices. ``codeword`` (optional, uint8 [n]) replaces the all-zero
    codeword; bit 1 is sent as -1.
    """
    frames = np.asarray(list(frames), dtype=np.int64)
    eb = np.broadcast_to(np.asarray(ebn0_db, dtype=np.float64), frames.shape)
    out = np.empty((frames.size, n), dtype=np.float64)
    sym = np.ones(n) if codeword is None else 1.0 - 2.0 * np.asarray(codeword, dtype=np.float64)
    for t, (f, e) in enumerate(zip(frames, eb)):
        s2 = sigma2_for_ebn0(float(e), rate)
        rng = np.random.default_rng([int(seed), int(f)])
        y = sym + np.sqrt(s2) * rng.standard_normal(n)
        out[t] = 2.0 * y / s2
    return out
