"""Helpers shared by the GPU tests: device buffers through torch, the
decoder handle, and LP states taken from oracle runs."""

from __future__ import annotations

import functools

import numpy as np

import oracle
from oracle import lp as olp
from synth import awgn_llr_frames, named_code


def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        import pytest
        pytest.skip("no CUDA device")
    return torch


def dev(a):
    torch = torch_cuda()
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.cpu().numpy()


@functools.lru_cache(maxsize=None)
def oracle_history(code_name: str, ebn0: float, seed: int, nframes: int):
    """(gamma, list of LP records) of oracle decodes, for step-level tests."""
    code = named_code(code_name)
    G = awgn_llr_frames(code.n, code.design_rate, ebn0, seed, range(nframes))
    out = []
    for g in G:
        res = oracle.decode(code, g)
        for h in res.history:
            out.append((g, h))
    return code, out


def lp_state_arrays(code, records):
    """Stack (gamma, in_lp, mask) of LP records into frame-major arrays."""
    g = np.stack([r[0] for r in records]).astype(np.float64)
    in_lp = np.stack([r[1].in_lp.astype(np.uint8) for r in records])
    mask = np.stack([np.where(r[1].in_lp, r[1].masks, 0).astype(np.uint32) for r in records])
    lps = [olp.build(code, r[0], r[1].in_lp, r[1].masks) for r in records]
    return g, in_lp, mask, lps
