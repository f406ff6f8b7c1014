"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every function include/lpdec.h declares, sizes and validates workspaces,
rejects bad arguments, and reports the missing device instead of falling
back to the CPU."""

import ctypes
import os
import re

import numpy as np
import pytest

from paper_0902_0657_gb300 import build as B
from paper_0902_0657_gb300 import lpdec as L
from synth import named_code
from synth.codes import from_rows

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "lpdec.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.library()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lpdec_\w+)\s*\(", src)))


def test_all_declared_symbols_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_struct_sizes_match_header(lib):
    assert ctypes.sizeof(L.lpdec_params) == 13 * 8 + 16 * 4
    assert ctypes.sizeof(L.lpdec_stats) == 12 * 4 + 11 * 8
    assert L.STATS_DTYPE.itemsize == ctypes.sizeof(L.lpdec_stats)
    p = L.lpdec_default_params()
    assert (p.sigma, p.eta, p.tol_gap, p.tol_feas) == (0.1, 0.99, 1e-8, 1e-8)
    assert (p.tau_act, p.tau_cut, p.tau_int, p.tau_inc) == (1e-9, 1e-9, 1e-9, 1e-9)
    assert (p.max_alp, p.max_ipm, p.max_pcg, p.variant, p.precision) == (200, 60, 1000, 0, 0)
    assert p.lp_rows_cap == 0
    assert (p.order_frames, p.dense_switch, p.reserved) == (1, 64, 0)


@pytest.mark.parametrize("name", ["gallager_120", "peg_1008", "gallager_504", "gallager_4032",
                                  "gallager_16000", "gallager330_8000"])
@pytest.mark.parametrize("precision", [L.LPDEC_FP64, L.LPDEC_MIXED, L.LPDEC_M32])
@pytest.mark.parametrize("budget", [0, 4096, 20000, 60000, 100000])
def test_workspace_layouts_validate(lib, name, precision, budget):
    c = named_code(name)
    rc, smem, glob = L.lpdec_workspace_bytes(c.m, c.n, c.E, precision, budget)
    assert rc == 0 and smem > 0 and glob > 0
    if budget:
        # the always-shared arrays (bitmap, level pointers) may exceed a tiny budget
        must = 4 * ((c.n + c.m + 31) // 32) + 3 * 4 * (c.m + 2) + 2048
        assert smem <= max(budget, must) + 2048


def test_workspace_ragged_sizes(lib):
    rng = np.random.default_rng(0)
    for _ in range(30):
        m = int(rng.integers(1, 400))
        n = int(rng.integers(1, 900))
        E = int(rng.integers(m, min(32 * m, 6 * n) + m + 1))
        for prec in (0, 1, 2):
            rc, smem, glob = L.lpdec_workspace_bytes(m, n, E, prec, int(rng.integers(0, 80000)))
            assert rc == 0


def test_workspace_rejects_bad_sizes(lib):
    for m, n, E in [(0, 10, 10), (10, 0, 10), (40000, 10, 10), (10, 40000, 10), (2, 10, 100)]:
        assert L.lpdec_workspace_bytes(m, n, E, 0, 0)[0] == L.LPDEC_ERR_INVALID_ARG
    assert L.lpdec_workspace_bytes(10, 20, 30, 7, 0)[0] == L.LPDEC_ERR_INVALID_ARG
    # the FP32 M-solve vectors (3 x m floats) come on top of the FP64 layout
    c = named_code("peg_1008")
    s64 = L.lpdec_workspace_bytes(c.m, c.n, c.E, L.LPDEC_FP64, 0)[1]
    s32 = L.lpdec_workspace_bytes(c.m, c.n, c.E, L.LPDEC_M32, 0)[1]
    assert s32 - s64 == 12 * c.m   # three FP32 vectors over the main row capacity (m)


def test_no_device_is_reported_not_emulated(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(L.LpdecError) as e:
        L.lpdec_ctx_create(0)
    assert e.value.code == L.LPDEC_ERR_NO_DEVICE
    assert L.error_string(L.LPDEC_ERR_NOT_CONVERGED) == "iteration cap reached"
    assert L.error_string(L.LPDEC_ERR_CANCELLED) == "cancelled"


def test_null_handles_rejected(lib):
    rc = lib.lpdec_decode_batch(None, 1, None, None, None, None, None, None, None)
    assert rc == L.LPDEC_ERR_INVALID_ARG
    rc = lib.lpdec_decode_frames(None, None, 1, None, None, None, None, None, None)
    assert rc == L.LPDEC_ERR_INVALID_ARG
    rc = lib.lpdec_decode_mixed_device(None, 1, None, None, None, None, None, None, None, None)
    assert rc == L.LPDEC_ERR_INVALID_ARG
    rc = lib.lpdec_ctx_set_params(None, None)
    assert rc == L.LPDEC_ERR_INVALID_ARG
    assert lib.lpdec_batch_grid(None, None, 1, None, None) == L.LPDEC_ERR_INVALID_ARG


def test_server_reports_missing_device_and_null_handles(lib):
    import torch
    code = named_code("gallager_120")
    if not torch.cuda.is_available():
        with pytest.raises(L.LpdecError) as e:
            L.Server([code])
        assert e.value.code == L.LPDEC_ERR_NO_DEVICE
    assert lib.lpdec_submit(None, None, None, None) == L.LPDEC_ERR_INVALID_ARG
    assert lib.lpdec_poll(None, 0, None, None, None, None, None) == L.LPDEC_ERR_INVALID_ARG
    assert lib.lpdec_cancel(None, 0) == L.LPDEC_ERR_INVALID_ARG
    assert lib.lpdec_server_stats(None, None, None, None, None) == L.LPDEC_ERR_INVALID_ARG
    assert lib.lpdec_server_destroy(None) == L.LPDEC_ERR_INVALID_ARG
    out = ctypes.c_void_p()
    for ncodes, pending in ((0, 4), (1, 0), (1, 1 << 21)):
        rc = lib.lpdec_server_create(0, None, ncodes, None, 0, pending, ctypes.byref(out))
        assert rc == L.LPDEC_ERR_INVALID_ARG


def test_server_region_bytes():
    """The arena region of one frame: LLRs, u, hard, cut mask, cert and
    stats, 16-byte aligned parts, 256-byte multiple."""
    assert L.region_bytes(1008, 504) == 1024 * 19
    for n, m in ((120, 60), (1008, 504), (4032, 2016), (7, 3)):
        b = L.region_bytes(n, m)
        assert b % 256 == 0 and 17 * n + 4 * m + 4 + L.STATS_DTYPE.itemsize <= b
        assert b < 17 * n + 4 * m + 4 + L.STATS_DTYPE.itemsize + 64 + 256


def test_largest_decodable_sizes(lib):
    """The always-shared arrays (~12 B per LP row of the main workspace, m
    rows, plus 1 bit per column) bound the decodable size: a 16383 x 32767
    code fits one CTA's 227 KB of shared memory, a 32767 x 32767 one does
    not (its decode calls are rejected)."""
    cap = 227 * 1024
    assert L.lpdec_workspace_bytes(16383, 32767, 3 * 32767, 0, 0)[1] <= cap
    assert L.lpdec_workspace_bytes(32767, 32767, 3 * 32767, 0, 0)[1] > cap
    assert L.lpdec_workspace_bytes(1, 1, 1, 0, 0)[0] == 0          # smallest code
