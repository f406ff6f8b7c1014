"""Python binding of the decoder's C ABI (include/lpdec.h).

Functions carry the C names and only marshal arguments: numpy arrays for
host pointers, torch CUDA tensors (or integer addresses) for device
pointers, a torch stream (or integer handle) for ``stream``. Every
computation runs in the CUDA kernels of liblpdec.so; importing this module
raises if the library is missing, and there is no fallback.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

LPDEC_OK = 0
LPDEC_ERR_INVALID_ARG = -1
LPDEC_ERR_OUT_OF_BUDGET = -2
LPDEC_ERR_NOT_CONVERGED = -3
LPDEC_ERR_TIMEOUT = -4
LPDEC_ERR_PENDING = -5
LPDEC_ERR_CUDA = -6
LPDEC_ERR_NO_DEVICE = -7
LPDEC_ERR_CANCELLED = -8
LPDEC_MALP_A = 0
LPDEC_MALP_B = 1
LPDEC_ALP = 2
LPDEC_MTS_COLUMN = 0
LPDEC_MTS_INCREMENTAL = 1
LPDEC_MTS_ROWWISE = 2
LPDEC_MTS_ADAPTIVE = 3
LPDEC_MTS_ROWWISE_TRI = 4
LPDEC_FP64 = 0
LPDEC_MIXED = 1
LPDEC_M32 = 2


class lpdec_params(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("sigma", "eta", "tol_gap", "tol_feas", "tol_pcg", "tau_act", "tau_cut", "tau_int",
                 "pcg_gap_factor", "tol_inner", "tol_feas_loose", "tol_cert", "tau_inc")] + \
               [(k, ctypes.c_int32) for k in
                ("max_alp", "max_ipm", "max_pcg", "variant", "precision",
                 "threads_per_block", "smem_budget", "lp_rows_cap", "precond",
                 "precond_switch", "warm_start", "mts_reuse", "lane_policy", "order_frames",
                 "dense_switch", "reserved")]


class lpdec_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int32) for k in
                ("status", "alp_iters", "ipm_iters_total", "pcg_iters_total", "lp_rows_final",
                 "vertex_failures", "max_levels", "pcg_iters_fp64", "dense_solves", "alp_switch",
                 "lp_rows_max", "ipm_iters_refine")] + \
               [(k, ctypes.c_double) for k in
                ("objective", "pcg_flops", "seconds", "pcg_bytes", "t_start", "t_end",
                  "sec_mts", "sec_pcg", "sec_dense", "sec_certify", "sec_refine")]


STATS_DTYPE = np.dtype([(k, np.int32) for k in
                        ("status", "alp_iters", "ipm_iters_total", "pcg_iters_total",
                         "lp_rows_final", "vertex_failures", "max_levels", "pcg_iters_fp64",
                         "dense_solves", "alp_switch", "lp_rows_max", "ipm_iters_refine")] +
                       [(k, np.float64) for k in
                        ("objective", "pcg_flops", "seconds", "pcg_bytes", "t_start", "t_end",
                  "sec_mts", "sec_pcg", "sec_dense", "sec_certify", "sec_refine")])
assert STATS_DTYPE.itemsize == ctypes.sizeof(lpdec_stats)


class LpdecError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {error_string(code)} ({code})")
        self.code = code


_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"decoder library not built ({path}); run "
                           "paper_0902_0657_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i32 = ctypes.c_int32
    lib.lpdec_default_params.argtypes = [ctypes.POINTER(lpdec_params)]
    lib.lpdec_default_params.restype = None
    lib.lpdec_error_string.argtypes = [i32]
    lib.lpdec_error_string.restype = ctypes.c_char_p
    lib.lpdec_workspace_bytes.argtypes = [i32, i32, i32, i32, i32, ctypes.POINTER(ctypes.c_size_t),
                                          ctypes.POINTER(ctypes.c_size_t)]
    lib.lpdec_workspace_bytes.restype = i32
    lib.lpdec_ctx_create.argtypes = [i32, ctypes.POINTER(lpdec_params), ctypes.c_size_t,
                                     ctypes.POINTER(P)]
    lib.lpdec_ctx_destroy.argtypes = [P]
    lib.lpdec_ctx_destroy.restype = None
    lib.lpdec_ctx_set_params.argtypes = [P, ctypes.POINTER(lpdec_params)]
    lib.lpdec_code_create.argtypes = [P, i32, i32, P, P, ctypes.POINTER(P)]
    lib.lpdec_code_destroy.argtypes = [P]
    lib.lpdec_code_destroy.restype = None
    lib.lpdec_decode.argtypes = [P, P, P, P, P, P, P, P]
    lib.lpdec_decode_frames.argtypes = [P, P, i32, P, P, P, P, P, P]
    lib.lpdec_decode_batch.argtypes = [P, i32, P, P, P, P, P, P, P]
    lib.lpdec_decode_mixed_device.argtypes = [P, i32, P, P, P, P, P, P, P, P]
    lib.lpdec_autotune.argtypes = [P, P, i32, P, ctypes.POINTER(i32), P]
    lib.lpdec_decode_batch_device.argtypes = [P, P, i32, P, P, P, P, P, P, P]
    lib.lpdec_batch_grid.argtypes = [P, P, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.lpdec_cut_search_device.argtypes = [P, P, i32, P, P, P, P, P, P]
    lib.lpdec_mts_select_device.argtypes = [P, P, i32, P, P, P, P, P, P, P]
    lib.lpdec_pcg_device.argtypes = [P, P, i32, P, P, P, P, P, P, P, P]
    lib.lpdec_lp_solve_device.argtypes = [P, P, i32, P, P, P, P, P, P]
    lib.lpdec_pcg_trace_device.argtypes = [P, P, i32, P, P, P, P, P, i32, ctypes.c_double, i32,
                                           P, P, P, P]
    lib.lpdec_lp_solve_trace_device.argtypes = [P, P, i32, P, P, P, P, P, P, i32, P]
    lib.lpdec_decode_batch_device_noalloc.argtypes = [P, ctypes.POINTER(lpdec_params), i32, P, P,
                                                      P, P, P, P, P]
    lib.lpdec_server_create.argtypes = [i32, ctypes.POINTER(lpdec_params), i32, P,
                                        ctypes.c_size_t, i32, ctypes.POINTER(P)]
    lib.lpdec_submit.argtypes = [P, P, P, ctypes.POINTER(ctypes.c_uint64)]
    lib.lpdec_poll.argtypes = [P, ctypes.c_uint64, P, P, P, P, P]
    lib.lpdec_cancel.argtypes = [P, ctypes.c_uint64]
    lib.lpdec_server_stats.argtypes = [P, ctypes.POINTER(ctypes.c_size_t),
                                       ctypes.POINTER(ctypes.c_size_t),
                                       ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(i32)]
    lib.lpdec_server_destroy.argtypes = [P]
    for name in ("lpdec_server_create", "lpdec_submit", "lpdec_poll", "lpdec_cancel",
                 "lpdec_server_stats", "lpdec_server_destroy"):
        getattr(lib, name).restype = i32
    for name in ("lpdec_ctx_create", "lpdec_ctx_set_params", "lpdec_code_create",
                 "lpdec_decode", "lpdec_decode_batch", "lpdec_decode_frames", "lpdec_autotune",
                 "lpdec_decode_mixed_device", "lpdec_decode_batch_device", "lpdec_batch_grid",
                 "lpdec_cut_search_device", "lpdec_mts_select_device", "lpdec_pcg_device",
                 "lpdec_pcg_trace_device",
                 "lpdec_lp_solve_device", "lpdec_lp_solve_trace_device",
                 "lpdec_decode_batch_device_noalloc"):
        getattr(lib, name).restype = i32
    _lib = lib
    return lib


def library():
    """The loaded ctypes library (loads it on first use)."""
    return _load()


def _check(rc: int, what: str):
    if rc != LPDEC_OK:
        raise LpdecError(rc, what)


def _hptr(a, dtype):
    """Host pointer of a C-contiguous numpy array of the given dtype."""
    if a is None:
        return None
    if not (isinstance(a, np.ndarray) and a.dtype == dtype and a.flags.c_contiguous):
        raise TypeError(f"expected a C-contiguous numpy array of {dtype}")
    return a.ctypes.data


def _dptr(t):
    """Device pointer: a torch CUDA tensor (contiguous) or an integer."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not (t.is_cuda and t.is_contiguous()):
        raise TypeError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


# ---------------------------------------------------------------------------
# C entry points
# ---------------------------------------------------------------------------

def lpdec_default_params() -> lpdec_params:
    p = lpdec_params()
    _load().lpdec_default_params(ctypes.byref(p))
    return p


def error_string(code: int) -> str:
    return _load().lpdec_error_string(code).decode()


lpdec_error_string = error_string


def lpdec_workspace_bytes(m: int, n: int, E: int, precision: int = LPDEC_FP64,
                          smem_budget: int = 0):
    """(rc, shared bytes per CTA, global scratch bytes per frame)."""
    sm = ctypes.c_size_t()
    gl = ctypes.c_size_t()
    rc = _load().lpdec_workspace_bytes(m, n, E, precision, smem_budget, ctypes.byref(sm),
                                       ctypes.byref(gl))
    return rc, sm.value, gl.value


def lpdec_ctx_create(device: int = 0, params: lpdec_params | None = None,
                     hbm_budget_bytes: int = 0) -> int:
    out = ctypes.c_void_p()
    rc = _load().lpdec_ctx_create(device, ctypes.byref(params) if params is not None else None,
                                  hbm_budget_bytes, ctypes.byref(out))
    _check(rc, "lpdec_ctx_create")
    return out.value


def lpdec_ctx_destroy(ctx: int) -> None:
    _load().lpdec_ctx_destroy(ctx)


def lpdec_ctx_set_params(ctx: int, params: lpdec_params) -> None:
    _check(_load().lpdec_ctx_set_params(ctx, ctypes.byref(params)), "lpdec_ctx_set_params")


def lpdec_code_create(ctx: int, m: int, n: int, row_ptr: np.ndarray, col_idx: np.ndarray) -> int:
    out = ctypes.c_void_p()
    rc = _load().lpdec_code_create(ctx, m, n, _hptr(row_ptr, np.int32), _hptr(col_idx, np.int32),
                                   ctypes.byref(out))
    _check(rc, "lpdec_code_create")
    return out.value


def lpdec_code_destroy(code: int) -> None:
    _load().lpdec_code_destroy(code)


def lpdec_decode(ctx, code, gamma, u_out, hard_out, cert_out, cut_mask_out=None, stats=None) -> int:
    return _load().lpdec_decode(ctx, code, _hptr(gamma, np.float64), _hptr(u_out, np.float64),
                                _hptr(hard_out, np.uint8), _hptr(cert_out, np.int32),
                                _hptr(cut_mask_out, np.uint32), _hptr(stats, STATS_DTYPE))


def lpdec_decode_frames(ctx, code, nframes, gamma, u_out, hard_out, cert_out,
                        cut_mask_out=None, stats=None) -> int:
    return _load().lpdec_decode_frames(ctx, code, nframes, _hptr(gamma, np.float64),
                                       _hptr(u_out, np.float64), _hptr(hard_out, np.uint8),
                                       _hptr(cert_out, np.int32), _hptr(cut_mask_out, np.uint32),
                                       _hptr(stats, STATS_DTYPE))


def _ptr_array(arrays, dtype):
    """C array of host pointers (NULL entries for None) of 1-D numpy arrays."""
    out = (ctypes.c_void_p * len(arrays))()
    for k, a in enumerate(arrays):
        out[k] = _hptr(a, dtype)
    return out


def lpdec_decode_batch(ctx, codes, gammas, u_out, hard_out, cert_out, cut_mask_out=None,
                       stats=None) -> int:
    """Per-frame codes (list of handles) and per-frame host arrays (lists of
    1-D numpy arrays); cert_out / stats one entry per frame."""
    nf = len(codes)
    ch = (ctypes.c_void_p * nf)(*codes)
    return _load().lpdec_decode_batch(
        ctx, nf, ch, _ptr_array(gammas, np.float64), _ptr_array(u_out, np.float64),
        _ptr_array(hard_out, np.uint8), _hptr(cert_out, np.int32),
        None if cut_mask_out is None else _ptr_array(cut_mask_out, np.uint32),
        _hptr(stats, STATS_DTYPE))


def lpdec_decode_mixed_device(ctx, codes, d_gamma, d_u, d_hard, d_cert, d_cut_mask=None,
                              d_stats=None, stream=None) -> int:
    nf = len(codes)
    ch = (ctypes.c_void_p * nf)(*codes)
    return _load().lpdec_decode_mixed_device(ctx, nf, ch, _dptr(d_gamma), _dptr(d_u),
                                             _dptr(d_hard), _dptr(d_cert), _dptr(d_cut_mask),
                                             _dptr(d_stats), _stream(stream))


def lpdec_autotune(ctx, code, gamma):
    """(status, chosen lane policy, per-candidate total device seconds for
    policies 0, 1, 2, 4, 8) on the host sample gamma [nframes x n]."""
    gamma = np.ascontiguousarray(gamma, dtype=np.float64)
    nf = gamma.shape[0]
    pol = ctypes.c_int32()
    secs = np.zeros(5, np.float64)
    rc = _load().lpdec_autotune(ctx, code, nf, gamma.ctypes.data, ctypes.byref(pol),
                                secs.ctypes.data)
    return rc, pol.value, secs


def lpdec_decode_batch_device(ctx, code, nframes, d_gamma, d_u, d_hard, d_cert,
                              d_cut_mask=None, d_stats=None, stream=None) -> int:
    return _load().lpdec_decode_batch_device(ctx, code, nframes, _dptr(d_gamma), _dptr(d_u),
                                             _dptr(d_hard), _dptr(d_cert), _dptr(d_cut_mask),
                                             _dptr(d_stats), _stream(stream))


def lpdec_batch_grid(ctx, code, nframes):
    """(rc, grid, ordered): CTAs of a one-code batch of nframes, and whether
    it is handed out hardest-first (two extra small kernels)."""
    grid, ordered = ctypes.c_int32(0), ctypes.c_int32(0)
    rc = _load().lpdec_batch_grid(ctx, code, nframes, ctypes.byref(grid), ctypes.byref(ordered))
    return rc, grid.value, ordered.value


def lpdec_cut_search_device(ctx, code, nframes, d_u, d_active, d_in_lp, d_mask, d_flag,
                            stream=None) -> int:
    return _load().lpdec_cut_search_device(ctx, code, nframes, _dptr(d_u), _dptr(d_active),
                                           _dptr(d_in_lp), _dptr(d_mask), _dptr(d_flag),
                                           _stream(stream))


def lpdec_mts_select_device(ctx, code, nframes, d_gamma, d_in_lp, d_mask, d_w, d_col, d_row,
                            stream=None) -> int:
    return _load().lpdec_mts_select_device(ctx, code, nframes, _dptr(d_gamma), _dptr(d_in_lp),
                                           _dptr(d_mask), _dptr(d_w), _dptr(d_col), _dptr(d_row),
                                           _stream(stream))


def lpdec_pcg_device(ctx, code, nframes, d_gamma, d_in_lp, d_mask, d_d2, d_w, d_dy, d_iters,
                     stream=None) -> int:
    return _load().lpdec_pcg_device(ctx, code, nframes, _dptr(d_gamma), _dptr(d_in_lp),
                                    _dptr(d_mask), _dptr(d_d2), _dptr(d_w), _dptr(d_dy),
                                    _dptr(d_iters), _stream(stream))


def lpdec_pcg_trace_device(ctx, code, nframes, d_gamma, d_in_lp, d_mask, d_d2, d_w, identity,
                           tol, max_hist, d_dy, d_iters, d_hist, stream=None) -> int:
    return _load().lpdec_pcg_trace_device(ctx, code, nframes, _dptr(d_gamma), _dptr(d_in_lp),
                                          _dptr(d_mask), _dptr(d_d2), _dptr(d_w), int(identity),
                                          float(tol), max_hist, _dptr(d_dy), _dptr(d_iters),
                                          _dptr(d_hist), _stream(stream))


def lanczos_condition(hist_row, iters):
    """Extreme eigenvalues (min, max) of the Lanczos tridiagonal that the CG
    coefficients (alpha_k, nu_k) of one traced run define (host-side
    post-processing of lpdec_pcg_trace_device's output)."""
    k = int(iters)
    if k < 1:
        return float("nan"), float("nan")
    a = np.asarray(hist_row).reshape(-1, 3)[:k, 1]
    nu = np.asarray(hist_row).reshape(-1, 3)[:k, 2]
    d = 1.0 / a
    d[1:] += nu[:-1] / a[:-1]
    e = np.sqrt(np.maximum(nu[:-1], 0.0)) / a[:-1]
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    ev = np.linalg.eigvalsh(T)
    return float(ev[0]), float(ev[-1])


def lpdec_lp_solve_device(ctx, code, nframes, d_gamma, d_in_lp, d_mask, d_x, d_stats,
                          stream=None) -> int:
    return _load().lpdec_lp_solve_device(ctx, code, nframes, _dptr(d_gamma), _dptr(d_in_lp),
                                         _dptr(d_mask), _dptr(d_x), _dptr(d_stats),
                                         _stream(stream))


def lpdec_lp_solve_trace_device(ctx, code, nframes, d_gamma, d_in_lp, d_mask, d_x, d_stats,
                                d_trace, max_trace, stream=None) -> int:
    return _load().lpdec_lp_solve_trace_device(ctx, code, nframes, _dptr(d_gamma), _dptr(d_in_lp),
                                               _dptr(d_mask), _dptr(d_x), _dptr(d_stats),
                                               _dptr(d_trace), max_trace, _stream(stream))


def lpdec_decode_batch_device_noalloc(code, params, nframes, d_gamma, d_u, d_hard, d_cert,
                                      d_cut_mask=None, d_stats=None, stream=None) -> int:
    """Batch decode without any device allocation (see include/lpdec.h)."""
    return _load().lpdec_decode_batch_device_noalloc(
        code, ctypes.byref(params) if params is not None else None, nframes, _dptr(d_gamma),
        _dptr(d_u), _dptr(d_hard), _dptr(d_cert), _dptr(d_cut_mask), _dptr(d_stats),
        _stream(stream))


# ---------------------------------------------------------------------------
# Convenience owner of a context + code (still only marshalling)
# ---------------------------------------------------------------------------

class Decoder:
    """Owns one context and one code; frees both on close()."""

    def __init__(self, code, device: int = 0, params: lpdec_params | None = None,
                 hbm_budget_bytes: int = 0):
        self.n, self.m = int(code.n), int(code.m)
        self.params = params if params is not None else lpdec_default_params()
        self.ctx = lpdec_ctx_create(device, self.params, hbm_budget_bytes)
        try:
            self.code = lpdec_code_create(self.ctx, self.m, self.n,
                                          np.ascontiguousarray(code.row_ptr, dtype=np.int32),
                                          np.ascontiguousarray(code.col_idx, dtype=np.int32))
        except Exception:
            lpdec_ctx_destroy(self.ctx)
            raise
        self.extra = []
        self.m_of = {self.code: self.m}

    def set_params(self, params: lpdec_params):
        self.params = params
        lpdec_ctx_set_params(self.ctx, params)

    def decode_batch(self, gamma: np.ndarray):
        """Host-pointer batch decode. Returns (u, hard, cert, masks, stats)."""
        gamma = np.ascontiguousarray(gamma, dtype=np.float64).reshape(-1, self.n)
        nf = gamma.shape[0]
        u = np.empty((nf, self.n), np.float64)
        hard = np.empty((nf, self.n), np.uint8)
        cert = np.empty(nf, np.int32)
        masks = np.empty((nf, self.m), np.uint32)
        stats = np.empty(nf, STATS_DTYPE)
        _check(lpdec_decode_frames(self.ctx, self.code, nf, gamma, u, hard, cert, masks, stats),
               "lpdec_decode_frames")
        return u, hard, cert, masks, stats

    def add_code(self, code) -> int:
        """Uploads another code on this context; returns its handle (freed by
        close())."""
        h = lpdec_code_create(self.ctx, int(code.m), int(code.n),
                              np.ascontiguousarray(code.row_ptr, dtype=np.int32),
                              np.ascontiguousarray(code.col_idx, dtype=np.int32))
        self.extra.append(h)
        self.m_of[h] = int(code.m)
        return h

    def decode_mixed(self, handles, gammas):
        """lpdec_decode_batch over frames of several codes: handles[f] and
        gammas[f] (1-D). Returns lists (u, hard, masks) and arrays (cert,
        stats)."""
        nf = len(handles)
        gammas = [np.ascontiguousarray(g, dtype=np.float64) for g in gammas]
        ms = [int(m) for m in self._code_m(handles)]
        u = [np.empty(g.size, np.float64) for g in gammas]
        hard = [np.empty(g.size, np.uint8) for g in gammas]
        masks = [np.empty(m, np.uint32) for m in ms]
        cert = np.empty(nf, np.int32)
        stats = np.empty(nf, STATS_DTYPE)
        _check(lpdec_decode_batch(self.ctx, list(handles), gammas, u, hard, cert, masks, stats),
               "lpdec_decode_batch")
        return u, hard, cert, masks, stats

    def _code_m(self, handles):
        return [self.m_of[h] for h in handles]

    def close(self):
        for h in getattr(self, "extra", []):
            lpdec_code_destroy(h)
        self.extra = []
        if self.code:
            lpdec_code_destroy(self.code)
            self.code = None
        if self.ctx:
            lpdec_ctx_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ---------------------------------------------------------------------------
# Serving (lpdec_server_create / lpdec_submit / lpdec_poll / lpdec_cancel)
# ---------------------------------------------------------------------------

def lpdec_server_create(device: int, params: lpdec_params | None, code_handles,
                        hbm_budget_bytes: int = 0, max_pending: int = 1 << 16):
    nc = len(code_handles)
    arr = (ctypes.c_void_p * nc)(*code_handles)
    out = ctypes.c_void_p()
    rc = _load().lpdec_server_create(device, ctypes.byref(params) if params is not None else None,
                                     nc, arr, hbm_budget_bytes, max_pending, ctypes.byref(out))
    _check(rc, "lpdec_server_create")
    return out.value


def lpdec_submit(server, code_handle, gamma) -> tuple[int, int]:
    """Returns (status, ticket)."""
    g = np.ascontiguousarray(gamma, dtype=np.float64)
    t = ctypes.c_uint64()
    rc = _load().lpdec_submit(server, code_handle, g.ctypes.data, ctypes.byref(t))
    return rc, t.value


def lpdec_poll(server, ticket: int, u_out=None, hard_out=None, cert_out=None, cut_mask_out=None,
               stats_out=None):
    return _load().lpdec_poll(server, ticket, _hptr(u_out, np.float64),
                              _hptr(hard_out, np.uint8), _hptr(cert_out, np.int32),
                              _hptr(cut_mask_out, np.uint32),
                              None if stats_out is None else stats_out.ctypes.data)


def lpdec_cancel(server, ticket: int) -> int:
    return _load().lpdec_cancel(server, ticket)


def lpdec_server_stats(server):
    """(status, device bytes held, arena size, arena bytes in use, outstanding
    tickets)."""
    hb, ab, used = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
    out = ctypes.c_int32()
    rc = _load().lpdec_server_stats(server, ctypes.byref(hb), ctypes.byref(ab), ctypes.byref(used),
                                    ctypes.byref(out))
    return rc, hb.value, ab.value, used.value, out.value


def region_bytes(n: int, m: int) -> int:
    """Arena bytes one frame of a code with n bits and m checks holds in a
    server (the layout lpdec_server_stats documents)."""
    up = lambda v, a: (v + a - 1) // a * a  # noqa: E731
    u = up(8 * n, 16)
    hard = up(u + 8 * n, 16)
    mask = up(hard + n, 16)
    cert = up(mask + 4 * m, 16)
    st = up(cert + 4, 16)
    return up(st + STATS_DTYPE.itemsize, 256)


def lpdec_server_destroy(server):
    return _load().lpdec_server_destroy(server)


class Server:
    """Submit frames of several codes as they arrive, poll their results (a
    thin wrapper of the C serving entry points; it owns a context holding
    the codes' device copies)."""

    def __init__(self, codes, device: int = 0, params: lpdec_params | None = None,
                 hbm_budget_bytes: int = 0, max_pending: int = 1 << 16):
        codes = list(codes) if isinstance(codes, (list, tuple)) else [codes]
        self.ctx = lpdec_ctx_create(device, params)
        self.handles, self.dims = [], {}
        try:
            for c in codes:
                h = lpdec_code_create(self.ctx, int(c.m), int(c.n),
                                      np.ascontiguousarray(c.row_ptr, dtype=np.int32),
                                      np.ascontiguousarray(c.col_idx, dtype=np.int32))
                self.handles.append(h)
                self.dims[h] = (int(c.n), int(c.m))
            self.handle = lpdec_server_create(device, params, self.handles, hbm_budget_bytes,
                                              max_pending)
        except Exception:
            self._free_codes()
            raise
        self.code_of_ticket = {}

    def _free_codes(self):
        for h in self.handles:
            lpdec_code_destroy(h)
        self.handles = []
        if self.ctx:
            lpdec_ctx_destroy(self.ctx)
            self.ctx = None

    def submit(self, gamma, code: int = 0) -> int:
        """Queues one frame of code index `code`; returns its ticket."""
        h = self.handles[code]
        rc, t = lpdec_submit(self.handle, h, gamma)
        _check(rc, "lpdec_submit")
        self.code_of_ticket[t] = h
        return t

    def try_submit(self, gamma, code: int = 0):
        """(status, ticket) without raising (admission may refuse)."""
        h = self.handles[code]
        rc, t = lpdec_submit(self.handle, h, gamma)
        if rc == LPDEC_OK:
            self.code_of_ticket[t] = h
        return rc, t

    def poll(self, ticket: int):
        """(u, hard, cert, cut mask, stats) once the frame is decoded, else None."""
        if ticket not in self.code_of_ticket:   # never issued, polled or cancelled here
            _check(lpdec_poll(self.handle, ticket), "lpdec_poll")
        n, m = self.dims[self.code_of_ticket[ticket]]
        u = np.empty(n, np.float64)
        h = np.empty(n, np.uint8)
        c = np.zeros(1, np.int32)
        mk = np.zeros(m, np.uint32)
        st = np.zeros(1, STATS_DTYPE)
        rc = lpdec_poll(self.handle, ticket, u, h, c, mk, st)
        if rc == LPDEC_ERR_PENDING:
            return None
        _check(rc, "lpdec_poll")
        self.code_of_ticket.pop(ticket, None)
        return u, h, int(c[0]), mk, st[0]

    def cancel(self, ticket: int):
        _check(lpdec_cancel(self.handle, ticket), "lpdec_cancel")
        self.code_of_ticket.pop(ticket, None)

    def stats(self):
        """(device bytes held, arena size, arena bytes in use, outstanding)."""
        rc, hb, ab, used, out = lpdec_server_stats(self.handle)
        _check(rc, "lpdec_server_stats")
        return hb, ab, used, out

    def close(self):
        if getattr(self, "handle", None):
            lpdec_server_destroy(self.handle)
            self.handle = None
        self._free_codes()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
