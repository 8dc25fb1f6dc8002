"""qless: Q-less QR of tall, very skinny matrices on GB300 -- Python binding.

A thin ctypes layer over the C ABI in include/qless.h (libqless.so, built in-tree by
``build.py``).  It marshals arguments only: every step of every factorisation runs in the
library's CUDA kernels.  PyTorch provides device memory and the current stream.

Matrices are column-major: an m x n matrix is a torch tensor of shape (m, n) with
stride(0) == 1 (for example ``Xt.T`` for a contiguous (n, m) tensor ``Xt``); its leading
dimension is stride(1).

Raw entry points (same names and argument order as the C ABI) are available as
``lib.ql_tsqr_qless`` etc.; the functions below are conveniences that allocate outputs
and workspace with torch.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libqless.so")

QL_OK, QL_ERR_ARG, QL_ERR_ALIGN, QL_ERR_WORKSPACE, QL_ERR_CUDA = 0, 1, 2, 3, 4
QL_ERR_NOT_SPD, QL_ERR_TIMEOUT, QL_ERR_NONFINITE, QL_ERR_BUDGET, QL_ERR_BUSY, QL_ERR_UNKNOWN = 5, 6, 7, 8, 9, 10
QL_F64, QL_F32 = 0, 1
QL_TSQR, QL_CHOLQR2, QL_SVQB2, QL_AUTO, QL_SCHOLQR3 = 0, 1, 2, 3, 4
QL_ARITH_DF, QL_ARITH_F64 = 0, 1

STATUS_NAMES = {0: "QL_OK", 1: "QL_ERR_ARG", 2: "QL_ERR_ALIGN", 3: "QL_ERR_WORKSPACE", 4: "QL_ERR_CUDA",
                5: "QL_ERR_NOT_SPD", 6: "QL_ERR_TIMEOUT", 7: "QL_ERR_NONFINITE", 8: "QL_ERR_BUDGET",
                9: "QL_ERR_BUSY", 10: "QL_ERR_UNKNOWN"}

# Every symbol include/qless.h declares, with its ctypes signature.
_i64, _i32, _vp, _dp, _sz, _f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_double
SIGNATURES = {
    "ql_set_arith": (_i32, [_i32]),
    "ql_version": (ctypes.c_char_p, []),
    "ql_launch_count": (ctypes.c_uint64, []),
    "ql_measure_peaks": (_i32, [_vp, _vp]),
    "ql_check_bounded_wait": (_i32, [_i32, _i64, _vp, _vp]),
    "ql_workspace_bytes": (_sz, [_i32, _i64, _i64, _i32]),
    "ql_tsqr_qless": (_i32, [_i64, _i64, _vp, _i32, _i64, _dp, _i64, _vp, _vp, _sz, _vp]),
    "ql_tsqr_qless_noalloc": (_i32, [_i64, _i64, _vp, _i32, _i64, _dp, _i64, _vp, _vp]),
    "ql_cholqr2_qless": (_i32, [_i64, _i64, _vp, _i32, _i64, _dp, _i64, _vp, _vp, _sz, _vp]),
    "ql_scholqr3_qless": (_i32, [_i64, _i64, _vp, _i32, _i64, _dp, _i64, _vp, _vp, _sz, _vp]),
    "ql_q_from_r": (_i32, [_i64, _i64, _vp, _i32, _i64, _dp, _i64, _vp, _i64, _vp, _vp]),
    "ql_project_workspace_bytes": (_sz, [_i64, _i64]),
    "ql_qr_wide_workspace_bytes": (_sz, [_i64, _i64, _i32]),
    "ql_qr_wide": (_i32, [_i64, _i64, _vp, _i32, _i64, _dp, _i64, _vp, _i64, _vp, _vp, _sz, _vp]),
    "ql_project_out": (_i32, [_i64, _i64, _vp, _i64, _i64, _vp, _i64, _i32, _vp, _i64, _dp, _i64, _vp, _sz, _vp]),
    "ql_svqb_qless": (_i32, [_i64, _i64, _vp, _i32, _i64, _dp, _i64, _dp, _f64, _vp, _vp, _sz, _vp]),
    "ql_lstsq_qless": (_i32, [_i64, _i64, _vp, _i64, _vp, _i32, _i32, _dp, _dp, _dp, _vp, _vp, _sz, _vp]),
    "ql_batch_workspace_bytes": (_sz, [_i32, _vp]),
    "ql_batch_qless": (_i32, [_i32, _vp, _vp, _sz, _vp]),
    "ql_batch_prepare": (_i32, [_i32, _vp, _vp, _sz, _vp]),
    "ql_batch_launch": (_i32, [_vp, _vp]),
    "ql_batch_methods": (_i32, [_vp, _vp, _i32]),
    "ql_autotune_workspace_bytes": (_sz, [_i64, _i64, _i32]),
    "ql_autotune": (_i32, [_i64, _i64, _i32, _f64, _vp, _sz, _vp, _vp, _vp]),
    "ql_autotune_save": (_i32, [ctypes.c_char_p]),
    "ql_autotune_load": (_i32, [ctypes.c_char_p]),
    "ql_autotune_choose": (_i32, [_i64, _i64, _i32, _f64]),
    "ql_server_create": (_vp, [_sz, _i32, _i32]),
    "ql_server_submit": (_i32, [_vp, _vp, _vp]),
    "ql_server_poll": (_i32, [_vp, ctypes.c_uint64, _vp]),
    "ql_server_release": (_i32, [_vp, ctypes.c_uint64]),
    "ql_server_cancel": (_i32, [_vp, ctypes.c_uint64]),
    "ql_server_drain": (_i32, [_vp, _f64]),
    "ql_server_stats": (_i32, [_vp, _vp]),
    "ql_server_destroy": (None, [_vp]),
}


class Problem(ctypes.Structure):
    """ql_problem: one problem of a batch (device pointers)."""
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("ld", ctypes.c_int64), ("X", ctypes.c_void_p),
                ("dtype", ctypes.c_int32), ("kind", ctypes.c_int32), ("b", ctypes.c_void_p),
                ("R", ctypes.c_void_p), ("x", ctypes.c_void_p), ("info", ctypes.c_void_p),
                ("method_hint", ctypes.c_int32), ("kappa_hint", ctypes.c_double)]


class Request(ctypes.Structure):
    """ql_request: one serving request (device pointers)."""
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("ld", ctypes.c_int64), ("X", ctypes.c_void_p),
                ("dtype", ctypes.c_int32), ("kind", ctypes.c_int32), ("b", ctypes.c_void_p),
                ("kappa_hint", ctypes.c_double), ("method_hint", ctypes.c_int32)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("index", ctypes.c_int32), ("latency_ms", ctypes.c_double),
                ("R", ctypes.c_void_p), ("x", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("rejected", ctypes.c_int64),
                ("in_flight", ctypes.c_int64), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("mean_ms", ctypes.c_double), ("solves_per_s", ctypes.c_double),
                ("hbm_in_use_bytes", ctypes.c_double), ("hbm_peak_bytes", ctypes.c_double)]


class QlError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = int(status)
        super().__init__(f"{what}: {STATUS_NAMES.get(self.status, self.status)}")


_lib = None


def load_library(path: str | None = None):
    """Load libqless.so (raises if it was not built: there is no fallback path)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"qless CUDA library not built: {p} is missing (run build.py / __graft_entry__.build())")
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name, None)
        if f is None:
            continue
        f.restype = res
        f.argtypes = args
    if path is None:
        _lib = lib
    return lib


def __getattr__(name):
    if name == "lib":
        return load_library()
    raise AttributeError(name)


# ------------------------------------------------------------------ torch conveniences


def _torch():
    import torch

    return torch


def _stream_ptr(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _colmajor(X):
    """(m, n, ld, dtype code) of a column-major (m, n) tensor view."""
    torch = _torch()
    if X.dim() == 1:
        X = X.unsqueeze(1)
    m, n = X.shape
    if X.dtype == torch.float64:
        dt = QL_F64
    elif X.dtype == torch.float32:
        dt = QL_F32
    else:
        raise TypeError("X must be float64 or float32")
    if not X.is_cuda:
        raise TypeError("X must be a CUDA tensor")
    if n > 1 and X.stride(0) != 1:
        raise ValueError("X must be column-major: an (m, n) view with stride(0) == 1 (e.g. Xt.T)")
    ld = X.stride(1) if n > 1 else max(m, 1)
    return m, n, max(ld, max(m, 1)), dt


def measure_peaks(stream=None) -> dict:
    """Measured compute throughput of the current GPU in TFLOP/s (ql_measure_peaks)."""
    out = (ctypes.c_double * 5)()
    _check(load_library().ql_measure_peaks(ctypes.cast(out, ctypes.c_void_p), _stream_ptr(stream)),
           "ql_measure_peaks")
    return {"fp32_fma": out[0], "fp64_fma": out[1], "fp64_mma": out[2], "df_fma": out[3], "fp32x2_fma": out[4]}


def set_arith(mode: int) -> int:
    return load_library().ql_set_arith(mode)


def workspace(method: int, m: int, n: int, dtype: int, device=None):
    torch = _torch()
    nb = load_library().ql_workspace_bytes(method, m, n, dtype)
    if nb == 0:
        raise QlError(QL_ERR_ARG, "ql_workspace_bytes")
    return torch.empty(nb, dtype=torch.uint8, device=device or "cuda")


def _check(st, what):
    if st != QL_OK:
        raise QlError(st, what)


def tsqr_qless(X, R=None, info=None, ws=None, stream=None):
    """R (n x n, float64, column-major) of X by Q-less Householder TSQR.  Returns (R, info)."""
    torch = _torch()
    m, n, ld, dt = _colmajor(X)
    R = R if R is not None else torch.empty((n, n), dtype=torch.float64, device=X.device).T
    info = info if info is not None else torch.zeros(2, dtype=torch.int32, device=X.device)
    ws = ws if ws is not None else workspace(QL_TSQR, m, n, dt, X.device)
    st = load_library().ql_tsqr_qless(m, n, X.data_ptr(), dt, ld, R.data_ptr(), R.stride(1) if n > 1 else n,
                                      info.data_ptr(), ws.data_ptr(), ws.numel(), _stream_ptr(stream))
    _check(st, "ql_tsqr_qless")
    return R, info


def cholqr2_qless(X, R=None, info=None, ws=None, stream=None):
    """R of X by Q-less Cholesky-QR2 (Algorithm 1).  Returns (R, info)."""
    torch = _torch()
    m, n, ld, dt = _colmajor(X)
    R = R if R is not None else torch.empty((n, n), dtype=torch.float64, device=X.device).T
    info = info if info is not None else torch.zeros(2, dtype=torch.int32, device=X.device)
    ws = ws if ws is not None else workspace(QL_CHOLQR2, m, n, dt, X.device)
    st = load_library().ql_cholqr2_qless(m, n, X.data_ptr(), dt, ld, R.data_ptr(), R.stride(1) if n > 1 else n,
                                         info.data_ptr(), ws.data_ptr(), ws.numel(), _stream_ptr(stream))
    _check(st, "ql_cholqr2_qless")
    return R, info


def scholqr3_qless(X, R=None, info=None, ws=None, stream=None):
    """R of X by Q-less shifted Cholesky-QR3 (three Gram passes).  Returns (R, info)."""
    torch = _torch()
    m, n, ld, dt = _colmajor(X)
    R = R if R is not None else torch.empty((n, n), dtype=torch.float64, device=X.device).T
    info = info if info is not None else torch.zeros(2, dtype=torch.int32, device=X.device)
    ws = ws if ws is not None else workspace(QL_SCHOLQR3, m, n, dt, X.device)
    st = load_library().ql_scholqr3_qless(m, n, X.data_ptr(), dt, ld, R.data_ptr(), R.stride(1) if n > 1 else n,
                                          info.data_ptr(), ws.data_ptr(), ws.numel(), _stream_ptr(stream))
    _check(st, "ql_scholqr3_qless")
    return R, info


def q_from_r(X, R, Q=None, info=None, stream=None):
    """Q = X R^{-1} in X's dtype (column-major like X).  Returns (Q, info)."""
    torch = _torch()
    m, n, ld, dt = _colmajor(X)
    if R.dtype != torch.float64 or R.shape != (n, n) or (n > 1 and R.stride(0) != 1):
        raise ValueError("R must be a column-major n x n float64 tensor")
    Q = Q if Q is not None else torch.empty((n, m), dtype=X.dtype, device=X.device).T
    info = info if info is not None else torch.zeros(2, dtype=torch.int32, device=X.device)
    ldq = Q.stride(1) if n > 1 else max(m, 1)
    st = load_library().ql_q_from_r(m, n, X.data_ptr(), dt, ld, R.data_ptr(), R.stride(1) if n > 1 else n,
                                    Q.data_ptr(), ldq, info.data_ptr(), _stream_ptr(stream))
    _check(st, "ql_q_from_r")
    return Q, info


def project_out(Y, X, W=None, C=None, ws=None, stream=None):
    """Two-phase orthogonalisation against orthonormal Y: W = (I - Y Y^T) X (projected twice),
    C = Y^T X accumulated over both passes (X = Y C + W).  Returns (W, C)."""
    torch = _torch()
    m, k, ldy, dty = _colmajor(Y)
    m2, n, ldx, dt = _colmajor(X)
    if m2 != m or dty != dt:
        raise ValueError("Y and X need the same rows and dtype")
    W = W if W is not None else torch.empty((n, m), dtype=X.dtype, device=X.device).T
    C = C if C is not None else torch.empty((n, k), dtype=torch.float64, device=X.device).T
    lib = load_library()
    if ws is None:
        nb = lib.ql_project_workspace_bytes(k, n)
        if nb == 0:
            raise QlError(QL_ERR_ARG, "ql_project_workspace_bytes")
        ws = torch.empty(nb, dtype=torch.uint8, device=X.device)
    ldw = W.stride(1) if n > 1 else max(m, 1)
    st = lib.ql_project_out(m, k, Y.data_ptr(), ldy, n, X.data_ptr(), ldx, dt, W.data_ptr(), ldw, C.data_ptr(),
                            C.stride(1) if n > 1 else k, ws.data_ptr(), ws.numel(), _stream_ptr(stream))
    _check(st, "ql_project_out")
    return W, C


def qr_wide(X, R=None, Q=None, info=None, ws=None, stream=None):
    """QR of an m x n matrix with any n (64-column panels): returns (Q, R, info)."""
    torch = _torch()
    m, n, ld, dt = _colmajor(X)
    R = R if R is not None else torch.empty((n, n), dtype=torch.float64, device=X.device).T
    Q = Q if Q is not None else torch.empty((n, m), dtype=X.dtype, device=X.device).T
    info = info if info is not None else torch.zeros(2, dtype=torch.int32, device=X.device)
    lib = load_library()
    if ws is None:
        nb = lib.ql_qr_wide_workspace_bytes(m, n, dt)
        if nb == 0:
            raise QlError(QL_ERR_ARG, "ql_qr_wide_workspace_bytes")
        ws = torch.empty(nb, dtype=torch.uint8, device=X.device)
    st = lib.ql_qr_wide(m, n, X.data_ptr(), dt, ld, R.data_ptr(), R.stride(1) if n > 1 else n, Q.data_ptr(),
                        Q.stride(1) if n > 1 else max(m, 1), info.data_ptr(), ws.data_ptr(), ws.numel(),
                        _stream_ptr(stream))
    _check(st, "ql_qr_wide")
    return Q, R, info


def svqb_qless(X, R=None, Z=None, rank_tol=0.0, info=None, ws=None, stream=None, want_z=False):
    """R (and optionally Z of X = Q Z) by Q-less SVQB2.  Returns (R, Z or None, info)."""
    torch = _torch()
    m, n, ld, dt = _colmajor(X)
    R = R if R is not None else torch.empty((n, n), dtype=torch.float64, device=X.device).T
    if want_z and Z is None:
        Z = torch.empty((n, n), dtype=torch.float64, device=X.device).T
    info = info if info is not None else torch.zeros(2, dtype=torch.int32, device=X.device)
    ws = ws if ws is not None else workspace(QL_SVQB2, m, n, dt, X.device)
    st = load_library().ql_svqb_qless(m, n, X.data_ptr(), dt, ld, R.data_ptr(), R.stride(1) if n > 1 else n,
                                      Z.data_ptr() if Z is not None else None, float(rank_tol), info.data_ptr(),
                                      ws.data_ptr(), ws.numel(), _stream_ptr(stream))
    _check(st, "ql_svqb_qless")
    return R, Z, info


def lstsq_qless(A, b, method=QL_TSQR, want_rext=False, info=None, ws=None, stream=None):
    """min ||A x - b|| via the Q-less QR of [A b].  Returns (x, resnorm, R_ext or None, info)."""
    torch = _torch()
    m, n, ld, dt = _colmajor(A)
    if b.dtype != A.dtype or b.numel() != m or (b.dim() == 2 and b.stride(0) != 1):
        raise ValueError("b must have m contiguous entries of A's dtype")
    x = torch.empty(n, dtype=torch.float64, device=A.device)
    rn = torch.empty(1, dtype=torch.float64, device=A.device)
    Rext = torch.empty((n + 1, n + 1), dtype=torch.float64, device=A.device).T if want_rext else None
    info = info if info is not None else torch.zeros(2, dtype=torch.int32, device=A.device)
    ws = ws if ws is not None else workspace(QL_AUTO, m, n, dt, A.device)
    st = load_library().ql_lstsq_qless(m, n, A.data_ptr(), ld, b.data_ptr(), dt, method, x.data_ptr(),
                                       rn.data_ptr(), Rext.data_ptr() if Rext is not None else None,
                                       info.data_ptr(), ws.data_ptr(), ws.numel(), _stream_ptr(stream))
    _check(st, "ql_lstsq_qless")
    return x, rn, Rext, info


def batch_qless(problems, ws=None, stream=None, device=None):
    """Run a list of Problem structs in one batched launch; returns the workspace used."""
    torch = _torch()
    arr = (Problem * len(problems))(*problems)
    lib = load_library()
    nb = lib.ql_batch_workspace_bytes(len(problems), arr)
    if nb == 0:
        raise QlError(QL_ERR_ARG, "ql_batch_workspace_bytes")
    if ws is None or ws.numel() < nb:
        ws = torch.empty(nb, dtype=torch.uint8, device=device or "cuda")
    _check(lib.ql_batch_qless(len(problems), arr, ws.data_ptr(), ws.numel(), _stream_ptr(stream)), "ql_batch_qless")
    return ws


class Server:
    """Thin owner of a ql_server handle."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 4096, streams: int = 4):
        self.lib = load_library()
        self.h = self.lib.ql_server_create(hbm_budget_bytes, max_slots, streams)
        if not self.h:
            raise QlError(QL_ERR_CUDA, "ql_server_create")

    def submit(self, req: Request) -> int:
        t = ctypes.c_uint64(0)
        _check(self.lib.ql_server_submit(self.h, ctypes.byref(req), ctypes.byref(t)), "ql_server_submit")
        return t.value

    def poll(self, ticket: int):
        r = Result()
        st = self.lib.ql_server_poll(self.h, ticket, ctypes.byref(r))
        return st, r

    def release(self, ticket: int):
        return self.lib.ql_server_release(self.h, ticket)

    def drain(self, timeout_s: float = 60.0):
        return self.lib.ql_server_drain(self.h, timeout_s)

    def stats(self) -> Stats:
        st = Stats()
        _check(self.lib.ql_server_stats(self.h, ctypes.byref(st)), "ql_server_stats")
        return st

    def close(self):
        if self.h:
            self.lib.ql_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
