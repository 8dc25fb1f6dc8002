"""Oracle for the Q-less QR of tall, skinny matrices -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  The CUDA library never calls it and shares no code with it.

All routines take numpy arrays and return numpy arrays (float64, column-major inside).
The arithmetic lives in ``qless_oracle.c`` (FP64 storage, long-double accumulation);
this module only marshals arguments.  ``exact`` holds a second, exact-arithmetic
definition of R for tiny integer matrices.

Parity pins: every function here is checked by ``tests/test_oracle_pins.py`` against
closed forms, exact arithmetic, library routines and invariants.
"""
import ctypes

import numpy as np

from . import build as _build

_lib = None

_I64 = ctypes.c_int64
_DP = ctypes.POINTER(ctypes.c_double)


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        sig = {
            "qo_householder_r": [_I64, _I64, _DP, _I64, _DP, _I64],
            "qo_gram": [_I64, _I64, _DP, _I64, _DP, _I64],
            "qo_cholesky_upper": [_I64, _DP, _I64, _DP, _I64],
            "qo_cholqr2": [_I64, _I64, _DP, _I64, _DP, _I64, _DP],
            "qo_scholqr3": [_I64, _I64, _DP, _I64, _DP, _I64],
            "qo_q_from_r": [_I64, _I64, _DP, _I64, _DP, _I64, _DP, _I64],
            "qo_project_out": [_I64, _I64, _DP, _I64, _I64, _DP, _I64, _DP, _I64, _DP, _I64],
            "qo_jacobi_eig": [_I64, _DP, _I64, _DP, _DP, _I64],
            "qo_svqb2": [_I64, _I64, _DP, _I64, _DP, _I64, _DP],
            "qo_back_substitution": [_I64, _DP, _I64, _DP, _DP],
            "qo_lstsq": [_I64, _I64, _DP, _I64, _DP, _DP, _DP, _DP],
            "qo_singular_values": [_I64, _DP, _I64, _DP],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _f64(a):
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 1:
        a = a.reshape(-1, 1)
    return np.asfortranarray(a)


def _p(a):
    return a.ctypes.data_as(_DP)


class OracleError(RuntimeError):
    pass


def householder_r(X):
    """R of X = QR (Householder, long-double accumulation), nonnegative diagonal."""
    X = _f64(X)
    m, n = X.shape
    R = np.zeros((n, n), order="F")
    info = _load().qo_householder_r(m, n, _p(X), max(m, 1), _p(R), max(n, 1))
    if info:
        raise OracleError(f"qo_householder_r info={info}")
    return R


def gram(X):
    """C = X^T X (long-double accumulation, rounded once to double)."""
    X = _f64(X)
    m, n = X.shape
    C = np.zeros((n, n), order="F")
    _load().qo_gram(m, n, _p(X), max(m, 1), _p(C), max(n, 1))
    return C


def cholesky_upper(C):
    """(R, info): R^T R = C; info = j+1 on a non-positive j-th pivot (LAPACK style)."""
    C = _f64(C)
    n = C.shape[0]
    R = np.zeros((n, n), order="F")
    info = _load().qo_cholesky_upper(n, _p(C), max(n, 1), _p(R), max(n, 1))
    return R, info


def cholqr2(X):
    """(R, R1, info) of Algorithm 1; info: j+1 (first chol) or 1000+j+1 (second chol)."""
    X = _f64(X)
    m, n = X.shape
    R = np.zeros((n, n), order="F")
    R1 = np.zeros((n, n), order="F")
    info = _load().qo_cholqr2(m, n, _p(X), max(m, 1), _p(R), n, _p(R1))
    return R, R1, info


def scholqr3(X):
    """(R, info) of shifted Cholesky-QR3; info: j+1, 1000+j+1 or 2000+j+1 by failing pass."""
    X = _f64(X)
    m, n = X.shape
    R = np.zeros((n, n), order="F")
    info = _load().qo_scholqr3(m, n, _p(X), max(m, 1), _p(R), n)
    return R, info


def q_from_r(X, R):
    """(Q, info): Q = X R^{-1}; info j+1 when R(j, j) = 0."""
    X = _f64(X)
    R = _f64(R)
    m, n = X.shape
    Q = np.zeros((m, n), order="F")
    info = _load().qo_q_from_r(m, n, _p(X), max(m, 1), _p(R), n, _p(Q), max(m, 1))
    return Q, info


def project_out(Y, X):
    """(W, C): two projections of X against orthonormal Y, X = Y C + W."""
    Y = _f64(Y)
    X = _f64(X)
    m, k = Y.shape
    n = X.shape[1]
    W = np.zeros((m, n), order="F")
    C = np.zeros((k, n), order="F")
    info = _load().qo_project_out(m, k, _p(Y), max(m, 1), n, _p(X), max(m, 1), _p(W), max(m, 1), _p(C), k)
    if info:
        raise OracleError(f"qo_project_out info={info}")
    return W, C


def jacobi_eig(C):
    """(lambda ascending, U) with C = U diag(lambda) U^T (cyclic Jacobi)."""
    C = _f64(C)
    n = C.shape[0]
    lam = np.zeros(n)
    U = np.zeros((n, n), order="F")
    info = _load().qo_jacobi_eig(n, _p(C), n, _p(lam), _p(U), n)
    if info:
        raise OracleError(f"qo_jacobi_eig info={info}")
    return lam, U


def svqb2(X):
    """(R, Z) of SVQB applied twice: X = Q Z, R = qr_r(Z)."""
    X = _f64(X)
    m, n = X.shape
    R = np.zeros((n, n), order="F")
    Z = np.zeros((n, n), order="F")
    info = _load().qo_svqb2(m, n, _p(X), max(m, 1), _p(R), n, _p(Z))
    if info:
        raise OracleError(f"qo_svqb2 info={info}")
    return R, Z


def back_substitution(R, z):
    R = _f64(R)
    n = R.shape[0]
    z = np.ascontiguousarray(z, dtype=np.float64)
    x = np.zeros(n)
    info = _load().qo_back_substitution(n, _p(R), n, _p(z), _p(x))
    return x, info


def lstsq(A, b):
    """(x, resnorm, R_ext, info) of min ||A x - b|| via the Q-less QR of [A b]."""
    A = _f64(A)
    m, n = A.shape
    b = np.ascontiguousarray(np.asarray(b, dtype=np.float64).reshape(-1))
    x = np.zeros(n)
    rn = np.zeros(1)
    Re = np.zeros((n + 1, n + 1), order="F")
    info = _load().qo_lstsq(m, n, _p(A), max(m, 1), _p(b), _p(x), _p(rn), _p(Re))
    return x, float(rn[0]), Re, info


def singular_values(A):
    """Singular values (descending) of a square matrix, one-sided Jacobi."""
    A = _f64(A)
    n = A.shape[0]
    s = np.zeros(n)
    info = _load().qo_singular_values(n, _p(A), n, _p(s))
    if info:
        raise OracleError(f"qo_singular_values info={info}")
    return s


def kappa2(R):
    """kappa_2 of R (= kappa_2(X) when R is X's triangular factor); inf if singular."""
    s = singular_values(R)
    return float(s[0] / s[-1]) if s[-1] > 0 else float("inf")


def rel_err(R, R_ref):
    """||R - R_ref||_F / ||R_ref||_F -- the parity measure (Frobenius, the stated reading)."""
    R = np.asarray(R, dtype=np.float64)
    R_ref = np.asarray(R_ref, dtype=np.float64)
    den = np.linalg.norm(R_ref)
    return float(np.linalg.norm(R - R_ref) / (den if den > 0 else 1.0))


def row_err(R, R_ref):
    """max_ij |R_ij - R_ref_ij| / |R_ref_ii| over the upper triangle: the error of every
    entry relative to its row's diagonal (rows whose reference diagonal is zero are scaled
    by ||R_ref||_F).  A backward-stable R has |dR_ij| <= c u ||X|| <= c u kappa |R_ii|, so
    the parity bound applies row by row; a wrong small last row, invisible in the
    Frobenius ratio at large kappa, fails it."""
    R = np.asarray(R, dtype=np.float64)
    R_ref = np.asarray(R_ref, dtype=np.float64)
    fro = float(np.linalg.norm(R_ref)) or 1.0
    d = np.abs(np.diag(R_ref)).copy()
    d[d == 0] = fro
    D = np.triu(np.abs(R - R_ref)) / d[:, None]
    return float(D.max()) if D.size else 0.0


def tolerance(n, kappa):
    """Parity bound ||R - R_ref||_F / ||R_ref||_F <= 1e-13 * n * kappa(X)."""
    return 1e-13 * n * max(float(kappa), 1.0)
