"""The workspace-free TSQR entry point, for callers that cannot allocate device memory
(inside CUDA-graph capture, in host callbacks, or in framework plugins whose host owns
every allocation).  It must give the same R as the regular entry point, and the oracle's R
within the parity tolerance, call after call, although every call reuses the same
library-owned scratch array.

Collected last on purpose (file name), so a stop-at-first-failure run has already run
every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2603_20889_gb300 import synth

from gpu_util import info_of, to_dev, to_host

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_20889_gb300 as q

    q.load_library()
    q.set_arith(q.QL_ARITH_DF)
    return q


def _noalloc(q, Xd, n):
    R = torch.empty((n, n), dtype=torch.float64, device="cuda")
    info = torch.full((2,), -1, dtype=torch.int32, device="cuda")
    m = Xd.shape[0]
    dt = q.QL_F64 if Xd.dtype == torch.float64 else q.QL_F32
    ld = Xd.stride(1) if n > 1 else m
    st = q.load_library().ql_tsqr_qless_noalloc(m, n, Xd.data_ptr(), dt, ld, R.data_ptr(), n, info.data_ptr(),
                                                q._stream_ptr())
    assert st == q.QL_OK
    Rh = to_host(R)
    return Rh.reshape(-1).reshape(Rh.shape, order="F"), info_of(info)


@pytest.mark.parametrize("m,n,kappa,dtype", [(300007, 16, 1e4, np.float64), (65537, 8, 1e2, np.float32),
                                             (1000, 3, 1.0, np.float64)])
def test_noalloc_matches_regular_entry_twice(q, m, n, kappa, dtype):
    X = synth.conditioned(m, n, kappa, seed=m + n).astype(dtype)
    Xd = to_dev(X)
    R_ref, info_ref = q.tsqr_qless(Xd)
    R_ref = to_host(R_ref)
    assert info_of(info_ref) == [0, 0]
    R_or = oracle.householder_r(X.astype(np.float64))  # the stored (possibly float-rounded) X
    tol = oracle.tolerance(n, kappa)
    for _ in range(2):  # the shared scratch keeps the previous call's contents
        R, info = _noalloc(q, Xd, n)
        assert info == [0, 0]
        assert oracle.rel_err(R, R_ref) <= tol
        assert oracle.rel_err(R, R_or) <= tol


def test_noalloc_rejects_columns_beyond_its_scratch(q):
    X = torch.zeros((17, 64), dtype=torch.float64, device="cuda").T
    R = torch.empty((17, 17), dtype=torch.float64, device="cuda")
    st = q.load_library().ql_tsqr_qless_noalloc(64, 17, X.data_ptr(), q.QL_F64, 64, R.data_ptr(), 17, None,
                                                q._stream_ptr())
    assert st == q.QL_ERR_WORKSPACE
