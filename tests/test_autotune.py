"""The autotuner: its persisted table round-trips through ql_autotune_save / _load on the
host (no GPU), and on the GPU ql_autotune times the candidates (TSQR CTAs per SM, tile
height, R-tree arity; Cholesky-QR2 when kappa allows), records the fastest, and the calls
that then use the tuned configuration still match the oracle."""
import ctypes
import json
import os

import numpy as np
import pytest

import oracle
from paper_2603_20889_gb300 import synth


@pytest.fixture(scope="module")
def q():
    import paper_2603_20889_gb300 as q
    from paper_2603_20889_gb300 import build

    build.build()
    q.load_library()
    return q


def test_table_round_trips_through_json(q, tmp_path):
    L = q.load_library()
    src = tmp_path / "in.json"
    entries = [
        {"dtype": 0, "n": 24, "mlog2": 20, "kbucket": 0, "method": q.QL_CHOLQR2, "ctas": 0, "variant": 0, "arity": 0,
         "ms": 0.5},
        {"dtype": 0, "n": 12, "mlog2": 18, "kbucket": 0, "method": q.QL_TSQR, "ctas": 2, "variant": 1, "arity": 2,
         "ms": 0.25},
    ]
    src.write_text(json.dumps({"arch": "sm_103a", "entries": entries}, separators=(", ", ": ")))
    assert L.ql_autotune_load(str(src).encode()) == q.QL_OK
    assert L.ql_autotune_choose(1 << 20, 24, q.QL_F64, 1e3) == q.QL_CHOLQR2
    assert L.ql_autotune_choose((1 << 18) + 5, 12, q.QL_F64, 10.0) == q.QL_TSQR
    assert L.ql_autotune_choose(1 << 20, 24, q.QL_F64, 1e9) == q.QL_TSQR  # other kappa class: the model
    out = tmp_path / "out.json"
    assert L.ql_autotune_save(str(out).encode()) == q.QL_OK
    got = json.loads(out.read_text())["entries"]
    for e in entries:
        assert any(all(g[k] == e[k] for k in e if k != "ms") and abs(g["ms"] - e["ms"]) < 1e-9 for g in got), e
    # malformed entries are refused
    bad = tmp_path / "bad.json"
    bad.write_text('{"entries": [\n {"dtype": 0, "n": 5, "mlog2": 10, "kbucket": 0, "method": 7, "ctas": 1, '
                   '"variant": 9, "arity": 1, "ms": 1.0}\n]}')
    L.ql_autotune_load(str(bad).encode())
    assert L.ql_autotune_choose(1 << 10, 5, q.QL_F64, 1.0) == q.QL_TSQR


@pytest.mark.gpu
@pytest.mark.parametrize("m,n,kappa", [(1 << 20, 20, 1e3), (1 << 19, 3, 1e8), (1 << 18, 40, 1e2)])
def test_autotune_times_and_applies_its_choice(q, m, n, kappa):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L = q.load_library()
    wsb = L.ql_autotune_workspace_bytes(m, n, q.QL_F64)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    meth = ctypes.c_int32(-1)
    ms = ctypes.c_double(0.0)
    st = L.ql_autotune(m, n, q.QL_F64, kappa, ws.data_ptr(), wsb, q._stream_ptr(), ctypes.byref(meth),
                       ctypes.byref(ms))
    assert st == q.QL_OK
    assert meth.value in (q.QL_TSQR, q.QL_CHOLQR2) and ms.value > 0.0
    if kappa > 1e6:
        assert meth.value == q.QL_TSQR  # the Gram method is not accurate there
    assert L.ql_autotune_choose(m, n, q.QL_F64, kappa) == meth.value
    # the tuned configuration (CTAs per SM, tile layout, tree arity) is what ql_tsqr_qless runs now
    X = synth.conditioned(m, n, min(kappa, 1e4), seed=n)
    from gpu_util import to_dev, to_host

    R, info = q.tsqr_qless(to_dev(X))
    assert info.cpu().tolist() == [0, 0]
    R_ref = oracle.householder_r(X)
    assert oracle.rel_err(to_host(R), R_ref) <= oracle.tolerance(n, min(kappa, 1e4))
    assert oracle.row_err(to_host(R), R_ref) <= oracle.tolerance(n, min(kappa, 1e4))
