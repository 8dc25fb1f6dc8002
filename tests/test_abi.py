"""The C ABI boundary without a GPU: the library loads, exports every function that
include/qless.h declares, and the Python ctypes mirrors of the header's structs have the
C layout (checked against gcc's sizeof/offsetof of the real header)."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qless.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(ql_\w+)\s*\(", text))
    return sorted(n for n in names if not n.endswith("_t"))


@pytest.fixture(scope="module")
def lib():
    from paper_2603_20889_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ql_tsqr_qless", "ql_cholqr2_qless", "ql_svqb_qless", "ql_lstsq_qless", "ql_batch_qless",
                     "ql_server_create", "ql_server_submit", "ql_server_poll", "ql_server_stats",
                     "ql_server_destroy", "ql_workspace_bytes"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_python_binding_covers_every_symbol():
    import paper_2603_20889_gb300 as q

    assert set(declared_functions()) <= set(q.SIGNATURES)


def test_host_only_calls(lib):
    """Calls that touch no device: argument validation and the version string."""
    import paper_2603_20889_gb300 as q

    L = q.load_library()
    assert L.ql_version().startswith(b"qless")
    assert L.ql_workspace_bytes(q.QL_TSQR, 1000, 0, q.QL_F64) == 0  # n < 1
    assert L.ql_workspace_bytes(q.QL_TSQR, 1000, 65, q.QL_F64) == 0  # n > 64
    # argument errors are reported before any device work
    assert L.ql_tsqr_qless(10, 0, None, q.QL_F64, 10, None, 1, None, None, 0, None) == q.QL_ERR_ARG
    assert L.ql_tsqr_qless(10, 3, None, q.QL_F64, 10, None, 3, None, None, 0, None) == q.QL_ERR_ARG
    assert L.ql_tsqr_qless(10, 3, ctypes.c_void_p(8), q.QL_F64, 5, None, 3, None, None, 0, None) == q.QL_ERR_ARG
    assert L.ql_tsqr_qless(10, 3, ctypes.c_void_p(12), q.QL_F64, 10, ctypes.c_void_p(16), 3, None, None, 0,
                           None) == q.QL_ERR_ALIGN
    assert L.ql_lstsq_qless(10, 64, ctypes.c_void_p(16), 10, ctypes.c_void_p(16), q.QL_F64, q.QL_TSQR,
                            ctypes.c_void_p(16), ctypes.c_void_p(16), None, None, None, 0, None) == q.QL_ERR_ARG
    # the workspace-free TSQR makes the same checks before any device work
    V = ctypes.c_void_p
    assert L.ql_tsqr_qless_noalloc(10, 3, V(12), q.QL_F64, 10, V(16), 3, None, None) == q.QL_ERR_ALIGN
    assert L.ql_tsqr_qless_noalloc(10, 3, V(16), q.QL_F64, 10, V(20), 3, None, None) == q.QL_ERR_ALIGN
    assert L.ql_tsqr_qless_noalloc(10, 3, V(18), q.QL_F32, 10, V(16), 3, None, None) == q.QL_ERR_ALIGN
    assert L.ql_tsqr_qless_noalloc(10, 3, V(16), q.QL_F64, 5, V(16), 3, None, None) == q.QL_ERR_ARG
    assert L.ql_tsqr_qless_noalloc(10, 3, V(16), q.QL_F64, 10, None, 3, None, None) == q.QL_ERR_ARG
    assert L.ql_tsqr_qless_noalloc(10, 65, V(16), q.QL_F64, 10, V(16), 65, None, None) == q.QL_ERR_ARG
    # the Gram methods check R's alignment as well
    assert L.ql_cholqr2_qless(10, 3, V(16), q.QL_F64, 10, V(20), 3, None, None, 0, None) == q.QL_ERR_ALIGN
    assert L.ql_server_create(0, 1, 1) is None
    assert L.ql_autotune_choose(1 << 20, 8, q.QL_F64, 1e9) == q.QL_TSQR


def test_struct_layouts_match_the_header():
    import paper_2603_20889_gb300 as q

    src = r"""
#include <stdio.h>
#include <stddef.h>
#include "qless.h"
#define O(T, f) printf(#T "." #f " %zu\n", offsetof(T, f))
int main(void) {
  printf("ql_problem %zu\nql_request %zu\nql_result %zu\nql_stats %zu\n", sizeof(ql_problem),
         sizeof(ql_request), sizeof(ql_result), sizeof(ql_stats));
  O(ql_problem, X); O(ql_problem, dtype); O(ql_problem, b); O(ql_problem, info);
  O(ql_problem, method_hint); O(ql_problem, kappa_hint); O(ql_request, method_hint);
  O(ql_request, kappa_hint); O(ql_result, R); O(ql_stats, hbm_peak_bytes);
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    got = dict(line.rsplit(" ", 1) for line in out.strip().splitlines())
    got = {k: int(v) for k, v in got.items()}
    assert got["ql_problem"] == ctypes.sizeof(q.Problem)
    assert got["ql_request"] == ctypes.sizeof(q.Request)
    assert got["ql_result"] == ctypes.sizeof(q.Result)
    assert got["ql_stats"] == ctypes.sizeof(q.Stats)
    assert got["ql_problem.X"] == q.Problem.X.offset
    assert got["ql_problem.dtype"] == q.Problem.dtype.offset
    assert got["ql_problem.b"] == q.Problem.b.offset
    assert got["ql_problem.info"] == q.Problem.info.offset
    assert got["ql_problem.method_hint"] == q.Problem.method_hint.offset
    assert got["ql_problem.kappa_hint"] == q.Problem.kappa_hint.offset
    assert got["ql_request.method_hint"] == q.Request.method_hint.offset
    assert got["ql_request.kappa_hint"] == q.Request.kappa_hint.offset
    assert got["ql_result.R"] == q.Result.R.offset
    assert got["ql_stats.hbm_peak_bytes"] == q.Stats.hbm_peak_bytes.offset
