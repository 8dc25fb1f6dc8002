"""GPU tests of the batched form (one persistent launch over uneven problems, CUDA-graph
replay) and of the continuous-batching server (alone vs in the mix, budget, stats)."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2603_20889_gb300 import synth

from gpu_util import info_of, to_dev, to_host

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_20889_gb300 as q

    q.load_library()
    q.set_arith(q.QL_ARITH_DF)


def _instances(count, seed, m_lo=16, m_hi=1 << 16, n_lo=1, n_hi=64, lstsq_every=5, f32_every=4):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        m = int(np.exp(rng.uniform(np.log(m_lo), np.log(m_hi))))
        kind = 1 if k % lstsq_every == 3 else 0
        n = int(rng.integers(n_lo, (n_hi if kind == 0 else n_hi - 1) + 1))
        m = max(m, n + 2)
        kappa = float(np.exp(rng.uniform(0, np.log(1e5))))
        dt = np.float32 if k % f32_every == 1 else np.float64
        X = synth.conditioned(m, n, kappa, seed=seed * 1000 + k).astype(dt)
        b = (synth.gaussian(m, 1, seed=seed * 1000 + k + 7)[:, 0]).astype(dt) if kind else None
        out.append(dict(m=m, n=n, kind=kind, kappa=kappa, X=X, b=b, dt=dt))
    return out


def _expected(inst):
    X = inst["X"].astype(np.float64)
    if inst["kind"] == 0:
        return oracle.householder_r(X)
    x, rho, Re, _ = oracle.lstsq(X, inst["b"].astype(np.float64))
    return Re


def _problems(insts, q):
    probs, keep = [], []
    for it in insts:
        Xd = to_dev(it["X"])
        n1 = it["n"] + (1 if it["kind"] else 0)
        R = torch.full((n1, n1), float("nan"), dtype=torch.float64, device="cuda")
        x = torch.zeros(it["n"] + 1, dtype=torch.float64, device="cuda")
        info = torch.full((2,), -1, dtype=torch.int32, device="cuda")
        bd = torch.from_numpy(it["b"]).cuda() if it["kind"] else None
        p = q.Problem(m=it["m"], n=it["n"], ld=Xd.stride(1) if it["n"] > 1 else it["m"], X=Xd.data_ptr(),
                      dtype=q.QL_F64 if it["dt"] == np.float64 else q.QL_F32, kind=it["kind"],
                      b=bd.data_ptr() if bd is not None else None, R=R.data_ptr(), x=x.data_ptr(),
                      info=info.data_ptr())
        probs.append(p)
        keep.append((Xd, bd, R, x, info))
    return probs, keep


def _check_outputs(insts, keep, tol_scale=1.0):
    for it, (_, _, R, x, info) in zip(insts, keep):
        assert info_of(info) == [0, 0], it["m"]
        Rh = to_host(R)  # row-major (n1, n1) tensor holding a column-major matrix: transpose
        Rh = Rh.reshape(-1).reshape(Rh.shape, order="F")
        ref = _expected(it)
        n1 = ref.shape[0]
        kappa = it["kappa"] if it["dt"] == np.float64 else it["kappa"]
        assert oracle.rel_err(Rh, ref) <= tol_scale * oracle.tolerance(n1, max(kappa, 10.0)), (it["m"], it["n"])


def test_batch_uneven_problems_one_launch():
    import paper_2603_20889_gb300 as q

    insts = _instances(40, seed=1)
    probs, keep = _problems(insts, q)
    l0 = q.load_library().ql_launch_count()
    q.batch_qless(probs)
    torch.cuda.synchronize()
    assert q.load_library().ql_launch_count() - l0 == 2  # the persistent launch + gated FP64 one
    _check_outputs(insts, keep)


def test_batch_lstsq_solution_matches_oracle():
    import paper_2603_20889_gb300 as q

    A, b, _ = synth.lstsq_case(30011, 20, 1e3, seed=5)
    it = dict(m=30011, n=20, kind=1, kappa=1e3, X=A, b=b, dt=np.float64)
    probs, keep = _problems([it], q)
    q.batch_qless(probs)
    x = to_host(keep[0][3])
    x_ref, rho, _, _ = oracle.lstsq(A, b)
    assert np.linalg.norm(x[:20] - x_ref) <= 1e-10 * np.linalg.norm(x_ref)
    assert abs(x[20] - rho) <= 1e-8 * rho


def test_batch_launch_replays_in_a_cuda_graph():
    import paper_2603_20889_gb300 as q

    lib = q.load_library()
    insts = _instances(12, seed=2, m_hi=1 << 14)
    probs, keep = _problems(insts, q)
    arr = (q.Problem * len(probs))(*probs)
    nb = lib.ql_batch_workspace_bytes(len(probs), arr)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        assert lib.ql_batch_prepare(len(probs), arr, ws.data_ptr(), nb, q._stream_ptr(s)) == 0
        assert lib.ql_batch_launch(ws.data_ptr(), q._stream_ptr(s)) == 0  # first launch outside capture
    torch.cuda.synchronize()
    for _, _, R, _, info in keep:
        R.fill_(float("nan"))
        info.fill_(-1)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        assert lib.ql_batch_launch(ws.data_ptr(), q._stream_ptr(s)) == 0
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    _check_outputs(insts, keep)


def test_batch_equals_single_calls():
    """Batched and single-call results agree within the parity tolerance."""
    import paper_2603_20889_gb300 as q

    insts = [i for i in _instances(10, seed=3, m_hi=1 << 15) if i["kind"] == 0]
    probs, keep = _problems(insts, q)
    q.batch_qless(probs)
    for it, (Xd, _, R, _, _) in zip(insts, keep):
        Rs, _ = q.tsqr_qless(Xd)
        Rb = to_host(R)
        Rb = Rb.reshape(-1).reshape(Rb.shape, order="F")
        assert oracle.rel_err(Rb, to_host(Rs)) <= oracle.tolerance(it["n"], max(it["kappa"], 10.0))


def _serve(q, insts, budget=8 << 30, slots=4096, streams=4):
    srv = q.Server(budget, slots, streams)
    keep, tickets = [], []
    for it in insts:
        Xd = to_dev(it["X"])
        bd = torch.from_numpy(it["b"]).cuda() if it["kind"] else None
        keep.append((Xd, bd))
        req = q.Request(m=it["m"], n=it["n"], ld=Xd.stride(1) if it["n"] > 1 else it["m"], X=Xd.data_ptr(),
                        dtype=q.QL_F64 if it["dt"] == np.float64 else q.QL_F32, kind=it["kind"],
                        b=bd.data_ptr() if bd is not None else None, kappa_hint=it["kappa"])
        tickets.append(srv.submit(req))
    assert srv.drain(120.0) == 0
    cudart = q.load_library()  # dlsym on the library handle also finds cudart's symbols
    res = []
    for it, t in zip(insts, tickets):
        st, r = srv.poll(t)
        assert st == 0
        n1 = it["n"] + 1 if it["kind"] else it["n"]
        buf = np.zeros(n1 * n1)
        assert cudart.cudaMemcpy(ctypes.c_void_p(buf.ctypes.data), ctypes.c_void_p(r.R),
                                 ctypes.c_size_t(n1 * n1 * 8), ctypes.c_int(2)) == 0
        res.append((r.status, r.index, buf.reshape((n1, n1), order="F").copy(), r.latency_ms))
        srv.release(t)
    stats = srv.stats()
    srv.close()
    return res, stats


def test_server_alone_and_in_the_mix():
    """Each request's R is the same (within tolerance) alone and inside a busy mix."""
    import paper_2603_20889_gb300 as q

    insts = _instances(60, seed=4, m_hi=1 << 15)
    mix, stats = _serve(q, insts)
    assert stats.completed == 60 and stats.p99_ms >= stats.p50_ms > 0.0
    for it, (status, index, R, lat) in list(zip(insts, mix))[:20]:
        assert status == 0
        alone, _ = _serve(q, [it])
        assert oracle.rel_err(R, alone[0][2]) <= oracle.tolerance(R.shape[0], max(it["kappa"], 10.0))
        assert oracle.rel_err(R, _expected(it)) <= oracle.tolerance(R.shape[0], max(it["kappa"], 10.0))


def test_server_rejects_over_budget_and_bad_requests():
    import paper_2603_20889_gb300 as q

    srv = q.Server(256 << 20, 16, 1)
    big = q.Request(m=1 << 26, n=64, ld=1 << 26, X=16, dtype=q.QL_F64, kind=0, b=None, kappa_hint=1.0)
    t = ctypes.c_uint64(0)
    assert srv.lib.ql_server_submit(srv.h, ctypes.byref(big), ctypes.byref(t)) == q.QL_ERR_BUDGET
    bad = q.Request(m=100, n=65, ld=100, X=16, dtype=q.QL_F64, kind=0, b=None, kappa_hint=1.0)
    assert srv.lib.ql_server_submit(srv.h, ctypes.byref(bad), ctypes.byref(t)) == q.QL_ERR_ARG
    st, _ = srv.poll(12345)
    assert st == q.QL_ERR_UNKNOWN
    assert srv.stats().rejected == 1
    srv.close()


def test_server_completes_when_the_budget_is_the_limit():
    """Requests whose data exceed the HBM budget many times over still all complete: the
    server admits what fits, shrinks a group until its workspace fits, and never stalls."""
    import paper_2603_20889_gb300 as q

    m, n = 1 << 18, 10  # 21 MB per request
    X = torch.randn((n, m), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()  # the server's streams do not wait on the default stream
    srv = q.Server(128 << 20, 4096, 2)  # room for ~4 requests' data at a time
    tickets = [srv.submit(q.Request(m=m, n=n, ld=m, X=X.data_ptr(), dtype=q.QL_F64, kind=0, b=None,
                                    kappa_hint=1.0)) for _ in range(40)]
    assert srv.drain(60.0) == 0
    st = srv.stats()
    assert st.completed == 40
    assert st.hbm_peak_bytes <= 128 << 20
    R0 = None
    for t in tickets:
        s, r = srv.poll(t)
        assert s == 0 and r.status == 0
    srv.close()


def test_server_cancel_withdraws_queued_requests_only():
    """A client that gives up (host-side injection: it cancels its tickets) withdraws the
    requests still queued; launched ones complete normally, and the rest of the stream is
    unaffected."""
    import paper_2603_20889_gb300 as q

    m_big, n_big = 1 << 23, 64  # tens of ms of work: keeps the only slot busy while the rest queue
    Xb = torch.randn((n_big, m_big), dtype=torch.float64, device="cuda")
    m, n = 4096, 8
    X = torch.randn((n, m), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    srv = q.Server(8 << 30, 1, 1)  # one request in flight at a time
    first = srv.submit(q.Request(m=m_big, n=n_big, ld=m_big, X=Xb.data_ptr(), dtype=q.QL_F64, kind=0, b=None,
                                 kappa_hint=1.0))
    rest = [srv.submit(q.Request(m=m, n=n, ld=m, X=X.data_ptr(), dtype=q.QL_F64, kind=0, b=None, kappa_hint=1.0))
            for _ in range(6)]
    L = srv.lib
    cancelled = rest[1::2]
    for t in cancelled:
        assert L.ql_server_cancel(srv.h, t) == q.QL_OK
        assert L.ql_server_cancel(srv.h, t) == q.QL_ERR_UNKNOWN  # the ticket is gone
    assert srv.drain(60.0) == 0
    s, r = srv.poll(first)
    assert s == 0 and r.status == 0
    assert L.ql_server_cancel(srv.h, first) == q.QL_ERR_BUSY  # done: poll and release instead
    for t in rest:
        s, r = srv.poll(t)
        if t in cancelled:
            assert s == q.QL_ERR_UNKNOWN
        else:
            assert s == 0 and r.status == 0
    st = srv.stats()
    assert st.completed == 1 + len(rest) - len(cancelled)
    srv.close()


def _method_test_instances(seed):
    """Uneven problems of every tensor-core Gram class (9..64 columns) and narrower ones."""
    rng = np.random.default_rng(seed)
    out = []
    for k, n in enumerate([3, 9, 16, 17, 24, 31, 32, 40, 48, 64, 12, 28]):
        m = int(rng.integers(3000, 70000))
        kind = 1 if k % 4 == 3 else 0
        n = min(n, 63) if kind else n
        kappa = float(10 ** rng.uniform(0, 5))
        dt = np.float32 if k % 5 == 2 else np.float64
        X = synth.conditioned(m, n, kappa, seed=seed * 100 + k).astype(dt)
        b = (synth.gaussian(m, 1, seed=seed * 100 + k + 7)[:, 0]).astype(dt) if kind else None
        out.append(dict(m=m, n=n, kind=kind, kappa=kappa, X=X, b=b, dt=dt))
    return out


@pytest.mark.parametrize("hint", ["cholqr2", "auto"])
def test_batch_gram_method_class(hint):
    """Cholesky-QR2 problems of a batch run as work items of the grouped tensor-core Gram
    launches; every R (or least-squares solution) matches the oracle, and the plan reports
    the method it chose per problem."""
    import paper_2603_20889_gb300 as q

    insts = _method_test_instances(7)
    probs, keep = _problems(insts, q)
    for p, it in zip(probs, insts):
        p.method_hint = q.QL_CHOLQR2 if hint == "cholqr2" else q.QL_AUTO
        p.kappa_hint = it["kappa"]
    ws = q.batch_qless(probs)
    torch.cuda.synchronize()
    _check_outputs(insts, keep)
    meth = (ctypes.c_int32 * len(probs))()
    assert q.load_library().ql_batch_methods(ws.data_ptr(), meth, len(probs)) == q.QL_OK
    for it, mth in zip(insts, meth):
        ncols = it["n"] + it["kind"]
        if ncols <= 8:
            assert mth == q.QL_TSQR
        elif hint == "cholqr2":
            assert mth == q.QL_CHOLQR2
        else:
            assert mth == (q.QL_CHOLQR2 if ncols >= 24 else q.QL_TSQR)


def test_batch_gram_problems_fall_back_to_tsqr():
    """A Gram problem outside the double-float range, and (method chosen automatically) a
    rank-deficient one whose Cholesky breaks down, are redone by the batch's FP64 TSQR
    launch: both end with a valid R and info = QL_OK."""
    import paper_2603_20889_gb300 as q

    X1 = synth.conditioned(20000, 20, 1e2, seed=3) * 2.0 ** 70  # beyond the double-float range
    x = synth.gaussian(30000, 25, seed=4)
    X2 = np.column_stack([x, np.zeros(30000)])  # 26 columns, rank 25: the last pivot is exactly 0
    insts = [dict(m=20000, n=20, kind=0, kappa=1e2, X=X1, b=None, dt=np.float64),
             dict(m=30000, n=26, kind=0, kappa=1e3, X=X2, b=None, dt=np.float64)]
    probs, keep = _problems(insts, q)
    probs[0].method_hint, probs[0].kappa_hint = q.QL_CHOLQR2, 1e2
    probs[1].method_hint, probs[1].kappa_hint = q.QL_AUTO, 1e3
    ws = q.batch_qless(probs)
    torch.cuda.synchronize()
    (_, _, Ra, _, ia), (_, _, Rb, _, ib) = keep
    assert info_of(ia) == [0, 0] and info_of(ib) == [0, 0]
    Ra = to_host(Ra).reshape(-1).reshape((20, 20), order="F")
    assert oracle.rel_err(Ra, oracle.householder_r(X1)) <= oracle.tolerance(20, 1e2)
    Rb = to_host(Rb).reshape(-1).reshape((26, 26), order="F")
    assert np.linalg.norm(Rb.T @ Rb - X2.T @ X2) <= 1e-12 * np.linalg.norm(X2) ** 2


def test_batch_gram_class_replays_in_a_cuda_graph():
    import paper_2603_20889_gb300 as q

    insts = _method_test_instances(8)[:6]
    probs, keep = _problems(insts, q)
    for p, it in zip(probs, insts):
        p.method_hint, p.kappa_hint = q.QL_CHOLQR2, it["kappa"]
    L = q.load_library()
    arr = (q.Problem * len(probs))(*probs)
    nb = L.ql_batch_workspace_bytes(len(probs), arr)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        assert L.ql_batch_prepare(len(probs), arr, ws.data_ptr(), nb, q._stream_ptr(s)) == 0
        assert L.ql_batch_launch(ws.data_ptr(), q._stream_ptr(s)) == 0  # first launch before capture
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        assert L.ql_batch_launch(ws.data_ptr(), q._stream_ptr(s)) == 0
    for (_, _, R, _, info) in keep:
        R.fill_(float("nan"))
        info.fill_(-1)
    g.replay()
    torch.cuda.synchronize()
    _check_outputs(insts, keep)


def test_batch_tcgen05_class_runs_many_items_per_cta():
    """More (problem, chunk) work items of the 64-column class than SMs, so every CTA of the
    persistent tcgen05 launches runs several items on the same barriers and tensor memory.
    No bounded wait gives up (the FP64 redo would report {QL_ERR_TIMEOUT, where} in info),
    and every R and least-squares solution matches the oracle."""
    import time

    import paper_2603_20889_gb300 as q

    insts = []
    for k in range(12):
        kind = 1 if k % 6 == 5 else 0
        n = (40, 48, 64)[k % 3] - kind
        m = (1 << 17) + 37 * k  # ragged last tiles
        dt = np.float32 if k % 4 == 1 else np.float64
        kappa = 10.0 ** (1 + k % 4)
        X = synth.conditioned(m, n, kappa, seed=900 + k).astype(dt)
        b = (synth.gaussian(m, 1, seed=950 + k)[:, 0]).astype(dt) if kind else None
        insts.append(dict(m=m, n=n, kind=kind, kappa=kappa, X=X, b=b, dt=dt))
    probs, keep = _problems(insts, q)
    for p, it in zip(probs, insts):
        p.method_hint, p.kappa_hint = q.QL_CHOLQR2, it["kappa"]
    q.batch_qless(probs)  # first call: plan, upload, module load
    torch.cuda.synchronize()
    for (_, _, R, _, info) in keep:
        R.fill_(float("nan"))
        info.fill_(-1)
    t = time.perf_counter()
    ws = q.batch_qless(probs)
    torch.cuda.synchronize()
    elapsed = time.perf_counter() - t
    _check_outputs(insts, keep)
    meth = (ctypes.c_int32 * len(probs))()
    assert q.load_library().ql_batch_methods(ws.data_ptr(), meth, len(probs)) == q.QL_OK
    assert list(meth) == [q.QL_CHOLQR2] * len(probs)
    assert elapsed < 1.0, elapsed  # a bounded wait that gives up costs about 2 s
