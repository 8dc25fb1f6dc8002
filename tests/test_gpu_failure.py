"""Device-side failure reporting without a GPU fault: a bounded mbarrier wait on which
nothing ever arrives gives up after its limit and the kernel returns {QL_ERR_TIMEOUT, where}
through info, leaving the context usable (the next call runs normally)."""
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_20889_gb300 as q

    q.load_library()
    return q


def _check(q, arrive, limit):
    info = torch.full((2,), -1, dtype=torch.int32, device="cuda")
    st = q.load_library().ql_check_bounded_wait(arrive, limit, info.data_ptr(), q._stream_ptr())
    assert st == q.QL_OK
    torch.cuda.synchronize()
    return info.cpu().tolist()


def test_wait_that_nothing_completes_reports_timeout(q):
    # about 1 ms at 2 GHz: nothing arrives, the wait runs out and the kernel returns
    assert _check(q, 0, 1 << 21) == [q.QL_ERR_TIMEOUT, 1]


def test_wait_that_completes_reports_ok_and_context_stays_usable(q):
    assert _check(q, 0, 1 << 20) == [q.QL_ERR_TIMEOUT, 1]
    assert _check(q, 1, 1 << 30) == [q.QL_OK, 0]
    # an ordinary factorisation right after the timed-out wait
    X = torch.randn(3, 5000, dtype=torch.float64, device="cuda").T
    R, info = q.tsqr_qless(X)
    torch.cuda.synchronize()
    assert info.cpu().tolist() == [0, 0]
    import oracle

    R_ref = oracle.householder_r(X.cpu().numpy())
    assert oracle.rel_err(R.cpu().numpy(), R_ref) <= oracle.tolerance(3, 10.0)


def test_bad_arguments_are_rejected_before_any_launch(q):
    L = q.load_library()
    info = torch.zeros(2, dtype=torch.int32, device="cuda")
    assert L.ql_check_bounded_wait(0, 1000, None, q._stream_ptr()) == q.QL_ERR_ARG
    assert L.ql_check_bounded_wait(0, -1, info.data_ptr(), q._stream_ptr()) == q.QL_ERR_ARG
    assert L.ql_check_bounded_wait(0, 1 << 40, info.data_ptr(), q._stream_ptr()) == q.QL_ERR_ARG
