"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, element by element.

Bar: ||R - R_ref||_F / ||R_ref||_F <= 1e-13 * n * kappa(X) for FP64 TSQR, and the same
bound row by row (every entry against its row's diagonal, oracle.row_err), which a wrong
small row at large kappa cannot pass; Cholesky-QR2 and SVQB2 are held to the same bounds for
kappa <= 1e6.  Sizes span several row tiles per CTA (at least three per CTA for every
column class of the TSQR kernels) and ragged tails; both the double-float default and the
native FP64 arithmetic are checked.
"""
import functools

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
    yield
    q.set_arith(q.QL_ARITH_DF)


@functools.lru_cache(maxsize=None)
def case(m, n, kappa, seed):
    X = synth.conditioned(m, n, kappa, seed)
    return X, oracle.householder_r(X)


ARITHS = ["df", "f64"]

TSQR_CASES = [
    (1, 1, 1.0), (5, 3, 1.0), (1000, 1, 1.0), (1000, 8, 1e4), (4097, 2, 1.0), (4097, 5, 1e2),
    (30011, 13, 1e4), (30011, 16, 1.0), (65537, 17, 1e3), (20000, 33, 1e2), (12000, 64, 1e2),
    (300007, 4, 1.0), (1048581, 8, 1e4), (200003, 16, 1e6), (60001, 32, 1e4), (40000, 48, 1e3),
]


# At least three row tiles per CTA for every column class of the TSQR kernel (tile rows B,
# CTAs per SM at the kernel's registers and shared memory): n <= 2: B = 2048, up to 4
# CTAs/SM; n <= 4: 1024, up to 4; n <= 8: 1024, 2; n <= 16: 1024, 1; n <= 32: 512, 1;
# n <= 64: 256, 1 -- m >= 3 x 152 x CTAs/SM x B, plus a ragged tail of 17 rows.
MULTI_TILE_CASES = [
    (3 * 304 * 4096 + 17, 1, 1.0), (3 * 304 * 4096 + 17, 2, 1e2), (3 * 304 * 2048 + 17, 4, 1e3),
    (3 * 304 * 1024 + 17, 7, 1e4), (3 * 152 * 1024 + 17, 9, 1e3), (3 * 152 * 1024 + 17, 16, 1e4),
    (3 * 152 * 512 + 17, 17, 1e3), (3 * 152 * 512 + 17, 32, 1e4), (3 * 152 * 256 + 17, 33, 1e2),
    (3 * 152 * 256 + 17, 64, 1e3),
]


def _arith(q, a):
    q.set_arith(q.QL_ARITH_DF if a == "df" else q.QL_ARITH_F64)


def check_r(R, R_ref, n, kappa):
    """The parity bound, normwise and row by row."""
    tol = oracle.tolerance(n, kappa)
    err, rerr = oracle.rel_err(R, R_ref), oracle.row_err(R, R_ref)
    assert err <= tol, ("frobenius", err, tol)
    assert rerr <= tol, ("row-scaled", rerr, tol)


@pytest.mark.parametrize("arith", ARITHS)
@pytest.mark.parametrize("m,n,kappa", TSQR_CASES)
def test_tsqr_matches_oracle(m, n, kappa, arith):
    import paper_2603_20889_gb300 as q

    _arith(q, arith)
    X, R_ref = case(m, n, kappa, m % 1000 + n)
    R, info = q.tsqr_qless(to_dev(X))
    R = to_host(R)
    assert info_of(info) == [0, 0]
    assert np.all(np.tril(R, -1) == 0.0) and np.all(np.diag(R) >= 0.0)
    check_r(R, R_ref, n, kappa)


@pytest.mark.parametrize("arith", ARITHS)
@pytest.mark.parametrize("m,n,kappa", MULTI_TILE_CASES)
def test_tsqr_multi_tile_per_cta(m, n, kappa, arith):
    """Every CTA folds at least three row tiles into its running triangle (the carry of R
    across tiles and the one-tile-ahead staging), in every column class."""
    import paper_2603_20889_gb300 as q

    _arith(q, arith)
    X, R_ref = case(m, n, kappa, n + 101)
    R, info = q.tsqr_qless(to_dev(X))
    R = to_host(R)
    assert info_of(info) == [0, 0]
    check_r(R, R_ref, n, kappa)


@pytest.mark.parametrize("arith", ARITHS)
@pytest.mark.parametrize("n", [1, 8, 16, 33, 64])
def test_exact_walsh_workload(n, arith):
    """X = H[:, J] H_64[:, K] R0 is exact in FP64 with R = sqrt(64 m) R0: every method against
    the exact R (no oracle rounding in the reference)."""
    import paper_2603_20889_gb300 as q

    _arith(q, arith)
    m, kappa = 1 << 18, 1e4
    X, R_exact = synth.hadamard_exact_case(m, n, kappa, seed=n + 5)
    Xd = to_dev(X)
    for fn in (q.tsqr_qless, q.cholqr2_qless, lambda x: q.svqb_qless(x)[::2]):
        R, info = fn(Xd)
        assert info_of(info) == [0, 0]
        check_r(to_host(R), R_exact, n, kappa)


@pytest.mark.parametrize("method", ["cholqr2", "svqb2"])
@pytest.mark.parametrize("arith", ARITHS)
@pytest.mark.parametrize("m,n,kappa", [
    (1000, 1, 1.0), (3001, 2, 1e2), (4097, 5, 1e4), (100003, 8, 1e6), (30011, 16, 1e3),
    (20011, 31, 1e4), (50000, 32, 1.0), (20000, 48, 1e2), (12000, 64, 1e3),
])
def test_gram_methods_match_oracle(m, n, kappa, arith, method):
    import paper_2603_20889_gb300 as q

    _arith(q, arith)
    X, R_ref = case(m, n, kappa, m % 997 + n)
    if method == "cholqr2":
        R, info = q.cholqr2_qless(to_dev(X))
    else:
        R, _, info = q.svqb_qless(to_dev(X))
    R = to_host(R)
    assert info_of(info) == [0, 0]
    check_r(R, R_ref, n, kappa)


@pytest.mark.parametrize("arith", ARITHS)
@pytest.mark.parametrize("m,n,kappa", [
    (1000, 1, 1.0), (4097, 5, 1e8), (100003, 8, 1e6), (30011, 16, 1e8), (20011, 31, 1e4),
    (50000, 32, 1e8), (12000, 64, 1e8), (20000, 48, 1e10),
])
def test_scholqr3_matches_oracle(m, n, kappa, arith):
    """Shifted Cholesky-QR3 (three Gram passes) against the Householder R, up to kappa = 1e10
    (beyond Cholesky-QR2's range); backward error ||R^T R - X^T X|| / ||X||^2 as well."""
    import paper_2603_20889_gb300 as q

    _arith(q, arith)
    X, R_ref = case(m, n, kappa, m % 991 + n)
    R, info = q.scholqr3_qless(to_dev(X))
    R = to_host(R)
    assert info_of(info) == [0, 0]
    err = oracle.rel_err(R, R_ref)
    assert err <= oracle.tolerance(n, kappa), (err, oracle.tolerance(n, kappa))
    assert np.linalg.norm(R.T @ R - X.T @ X) <= 1e-13 * n * np.linalg.norm(X) ** 2


def test_scholqr3_breakdown_reports_pass_and_pivot():
    """A zero column survives the shifted first pass and breaks the second at its pivot."""
    import paper_2603_20889_gb300 as q

    x = synth.gaussian(4000, 3, seed=9)
    R, info = q.scholqr3_qless(to_dev(np.column_stack([x, np.zeros(4000)])))
    assert info_of(info) == [q.QL_ERR_NOT_SPD, 1004]
    assert np.all(np.isnan(to_host(R)))


def _colmajor_dev(A):
    return torch.tensor(np.ascontiguousarray(A.T)).cuda().T


@pytest.mark.parametrize("m,n,kappa", [
    (1, 1, 1.0), (1000, 1, 1.0), (4097, 5, 1e2), (30011, 16, 1e4), (20011, 31, 1e4), (12000, 64, 1e3),
    (300007, 8, 1.0), (70001, 48, 1e6),
])
def test_q_from_r_matches_oracle(m, n, kappa):
    """Q = X R^{-1} element by element against the oracle's forward substitution, and
    orthonormal to kappa-scaled rounding."""
    import paper_2603_20889_gb300 as q

    X, R_ref = case(m, n, kappa, m % 977 + n)
    Q, info = q.q_from_r(to_dev(X), _colmajor_dev(R_ref))
    assert info_of(info) == [0, 0]
    Q = to_host(Q)
    Q_ref, st = oracle.q_from_r(X, R_ref)
    assert st == 0
    assert oracle.rel_err(Q, Q_ref) <= oracle.tolerance(n, kappa)
    if m >= n:
        assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= 1e-12 * n * kappa


def test_q_from_r_fp32_and_range_fallback():
    """FP32 X gives FP32 Q (to float rounding); X scaled by 2^70 (outside the double-float
    range, FP64 tiles) with R scaled alike gives the same Q."""
    import paper_2603_20889_gb300 as q

    X, R_ref = case(40003, 24, 1e3, 3)
    Q_ref, _ = oracle.q_from_r(X, R_ref)
    Q32, info = q.q_from_r(to_dev(X.astype(np.float32)), _colmajor_dev(R_ref))
    assert info_of(info) == [0, 0] and Q32.dtype == torch.float32
    X32 = X.astype(np.float32).astype(np.float64)
    Q_ref32, _ = oracle.q_from_r(X32, R_ref)
    assert oracle.rel_err(to_host(Q32).astype(np.float64), Q_ref32) <= 1e-6
    Qs, info = q.q_from_r(to_dev(X * 2.0 ** 70), _colmajor_dev(R_ref * 2.0 ** 70))
    assert info_of(info) == [0, 0]
    assert oracle.rel_err(to_host(Qs), Q_ref) <= oracle.tolerance(24, 1e3)


def test_q_from_r_zero_pivot_reports_and_fills_nan():
    import paper_2603_20889_gb300 as q

    X, R_ref = case(5000, 6, 1.0, 5)
    Rz = R_ref.copy()
    Rz[3, 3] = 0.0
    Q, info = q.q_from_r(to_dev(X), _colmajor_dev(Rz))
    assert info_of(info) == [q.QL_ERR_NOT_SPD, 4]
    assert np.all(np.isnan(to_host(Q)))


def _orthonormal_basis(m, k, seed):
    Y = synth.gaussian(m, k, seed=seed)
    Q, info = oracle.q_from_r(Y, oracle.householder_r(Y))
    assert info == 0
    return Q


@pytest.mark.parametrize("m,k,n", [(1, 1, 1), (1000, 3, 5), (30011, 16, 16), (20011, 31, 9), (12000, 64, 64),
                                   (100003, 8, 40)])
def test_project_out_matches_oracle(m, k, n):
    """Two-phase orthogonalisation: W and C element by element against the oracle, W
    orthogonal to Y and X = Y C + W."""
    import paper_2603_20889_gb300 as q

    Y = _orthonormal_basis(m, k, 31 + k) if m >= k else synth.gaussian(m, k, seed=3)
    X = synth.gaussian(m, n, seed=32 + n) + Y @ synth.gaussian(k, n, seed=33)  # largely in range(Y)
    W_ref, C_ref = oracle.project_out(Y, X)
    W, C = q.project_out(to_dev(Y), to_dev(X))
    W, C = to_host(W), to_host(C)
    scale = np.linalg.norm(X)
    assert np.linalg.norm(W - W_ref) <= 1e-13 * (k + n) * scale
    assert np.linalg.norm(C - C_ref) <= 1e-13 * (k + n) * scale
    if m >= k:
        assert np.linalg.norm(Y.T @ W) <= 1e-13 * (k + n) * scale
    assert np.linalg.norm(Y @ C + W - X) <= 1e-13 * (k + n) * scale


def test_project_out_fp32_inplace_and_exact_orthogonal_case():
    """FP32 storage (W to float rounding), W written over X, and Hadamard columns exactly
    orthogonal to Y giving C = 0 and W = X bitwise."""
    import paper_2603_20889_gb300 as q

    m, k, n = 40000, 12, 10
    Y = _orthonormal_basis(m, k, 41)
    X = synth.gaussian(m, n, seed=42)
    W_ref, C_ref = oracle.project_out(Y.astype(np.float32).astype(np.float64), X.astype(np.float32).astype(np.float64))
    Xd = to_dev(X.astype(np.float32))
    W, C = q.project_out(to_dev(Y.astype(np.float32)), Xd, W=Xd)  # in place
    assert W.data_ptr() == Xd.data_ptr()
    assert np.linalg.norm(to_host(W).astype(np.float64) - W_ref) <= 1e-6 * np.linalg.norm(X)
    assert np.linalg.norm(to_host(C) - C_ref) <= 1e-6 * np.linalg.norm(X)
    H = synth.hadamard_columns(65536, 24)
    Yh, Xh = H[:, :8] / 256.0, H[:, 8:]
    W, C = q.project_out(to_dev(Yh), to_dev(Xh))
    assert np.all(to_host(C) == 0.0) and np.array_equal(to_host(W), Xh)


@pytest.mark.parametrize("m,n,kappa,dtype", [
    (5000, 65, 1e2, "f64"), (20011, 100, 1e3, "f64"), (30000, 130, 1e2, "f64"), (8000, 200, 10.0, "f64"),
    (12000, 40, 1e3, "f64"), (20000, 96, 1e2, "f32"),
])
def test_qr_wide_matches_oracle(m, n, kappa, dtype):
    """n > 64 by 64-column panels (block Gram-Schmidt with two-phase projections + TSQR):
    R against the oracle's Householder R, Q orthonormal, Q R = X."""
    import paper_2603_20889_gb300 as q

    X, R_ref = case(m, n, kappa, m % 983 + n)
    Xs = X.astype(np.float32) if dtype == "f32" else X
    if dtype == "f32":
        R_ref = oracle.householder_r(Xs.astype(np.float64))
    Q, R, info = q.qr_wide(to_dev(Xs))
    assert info_of(info) == [0, 0]
    Q, R = to_host(Q).astype(np.float64), to_host(R)
    assert np.all(np.tril(R, -1) == 0.0) and np.all(np.diag(R) > 0.0)
    assert oracle.rel_err(R, R_ref) <= (oracle.tolerance(n, kappa) if dtype == "f64" else 1e-5)
    orth = 1e-12 * n * kappa if dtype == "f64" else 1e-4
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= orth
    assert np.linalg.norm(Q @ R - Xs.astype(np.float64)) <= (1e-13 if dtype == "f64" else 1e-5) * n * np.linalg.norm(X)


def test_extension_entry_points_on_empty_and_single_column_inputs():
    """m = 0 and n = 1 through Q = X R^-1, the two-phase projection and the wide QR."""
    import paper_2603_20889_gb300 as q

    X0 = torch.zeros((3, 0), dtype=torch.float64, device="cuda").T  # 0 x 3, column-major
    R = _colmajor_dev(np.triu(np.ones((3, 3))))
    Q, info = q.q_from_r(X0, R)
    assert info_of(info) == [0, 0] and Q.shape == (0, 3)
    W, C = q.project_out(torch.zeros((2, 0), dtype=torch.float64, device="cuda").T, X0)
    assert W.shape == (0, 3) and np.all(to_host(C) == 0.0)
    x = synth.gaussian(5000, 1, seed=8)
    Qw, Rw, info = q.qr_wide(to_dev(x))
    assert info_of(info) == [0, 0]
    assert abs(to_host(Rw)[0, 0] - np.linalg.norm(x)) <= 1e-14 * np.linalg.norm(x)
    assert np.max(np.abs(to_host(Qw)[:, 0] - x[:, 0] / np.linalg.norm(x))) <= 1e-14


def test_svqb_z_factor():
    import paper_2603_20889_gb300 as q

    X, _ = case(20000, 12, 1e3, 5)
    R, Z, info = q.svqb_qless(to_dev(X), want_z=True)
    Z = to_host(Z)
    G = X.T @ X
    assert info_of(info) == [0, 0]
    assert np.linalg.norm(Z.T @ Z - G) <= 1e-12 * np.linalg.norm(G)


@pytest.mark.parametrize("method", ["tsqr", "cholqr2", "svqb2", "scholqr3"])
@pytest.mark.parametrize("m,n", [(65536, 8), (131072, 16), (32768, 64)])
def test_hadamard_exact(m, n, method):
    """X = H[:, :n] R0 exactly, so R = sqrt(m) R0: an exact expected value at any size."""
    import paper_2603_20889_gb300 as q

    X, R_exact = synth.hadamard_case(m, n, seed=3)
    fn = {"tsqr": q.tsqr_qless, "cholqr2": q.cholqr2_qless, "svqb2": lambda x: q.svqb_qless(x)[::2],
          "scholqr3": q.scholqr3_qless}[method]
    R, info = fn(to_dev(X))
    assert info_of(info) == [0, 0]
    kappa = np.linalg.cond(R_exact)
    assert oracle.rel_err(to_host(R), R_exact) <= oracle.tolerance(n, kappa)


@pytest.mark.parametrize("method", ["tsqr", "cholqr2", "svqb2"])
@pytest.mark.parametrize("m,n,kappa", [(50001, 8, 1e2), (20000, 31, 1e4), (4097, 3, 1.0), (30000, 64, 1e3)])
def test_fp32_storage(m, n, kappa, method):
    """FP32-stored X: parity with the oracle on the float-rounded X widened to double
    (the kernel's arithmetic), and the stated storage error against the FP64 X."""
    import paper_2603_20889_gb300 as q

    X64, R64 = case(m, n, kappa, 11)
    X32 = X64.astype(np.float32)
    R_ref32 = oracle.householder_r(X32.astype(np.float64))
    fn = {"tsqr": q.tsqr_qless, "cholqr2": q.cholqr2_qless, "svqb2": lambda x: q.svqb_qless(x)[::2]}[method]
    R, info = fn(to_dev(X32))
    R = to_host(R)
    assert info_of(info) == [0, 0]
    check_r(R, R_ref32, n, kappa)
    # storage error: bounded by kappa * 2^-24 (rounding X to float)
    assert oracle.rel_err(R, R64) <= 10 * n * kappa * 2.0 ** -24


def test_leading_dimension_larger_than_m():
    import paper_2603_20889_gb300 as q

    X, R_ref = case(10007, 9, 1e2, 3)
    big = np.zeros((10007 + 13, 9), order="F")
    big[:10007] = X
    t = to_dev(big)[:10007]  # (m, n) view with ld = m + 13
    assert t.stride(1) == 10020
    for fn in (q.tsqr_qless, q.cholqr2_qless):
        R, info = fn(t)
        assert info_of(info) == [0, 0]
        assert oracle.rel_err(to_host(R), R_ref) <= oracle.tolerance(9, 1e2)


@pytest.mark.parametrize("scale", [2.0 ** 70, 2.0 ** -60, 2.0 ** 200])
def test_range_fallback_recomputes_in_fp64(scale):
    """Magnitudes outside the double-float range are detected on the device and the FP64
    launch recomputes R in the same call (R(s X) = s R(X))."""
    import paper_2603_20889_gb300 as q

    q.set_arith(q.QL_ARITH_DF)
    X, R_ref = case(20000, 7, 1e2, 4)
    for fn in (q.tsqr_qless, q.cholqr2_qless):
        R, info = fn(to_dev(X * scale))
        assert info_of(info) == [0, 0]
        assert oracle.rel_err(to_host(R) / scale, R_ref) <= oracle.tolerance(7, 1e2)


@pytest.mark.parametrize("lm,e", [(28, 50), (26, 50)])
def test_range_guard_accounts_for_m(lm, e):
    """A constant column x = 1.875 2^e: its entries sit inside the double-float range, but the
    running norm sqrt(m) |x| and the Gram entry m x^2 do not once m is large; the range check
    must send the call to FP64, which gives R = sqrt(m) x = 1.875 2^(e + lm/2) exactly."""
    import paper_2603_20889_gb300 as q

    q.set_arith(q.QL_ARITH_DF)
    m = 1 << lm
    x = torch.full((m,), 1.875 * 2.0 ** e, dtype=torch.float64, device="cuda")
    expect = 1.875 * 2.0 ** (e + lm // 2)
    for fn in (q.tsqr_qless, q.cholqr2_qless):
        R, info = fn(x.unsqueeze(1))
        assert info_of(info) == [0, 0]
        assert abs(float(to_host(R)[0, 0]) - expect) <= 1e-13 * expect
    del x
    torch.cuda.empty_cache()


def test_edge_cases():
    import paper_2603_20889_gb300 as q

    # m = 0: R = 0
    R, info = q.tsqr_qless(torch.empty((3, 0), dtype=torch.float64, device="cuda").T)
    assert info_of(info) == [0, 0] and np.all(to_host(R) == 0.0)
    # a zero column and a duplicated column: R^T R = X^T X, zero diagonal entry
    x = synth.gaussian(5000, 3, seed=2)
    X = np.column_stack([x[:, 0], np.zeros(5000), x[:, 1], 2.0 * x[:, 1], x[:, 2]])
    R, info = q.tsqr_qless(to_dev(X))
    R = to_host(R)
    assert info_of(info) == [0, 0]
    assert R[1, 1] == 0.0
    assert abs(R[3, 3]) <= 1e-12 * np.linalg.norm(X)
    assert np.linalg.norm(R.T @ R - X.T @ X) <= 1e-12 * np.linalg.norm(X) ** 2
    # m < n
    Xs = synth.gaussian(3, 6, seed=1)
    R, info = q.tsqr_qless(to_dev(Xs))
    R = to_host(R)
    assert np.all(R[3:] == 0.0)
    assert np.linalg.norm(R.T @ R - Xs.T @ Xs) <= 1e-13 * np.linalg.norm(Xs) ** 2
    # NaN in X -> non-finite status
    Xn = synth.gaussian(3000, 4, seed=1)
    Xn[1234, 2] = np.nan
    R, info = q.tsqr_qless(to_dev(Xn))
    assert info_of(info)[0] == q.QL_ERR_NONFINITE


def test_cholqr2_breakdown_reports_pivot():
    import paper_2603_20889_gb300 as q

    x = synth.gaussian(4000, 3, seed=9)
    X = np.column_stack([x, np.zeros(4000)])  # rank 3: pivot 4 is exactly zero
    R, info = q.cholqr2_qless(to_dev(X))
    st = info_of(info)
    assert st == [q.QL_ERR_NOT_SPD, 4]
    assert np.all(np.isnan(to_host(R)))


@functools.lru_cache(maxsize=None)
def _lstsq_case(m, dtype):
    A, b, _ = synth.lstsq_case(m, 31, 1e3, seed=3)
    if dtype == "f32":
        A, b = A.astype(np.float32), b.astype(np.float32)
    return (A, b) + tuple(oracle.lstsq(A.astype(np.float64), b.astype(np.float64)))


@pytest.mark.parametrize("method", ["tsqr", "cholqr2", "scholqr3"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
# unaligned columns; 16-byte aligned columns (bulk tile copies); three TSQR tiles per CTA
@pytest.mark.parametrize("m", [60013, 60000, 3 * 152 * 512 + 17])
def test_lstsq_matches_oracle(method, dtype, m):
    import paper_2603_20889_gb300 as q

    A, b, x_ref, rho_ref, Re_ref, info_ref = _lstsq_case(m, dtype)
    assert info_ref == 0
    x, rn, Rext, info = q.lstsq_qless(to_dev(A), torch.from_numpy(b).cuda(),
                                      method={"tsqr": q.QL_TSQR, "cholqr2": q.QL_CHOLQR2,
                                              "scholqr3": q.QL_SCHOLQR3}[method], want_rext=True)
    assert info_of(info) == [0, 0]
    x = to_host(x)
    kappa = 1e3
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) <= oracle.tolerance(32, kappa)
    assert abs(float(to_host(rn)[0]) - rho_ref) <= 1e-8 * rho_ref
    assert oracle.rel_err(to_host(Rext), Re_ref) <= oracle.tolerance(32, kappa)


def test_repeat_calls_are_bitwise_identical():
    """Deterministic reductions: the same call twice gives the same bits."""
    import paper_2603_20889_gb300 as q

    X, _ = case(300007, 16, 1e3, 1)
    Xd = to_dev(X)
    for fn in (q.tsqr_qless, q.cholqr2_qless):
        R1 = to_host(fn(Xd)[0]).copy()
        R2 = to_host(fn(Xd)[0])
        assert np.array_equal(R1, R2)
