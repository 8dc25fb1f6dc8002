"""Pins for the oracle: checks against closed forms, exact arithmetic, library routines and
invariants -- never against the oracle itself.  CPU only.

Each pin is chosen so that a plausible mistake (dropped term, wrong sign or index,
transposed operand) in the oracle fails at least one of them.
"""
import json
import math
import os
from decimal import Decimal, getcontext

import numpy as np
import pytest

import oracle
from oracle import exact
from paper_2603_20889_gb300 import synth

EPS = np.finfo(np.float64).eps
HERE = os.path.dirname(os.path.abspath(__file__))


# ---------------------------------------------------------------- closed forms


@pytest.mark.parametrize("m", [1, 2, 17, 1000])
def test_n1_is_the_column_norm(m):
    """n = 1: R = ||x||_2 (the 1 x 1 QR); compared with numpy's norm."""
    x = synth.gaussian(m, 1, seed=m)
    R = oracle.householder_r(x)
    assert R.shape == (1, 1)
    assert abs(R[0, 0] - np.linalg.norm(x[:, 0])) <= 4 * EPS * np.linalg.norm(x[:, 0])


def test_n1_negative_single_entry():
    R = oracle.householder_r(np.array([[-3.0]]))
    assert R[0, 0] == 3.0


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_n2_closed_form(seed):
    """n = 2: r11 = ||x1||, r12 = x1.x2 / r11, r22 = sqrt(||x2||^2 - r12^2), in 50 digits."""
    rng = np.random.default_rng(seed)
    X = rng.integers(-20, 21, size=(37, 2)).astype(np.float64)
    getcontext().prec = 50
    a = Decimal(int(np.dot(X[:, 0], X[:, 0])))
    b = Decimal(int(np.dot(X[:, 1], X[:, 1])))
    c = Decimal(int(np.dot(X[:, 0], X[:, 1])))
    r11 = a.sqrt()
    r12 = c / r11
    r22 = (b - r12 * r12).sqrt()
    R = oracle.householder_r(X)
    ref = np.array([[float(r11), float(r12)], [0.0, float(r22)]])
    assert np.max(np.abs(R - ref)) <= 8 * EPS * float(r11)


@pytest.mark.parametrize("m,n", [(256, 8), (1024, 16), (4096, 5), (2048, 33), (512, 64)])
def test_hadamard_construction_is_exact(m, n):
    """X = H[:, :n] R0 with H^T H = m I  =>  R = sqrt(m) R0 exactly."""
    X, R_exact = synth.hadamard_case(m, n, seed=n)
    R = oracle.householder_r(X)
    kappa = np.linalg.cond(R_exact)
    assert kappa < 10
    assert oracle.rel_err(R, R_exact) <= 1e-15 * n * kappa
    # each entry, not only the norm
    assert np.max(np.abs(R - R_exact)) <= 64 * EPS * np.max(np.abs(R_exact))


@pytest.mark.parametrize("m,n,kappa", [(1 << 12, 8, 1e4), (1 << 13, 16, 1e6), (1 << 12, 1, 1.0), (1 << 11, 33, 1e2)])
def test_random_walsh_columns_give_the_exact_r(m, n, kappa):
    """X = H[:, J] H_64[:, K] R0 with J, K random Hadamard columns and R0 a short-mantissa
    triangle: X is exact in FP64 and R = sqrt(64 m) R0 (the full-size accuracy reference of
    the benchmark)."""
    X, R_exact = synth.hadamard_exact_case(m, n, kappa, seed=n + 11)
    # both Hadamard factors have orthogonal columns: the exact Gram is 64 m R0^T R0
    R0 = R_exact / np.sqrt(synth.WALSH_MIX * m)
    G = synth.WALSH_MIX * m * (R0.T @ R0)
    assert np.allclose(X.T @ X, G, rtol=0, atol=64 * EPS * np.max(np.abs(G)) * n)
    R = oracle.householder_r(X)
    k = oracle.kappa2(R_exact)
    assert k < 10 * max(kappa, 1.0)
    assert oracle.rel_err(R, R_exact) <= 1e-15 * n * k
    assert oracle.row_err(R, R_exact) <= 1e-15 * n * k


def test_row_err_sees_a_wrong_last_row():
    """The row-scaled measure catches what the Frobenius ratio cannot at large kappa."""
    n, kappa = 16, 1e6
    R0 = synth.conditioned_upper(n, kappa, seed=5)
    bad = R0.copy()
    bad[-1, -1] *= 2.0  # the smallest row entirely wrong
    assert oracle.rel_err(bad, R0) <= oracle.tolerance(n, kappa)
    assert oracle.row_err(bad, R0) > oracle.tolerance(n, kappa)


# ---------------------------------------------------------------- exact arithmetic


def test_golden_tiny_integer_cases():
    with open(os.path.join(HERE, "golden", "tiny_integer_r.json")) as f:
        data = json.load(f)
    assert len(data["cases"]) >= 5
    for case in data["cases"]:
        X = np.array(case["X_rows"], dtype=np.float64)
        R_ref = np.array(case["R_rows"], dtype=np.float64)
        R = oracle.householder_r(X)
        assert np.max(np.abs(R - R_ref)) <= 16 * EPS * np.max(np.abs(R_ref)), case


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_random_tiny_integers(seed):
    """Brute force: exact Gram + 60-digit Cholesky on fresh tiny integer inputs."""
    rng = np.random.default_rng(100 + seed)
    m = int(rng.integers(4, 9))
    n = int(rng.integers(1, 5))
    X = rng.integers(-7, 8, size=(m, n))
    try:
        R_ref = np.array(exact.exact_r(X.tolist()))
    except ValueError:
        pytest.skip("singular draw")
    R = oracle.householder_r(X.astype(np.float64))
    assert np.max(np.abs(R - R_ref)) <= 16 * EPS * np.max(np.abs(R_ref))


# ---------------------------------------------------------------- invariants


@pytest.mark.parametrize("m,n,kappa", [(500, 8, 1.0), (3000, 16, 1e4), (800, 64, 1e2)])
def test_gram_identity_and_shape(m, n, kappa):
    """R^T R = X^T X (numpy's product), R upper triangular with nonnegative diagonal."""
    X = synth.conditioned(m, n, kappa, seed=m + n)
    R = oracle.householder_r(X)
    assert np.all(np.tril(R, -1) == 0.0)
    assert np.all(np.diag(R) >= 0.0)
    G = X.T @ X
    nx2 = np.linalg.norm(X) ** 2
    assert np.linalg.norm(R.T @ R - G) <= 10 * n * EPS * nx2


def test_invariance_row_permutation_and_zero_rows():
    X = synth.conditioned(400, 12, 1e3, seed=5)
    R = oracle.householder_r(X)
    perm = np.random.default_rng(0).permutation(400)
    Rp = oracle.householder_r(X[perm])
    Rz = oracle.householder_r(np.vstack([X[:150], np.zeros((77, 12)), X[150:]]))
    tol = oracle.tolerance(12, 1e3)
    assert oracle.rel_err(Rp, R) <= tol
    assert oracle.rel_err(Rz, R) <= tol


def test_power_of_two_scaling_is_bitwise():
    X = synth.conditioned(300, 7, 10.0, seed=9)
    R = oracle.householder_r(X)
    for k in (-40, -3, 5, 60):
        Rk = oracle.householder_r(np.ldexp(X, k))
        assert np.array_equal(Rk, np.ldexp(R, k))


def test_tsqr_stacking_identity():
    """R([X1; X2]) = R([R(X1); R(X2)]) -- the identity Algorithm 2 relies on."""
    X = synth.conditioned(1200, 9, 1e2, seed=11)
    R = oracle.householder_r(X)
    R1 = oracle.householder_r(X[:500])
    R2 = oracle.householder_r(X[500:])
    Rs = oracle.householder_r(np.vstack([R1, R2]))
    assert oracle.rel_err(Rs, R) <= oracle.tolerance(9, 1e2)


def test_rank_deficient_and_short_inputs():
    x = synth.gaussian(50, 1, seed=1)[:, 0]
    X = np.column_stack([x, 2 * x, synth.gaussian(50, 1, seed=2)[:, 0]])
    R = oracle.householder_r(X)
    assert abs(R[1, 1]) <= 1e-13 * np.linalg.norm(X)
    assert np.linalg.norm(R.T @ R - X.T @ X) <= 1e-13 * np.linalg.norm(X) ** 2
    Xs = synth.gaussian(3, 5, seed=3)  # m < n
    Rs = oracle.householder_r(Xs)
    assert np.all(Rs[3:, :] == 0.0)
    assert np.linalg.norm(Rs.T @ Rs - Xs.T @ Xs) <= 1e-13 * np.linalg.norm(Xs) ** 2
    R0 = oracle.householder_r(np.zeros((0, 4)))
    assert np.all(R0 == 0.0)
    Rzero = oracle.householder_r(np.zeros((10, 3)))
    assert np.all(Rzero == 0.0)


# ---------------------------------------------------------------- building blocks vs library


@pytest.mark.parametrize("n", [1, 4, 17, 64])
def test_cholesky_matches_numpy(n):
    X = synth.conditioned(4 * n + 10, n, 1e3, seed=n)
    C = X.T @ X
    R, info = oracle.cholesky_upper(C)
    assert info == 0
    L = np.linalg.cholesky(C)
    assert np.linalg.norm(R - L.T) <= 1e-10 * np.linalg.norm(L)


def test_cholesky_breakdown_index():
    assert oracle.cholesky_upper(np.array([[1.0, 2.0], [2.0, 1.0]]))[1] == 2
    assert oracle.cholesky_upper(np.array([[-1.0]]))[1] == 1
    assert oracle.cholesky_upper(np.array([[4.0, 2.0], [2.0, 1.0]]))[1] == 2  # exact zero pivot
    assert oracle.cholesky_upper(np.array([[4.0, 2.0, 0.0], [2.0, 5.0, 0.0], [0.0, 0.0, 0.0]]))[1] == 3


@pytest.mark.parametrize("n", [2, 7, 32, 64])
def test_jacobi_eig_matches_numpy(n):
    X = synth.conditioned(3 * n, n, 1e3, seed=n + 1)
    C = X.T @ X
    lam, U = oracle.jacobi_eig(C)
    ref = np.linalg.eigvalsh(C)
    assert np.max(np.abs(lam - ref)) <= 1e-12 * ref[-1]
    assert np.linalg.norm(U.T @ U - np.eye(n)) <= 1e-13 * n
    assert np.linalg.norm(C @ U - U * lam) <= 1e-12 * np.linalg.norm(C)


def test_singular_values_match_numpy():
    A = synth.conditioned(20, 20, 1e5, seed=3)[:20]
    s = oracle.singular_values(A)
    ref = np.linalg.svd(A, compute_uv=False)
    assert np.max(np.abs(s - ref) / ref) <= 1e-10


def test_kappa_of_conditioned_input():
    X = synth.conditioned(5000, 8, 1e4, seed=1)
    k = oracle.kappa2(oracle.householder_r(X))
    assert 1e3 < k < 1e5


# ---------------------------------------------------------------- the three methods agree


@pytest.mark.parametrize("kappa", [1.0, 1e3, 1e6])
def test_cholqr2_reaches_the_householder_r(kappa):
    """Algorithm 1 and Householder QR have the same R in exact arithmetic."""
    n = 10
    X = synth.conditioned(2000, n, kappa, seed=int(kappa) % 97)
    R_h = oracle.householder_r(X)
    R_c, R1, info = oracle.cholqr2(X)
    assert info == 0
    assert oracle.rel_err(R_c, R_h) <= oracle.tolerance(n, kappa)
    # the first pass alone is only good to ~kappa^2 eps
    assert oracle.rel_err(R1, R_h) <= max(1e-12, 1e3 * kappa * kappa * EPS)


def test_cholqr2_breaks_down_on_rank_deficiency():
    X = synth.gaussian(100, 3, seed=1)
    X = np.column_stack([X, X[:, 0] + X[:, 1]])
    X[:, 3] = X[:, 0] + X[:, 1]
    _, _, info = oracle.cholqr2(np.column_stack([X[:, :3], np.zeros(100)]))
    assert info == 4


@pytest.mark.parametrize("kappa", [1.0, 1e4, 1e6])
def test_svqb2_reaches_the_householder_r(kappa):
    n = 9
    X = synth.conditioned(1500, n, kappa, seed=3)
    R_h = oracle.householder_r(X)
    R_s, Z = oracle.svqb2(X)
    assert oracle.rel_err(R_s, R_h) <= oracle.tolerance(n, kappa)
    assert np.linalg.norm(Z.T @ Z - X.T @ X) <= 1e-12 * np.linalg.norm(X) ** 2


def test_svqb2_rank_deficient_gives_zero_diagonal():
    x = synth.gaussian(200, 3, seed=4)
    X = np.column_stack([x, x[:, 0] - x[:, 2]])
    R, _ = oracle.svqb2(X)
    assert np.min(np.abs(np.diag(R))) <= 1e-7 * np.linalg.norm(X)
    assert np.linalg.norm(R.T @ R - X.T @ X) <= 1e-12 * np.linalg.norm(X) ** 2


@pytest.mark.parametrize("kappa", [1.0, 1e4, 1e8, 1e10])
def test_scholqr3_reaches_the_householder_r(kappa):
    """Shifted Cholesky-QR3 has the exact R in exact arithmetic (the shift only changes the
    first, preconditioning pass), and stays backward stable far past Cholesky-QR2's range."""
    n = 12
    X = synth.conditioned(3000, n, kappa, seed=7)
    R_h = oracle.householder_r(X)
    R_s, info = oracle.scholqr3(X)
    assert info == 0
    assert oracle.rel_err(R_s, R_h) <= min(oracle.tolerance(n, kappa), 1e-9)
    assert np.linalg.norm(R_s.T @ R_s - X.T @ X) <= 1e-14 * n * np.linalg.norm(X) ** 2
    assert np.all(np.diag(R_s) > 0.0) and np.all(np.tril(R_s, -1) == 0.0)


def test_scholqr3_hadamard_exact_and_scaling():
    """X = H[:, :n] R0 gives R = sqrt(m) R0 exactly; X 2^k gives R 2^k bitwise (the shift
    scales with ||X||^2, every step commutes with a power-of-two scaling)."""
    X, R_exact = synth.hadamard_case(4096, 8, seed=2)
    R, info = oracle.scholqr3(X)
    assert info == 0
    assert oracle.rel_err(R, R_exact) <= oracle.tolerance(8, np.linalg.cond(R_exact))
    R_scaled, info2 = oracle.scholqr3(X * 2.0 ** -37)
    assert info2 == 0 and np.array_equal(R_scaled, R * 2.0 ** -37)


def test_scholqr3_breakdown_index_on_rank_deficiency():
    """A zero column leaves chol(C + s I) positive (the shift), so the breakdown comes in
    the second pass, at the zero column's pivot: 1000 + 4."""
    X = np.column_stack([synth.gaussian(200, 3, seed=5), np.zeros(200)])
    _, info = oracle.scholqr3(X)
    assert info == 1004


@pytest.mark.parametrize("kappa", [1.0, 1e4])
def test_q_from_r_is_orthonormal_and_reconstructs(kappa):
    """Q = X R^{-1} for the Householder R: Q^T Q = I (to kappa eps) and Q R = X."""
    n = 10
    X = synth.conditioned(2500, n, kappa, seed=11)
    R = oracle.householder_r(X)
    Q, info = oracle.q_from_r(X, R)
    assert info == 0
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= 1e-13 * n * kappa
    assert np.linalg.norm(Q @ R - X) <= 1e-14 * n * np.linalg.norm(X)


def test_q_from_r_hadamard_and_single_column():
    """X = H[:, :n] R0 has Q = H[:, :n] / sqrt(m); a single column gives x / ||x||."""
    m, n = 4096, 8
    X, R_exact = synth.hadamard_case(m, n, seed=4)
    Q, info = oracle.q_from_r(X, R_exact)
    assert info == 0
    H = X @ np.linalg.inv(R_exact / np.sqrt(m))  # exactly +-1 entries up to rounding
    assert np.max(np.abs(np.round(H) - H)) <= 1e-9 and np.all(np.abs(np.round(H)) == 1.0)
    assert np.max(np.abs(Q - np.round(H) / np.sqrt(m))) <= 1e-15
    x = synth.gaussian(333, 1, seed=5)
    q, _ = oracle.q_from_r(x, np.array([[np.linalg.norm(x)]]))
    assert np.max(np.abs(q[:, 0] - x[:, 0] / np.linalg.norm(x))) <= 1e-16


def test_q_from_r_zero_pivot():
    X = synth.gaussian(50, 3, seed=6)
    R = np.triu(np.ones((3, 3)))
    R[1, 1] = 0.0
    _, info = oracle.q_from_r(X, R)
    assert info == 2


def _orthonormal(m, k, seed):
    Y = synth.gaussian(m, k, seed=seed)
    Q, info = oracle.q_from_r(Y, oracle.householder_r(Y))
    assert info == 0
    return Q


def test_project_out_orthogonal_and_reconstructs():
    """Two projections leave W orthogonal to Y to rounding, and X = Y C + W."""
    m, k, n = 3000, 6, 5
    Y = _orthonormal(m, k, 21)
    X = synth.gaussian(m, n, seed=22)
    W, C = oracle.project_out(Y, X)
    assert np.linalg.norm(Y.T @ W) <= 1e-14 * np.linalg.norm(X)
    assert np.linalg.norm(Y @ C + W - X) <= 1e-14 * np.linalg.norm(X)
    assert np.linalg.norm(C - Y.T @ X) <= 1e-13 * np.linalg.norm(X)


def test_project_out_in_range_and_exactly_orthogonal():
    """X = Y B gives W ~ 0 and C ~ B; Hadamard columns orthogonal to Y give C = 0, W = X exactly."""
    m, k = 2000, 4
    Y = _orthonormal(m, k, 23)
    B = synth.gaussian(k, 3, seed=24)
    W, C = oracle.project_out(Y, Y @ B)
    assert np.linalg.norm(W) <= 1e-14 * np.linalg.norm(B)
    assert np.linalg.norm(C - B) <= 1e-14 * np.linalg.norm(B)
    H = synth.hadamard_columns(1024, 9)
    Yh, Xh = H[:, :4] / 32.0, H[:, 4:]
    Wh, Ch = oracle.project_out(Yh, Xh)
    assert np.all(Ch == 0.0) and np.array_equal(Wh, Xh)


# ---------------------------------------------------------------- least squares


def test_lstsq_consistent_integer_system():
    """b = A x* exactly  =>  x = x*, rho = 0."""
    A, _ = synth.hadamard_case(512, 6, seed=2)
    x_star = np.array([3.0, -1.0, 2.0, 0.0, 5.0, -4.0])
    b = A @ x_star  # exact: integers
    x, rho, Re, info = oracle.lstsq(A, b)
    assert info == 0
    assert np.max(np.abs(x - x_star)) <= 1e-13 * np.max(np.abs(x_star))
    assert rho <= 1e-12 * np.linalg.norm(b)


def test_lstsq_matches_numpy_and_residual():
    A, b, _ = synth.lstsq_case(3000, 11, 1e3, seed=8)
    x, rho, Re, info = oracle.lstsq(A, b)
    assert info == 0
    x_np = np.linalg.lstsq(A, b, rcond=None)[0]
    assert np.linalg.norm(x - x_np) <= 1e-10 * np.linalg.norm(x_np)
    r = b - A @ x
    assert abs(rho - np.linalg.norm(r)) <= 1e-8 * np.linalg.norm(r)
    assert np.linalg.norm(A.T @ r) <= 1e-9 * np.linalg.norm(A) * np.linalg.norm(b)
    assert Re.shape == (12, 12) and Re[11, 11] == rho


def test_back_substitution_against_numpy():
    R = np.triu(synth.gaussian(8, 8, seed=1)) + 4 * np.eye(8)
    z = synth.gaussian(8, 1, seed=2)[:, 0]
    x, info = oracle.back_substitution(R, z)
    assert info == 0
    assert np.allclose(x, np.linalg.solve(R, z), rtol=1e-13, atol=0)
    _, info0 = oracle.back_substitution(np.zeros((3, 3)), np.ones(3))
    assert info0 == 3


def test_tolerance_formula():
    assert oracle.tolerance(8, 1.0) == pytest.approx(8e-13)
    assert oracle.tolerance(16, 1e4) == pytest.approx(1.6e-8)
    assert math.isclose(oracle.rel_err(np.eye(2) * 2, np.eye(2)), 1.0)
