"""Seeded synthetic inputs shaped like the paper's workloads (Sec. 4.1).

This module is the only code that both the CUDA path's callers and the oracle's callers
use: it draws random matrices and nothing else.  It holds none of the factorisation's
arithmetic (no QR, Cholesky or eigensolver): random orthogonal factors come from the
Cayley transform of a random skew-symmetric matrix (one dense linear solve).

All host matrices are returned column-major (numpy Fortran order), m x n.
Device matrices are returned as torch tensors of shape (n, m), row-major, which is the
same memory as an m x n column-major matrix with leading dimension m.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


# --------------------------------------------------------------------------- host


def gaussian(m: int, n: int, seed: int, dtype=np.float64) -> np.ndarray:
    """X with i.i.d. N(0,1) entries (the plain workload of Sec. 4.1)."""
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.standard_normal((n, m)).T.astype(dtype))


def random_orthogonal(n: int, rng: np.random.Generator) -> np.ndarray:
    """A random n x n orthogonal matrix: Cayley transform (I - K)(I + K)^{-1}, K skew."""
    A = rng.standard_normal((n, n))
    K = (A - A.T) / (2.0 * math.sqrt(max(n, 1)))
    eye = np.eye(n)
    # (I - K)(I + K)^{-1} = solve((I + K)^T, (I - K)^T)^T
    return np.linalg.solve((eye + K).T, (eye - K).T).T


def spectrum(n: int, kappa: float) -> np.ndarray:
    """sigma_i = kappa^{-(i-1)/(n-1)}: geometric from 1 down to 1/kappa (sigma = 1 for n = 1)."""
    if n == 1:
        return np.ones(1)
    return kappa ** (-np.arange(n) / (n - 1.0))


def mixing_matrix(n: int, kappa: float, seed: int) -> np.ndarray:
    """S = V diag(sigma) W^T with V, W random orthogonal, so that X = G S has kappa_2 ~ kappa."""
    rng = np.random.default_rng(seed + 7919)
    V = random_orthogonal(n, rng)
    W = random_orthogonal(n, rng)
    return (V * spectrum(n, kappa)) @ W.T


def conditioned(m: int, n: int, kappa: float, seed: int, dtype=np.float64) -> np.ndarray:
    """X = G S with G m x n i.i.d. N(0,1) and S = V diag(sigma) W^T (condition sweep)."""
    G = gaussian(m, n, seed)
    X = G @ mixing_matrix(n, kappa, seed)
    return np.asfortranarray(X.astype(dtype))


def hadamard_columns(m: int, n: int) -> np.ndarray:
    """First n columns of the m x m Sylvester Hadamard matrix (m a power of two):
    H_ij = (-1)^popcount(i & j), so H^T H = m I."""
    if m & (m - 1) or m < n:
        raise ValueError("m must be a power of two and >= n")
    i = np.arange(m, dtype=np.int64)
    H = np.empty((m, n), order="F")
    for j in range(n):
        H[:, j] = 1.0 - 2.0 * (np.bitwise_count(i & j) & 1)
    return H


def small_upper(n: int, seed: int, lo: int = -3, hi: int = 3) -> np.ndarray:
    """A small-integer upper triangular R0: off-diagonal entries in lo..hi, diagonal in
    2n+1..2n+4 (rows are diagonally dominant, so R0 stays well conditioned at n = 64)."""
    rng = np.random.default_rng(seed + 104729)
    R0 = np.triu(rng.integers(lo, hi + 1, size=(n, n))).astype(np.float64)
    R0[np.diag_indices(n)] = rng.integers(2 * n + 1, 2 * n + 5, size=n)
    return R0


def hadamard_case(m: int, n: int, seed: int, dtype=np.float64):
    """(X, R_exact): X = H[:, :n] R0 is an exact integer matrix and R = sqrt(m) R0 exactly."""
    R0 = small_upper(n, seed)
    X = hadamard_columns(m, n) @ R0
    return np.asfortranarray(X.astype(dtype)), math.sqrt(m) * R0


def lstsq_case(m: int, n: int, kappa: float, seed: int, noise: float = 1e-6, dtype=np.float64):
    """(A, b, x_star): A = G S (kappa), x* ~ N(0,1), b = A x* + noise * N(0,1)."""
    A = conditioned(m, n, kappa, seed)
    rng = np.random.default_rng(seed + 31337)
    x_star = rng.standard_normal(n)
    b = A @ x_star + noise * rng.standard_normal(m)
    return np.asfortranarray(A.astype(dtype)), b.astype(dtype), x_star


def conditioned_upper(n: int, kappa: float, seed: int, bits: int = 36) -> np.ndarray:
    """An upper triangular R0 = T1 diag(sigma) T2 with positive diagonal, rounded to
    multiples of 2^-bits: T1, T2 unit upper triangular with off-diagonal entries uniform in
    [-1/(2n), 1/(2n)] (row sums below 1/2, so kappa(T) <= 3) and sigma the geometric
    spectrum from 1 to 1/kappa; kappa(R0) lies within a factor 9 of kappa.  Column j of R0
    carries the larger scales sigma_i (i < j) above its diagonal, so the columns of
    H R0 are nearly dependent in the way that makes Householder cancel."""
    rng = np.random.default_rng(seed + 7717)
    c = 0.5 / max(n, 1)
    T1 = np.eye(n) + np.triu(rng.uniform(-c, c, (n, n)), 1)
    T2 = np.eye(n) + np.triu(rng.uniform(-c, c, (n, n)), 1)
    R0 = np.triu((T1 * spectrum(n, kappa)) @ T2)
    return np.ldexp(np.rint(np.ldexp(R0, bits)), -bits)


def walsh_indices(m: int, n: int, seed: int) -> np.ndarray:
    """n distinct column indices of the m x m Sylvester Hadamard matrix, drawn at random."""
    rng = np.random.default_rng(seed + 3571)
    return np.sort(rng.choice(m, size=n, replace=False)).astype(np.int64)


WALSH_MIX = 64  # Walsh columns combined into every column of the exact workload


def walsh_mix(n: int, bits: int = 36, kappa: float = 1e4, seed: int = 0):
    """(B, R0): B = H_64[:, K] R0, 64 x n, with H_64 the 64 x 64 Sylvester Hadamard matrix and
    K n random distinct column indices (B^T B = 64 R0^T R0 exactly; for n >= 6 the 64 rows of
    B are distinct sign combinations of R0's rows), R0 = conditioned_upper(n, kappa, seed, bits)."""
    R0 = conditioned_upper(n, kappa, seed, bits)
    K = walsh_indices(WALSH_MIX, n, seed + 1)
    H = hadamard_columns(WALSH_MIX, WALSH_MIX)[:, K]
    return H @ R0, R0


def hadamard_exact_case(m: int, n: int, kappa: float, seed: int):
    """(X, R_exact) with X = H[:, J] B: J = 64 random distinct columns of the m x m Sylvester
    Hadamard matrix (orthogonal, norm sqrt(m)) and B = H_64[:, :n] R0 (walsh_mix, R0 a
    triangle of multiples of 2^-36 below 1.5 with kappa(R0) ~ kappa).  Each entry of X is a
    signed sum of 64 entries of B, so the rows of X take a new sign pattern almost every row
    (values close to Gaussian, no repeated rows for m < 2^64), every partial sum is a
    multiple of 2^-36 below 2^13, exact in FP64, and X^T X = 64 m R0^T R0 exactly: R =
    sqrt(64 m) R0 (m a power of two, n <= 64)."""
    if m & (m - 1) or m < WALSH_MIX or n > WALSH_MIX:
        raise ValueError("m must be a power of two >= 64 and n <= 64")
    B, R0 = walsh_mix(n, kappa=kappa, seed=seed)
    J = walsh_indices(m, WALSH_MIX, seed)
    i = np.arange(m, dtype=np.int64)
    X = np.zeros((m, n), order="F")
    for k in range(WALSH_MIX):
        h = 1.0 - 2.0 * (np.bitwise_count(i & J[k]) & 1)
        X += h[:, None] * B[k][None, :]
    return X, math.sqrt(WALSH_MIX * m) * R0


# --------------------------------------------------------------------------- device


def conditioned_device(m: int, n: int, kappa: float, seed: int, device="cuda", dtype=None,
                       chunk_rows: int = 1 << 22):
    """Device-resident X = G S as a (n, m) torch tensor (column-major m x n, ld = m).

    G is drawn by torch's seeded device generator in row chunks; S comes from the same
    host recipe as `conditioned`.  For kappa == 1 and S = I the plain Gaussian is returned.
    """
    import torch

    dtype = dtype or torch.float64
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    S = torch.from_numpy(mixing_matrix(n, kappa, seed)).to(device=device, dtype=torch.float64)
    Xt = torch.empty((n, m), dtype=dtype, device=device)
    for r0 in range(0, m, chunk_rows):
        r1 = min(m, r0 + chunk_rows)
        Gt = torch.randn((n, r1 - r0), generator=g, device=device, dtype=torch.float64)
        Xt[:, r0:r1] = (S.T @ Gt).to(dtype)
    return Xt


def hadamard_device(m: int, n: int, seed: int, device="cuda", dtype=None):
    """Device-resident Hadamard case: ((n, m) tensor, R_exact numpy)."""
    import torch

    dtype = dtype or torch.float64
    R0 = small_upper(n, seed)
    i = torch.arange(m, device=device, dtype=torch.int64)
    Xt = torch.zeros((n, m), dtype=torch.float64, device=device)
    for j in range(n):
        b = i & j
        par = torch.zeros_like(b)
        for _ in range(max(j.bit_length(), 1)):  # parity of popcount(i & j)
            par ^= b & 1
            b = b >> 1
        h = 1.0 - 2.0 * par.to(torch.float64)
        # X[:, c] += H[:, j] * R0[j, c]  (R0 is upper triangular)
        Xt += torch.from_numpy(R0[j, :]).to(device).unsqueeze(1) * h.unsqueeze(0)
    return Xt.to(dtype), math.sqrt(m) * R0


def hadamard_exact_device(m: int, n: int, kappa: float, seed: int, device="cuda"):
    """Device-resident `hadamard_exact_case`: ((n, m) FP64 tensor, R_exact numpy).  The sums
    are exact in any order, so the device X equals the host one bit for bit."""
    import torch

    if m & (m - 1) or m < WALSH_MIX or n > WALSH_MIX:
        raise ValueError("m must be a power of two >= 64 and n <= 64")
    B, R0 = walsh_mix(n, kappa=kappa, seed=seed)
    J = walsh_indices(m, WALSH_MIX, seed)
    i = torch.arange(m, device=device, dtype=torch.int64)
    Xt = torch.zeros((n, m), dtype=torch.float64, device=device)
    Bd = torch.from_numpy(np.ascontiguousarray(B)).to(device)
    for k in range(WALSH_MIX):
        b = i & int(J[k])
        for sh in (32, 16, 8, 4, 2, 1):  # parity of popcount(i & J_k)
            b = b ^ (b >> sh)
        h = 1.0 - 2.0 * (b & 1).to(torch.float64)
        Xt += Bd[k].unsqueeze(1) * h.unsqueeze(0)
        del b, h
    return Xt, math.sqrt(WALSH_MIX * m) * R0


# --------------------------------------------------------------------------- batched / serving


@dataclass
class Instance:
    m: int
    n: int
    kappa: float
    seed: int
    dtype: str = "f64"
    kind: str = "qr"  # "qr" or "lstsq"


def batched_instances(count: int = 512, seed: int = 4, m_lo: int = 1 << 10, m_hi: int = 1 << 20,
                      n_lo: int = 4, n_hi: int = 48, kappa_hi: float = 1e6):
    """Uneven batch: m log-uniform in [m_lo, m_hi], n uniform in {n_lo..n_hi},
    kappa log-uniform in [1, kappa_hi]."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        m = int(round(math.exp(rng.uniform(math.log(m_lo), math.log(m_hi)))))
        n = int(rng.integers(n_lo, n_hi + 1))
        kappa = float(math.exp(rng.uniform(0.0, math.log(kappa_hi))))
        out.append(Instance(max(m, n), n, kappa, seed * 100003 + k))
    return out


@dataclass
class Request(Instance):
    arrival_s: float = 0.0


def serving_stream(count: int = 20000, rate_per_s: float = 2000.0, seed: int = 5,
                   m_lo: int = 1 << 12, m_hi: int = 1 << 22, n_lo: int = 2, n_hi: int = 64,
                   frac_f32: float = 0.3, frac_lstsq: float = 0.2, kappa_hi: float = 1e6):
    """Poisson arrivals at `rate_per_s`; m log-uniform, n uniform, 30% FP32-stored,
    20% least-squares requests, kappa log-uniform in [1, kappa_hi]."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for k in range(count):
        t += float(rng.exponential(1.0 / rate_per_s))
        m = int(round(math.exp(rng.uniform(math.log(m_lo), math.log(m_hi)))))
        n = int(rng.integers(n_lo, n_hi + 1))
        dtype = "f32" if rng.uniform() < frac_f32 else "f64"
        kind = "lstsq" if rng.uniform() < frac_lstsq else "qr"
        if kind == "lstsq":
            n = min(n, n_hi - 1)  # [A b] has n + 1 <= n_hi columns
        kappa = float(math.exp(rng.uniform(0.0, math.log(kappa_hi))))
        out.append(Request(max(m, n + 1), n, kappa, seed * 1000003 + k, dtype, kind, t))
    return out
