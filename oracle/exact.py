"""Exact-arithmetic definition of R for tiny integer matrices -- TEST INFRASTRUCTURE ONLY.

A second, independent route to the same R as ``householder_r``: the Gram matrix of an
integer X is formed exactly with Python integers, then factored by Cholesky in 60-digit
decimal arithmetic (R^T R = X^T X with positive diagonal is the unique R of Sec. 1 when
rank(X) = n).  No floating point, no shared code with the C oracle.
"""
from decimal import Decimal, getcontext


def exact_gram(X):
    """Integer Gram matrix of a list-of-rows integer matrix."""
    m = len(X)
    n = len(X[0]) if m else 0
    return [[sum(int(X[i][p]) * int(X[i][q]) for i in range(m)) for q in range(n)] for p in range(n)]


def cholesky_decimal(C, digits=60):
    """Upper Cholesky factor of an integer SPD matrix in `digits`-digit decimal arithmetic.

    Returns R as a list of rows of Decimal, or raises ValueError on a non-positive pivot.
    """
    getcontext().prec = digits
    n = len(C)
    R = [[Decimal(0)] * n for _ in range(n)]
    for j in range(n):
        d = Decimal(C[j][j]) - sum((R[k][j] * R[k][j] for k in range(j)), Decimal(0))
        if d <= 0:
            raise ValueError(f"non-positive pivot at {j + 1}")
        R[j][j] = d.sqrt()
        for c in range(j + 1, n):
            s = Decimal(C[j][c]) - sum((R[k][j] * R[k][c] for k in range(j)), Decimal(0))
            R[j][c] = s / R[j][j]
    return R


def exact_r(X, digits=60):
    """R (as floats, rounded once from `digits`-digit decimals) of an integer matrix X."""
    R = cholesky_decimal(exact_gram(X), digits)
    return [[float(v) for v in row] for row in R]
