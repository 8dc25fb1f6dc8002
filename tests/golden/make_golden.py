"""Write tests/golden/tiny_integer_r.json -- exact R factors of tiny integer matrices.

Each case is an integer X (m <= 8, n <= 4); its R (the unique upper triangular factor with
positive diagonal of X = QR, Q^T Q = I, Sec. 1 of the paper) is computed by
`oracle.exact.exact_r`: exact integer Gram matrix, then Cholesky in 60-digit decimal
arithmetic, rounded once to double.  This script calls only `oracle/`.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import random
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import exact  # noqa: E402


def cases():
    rnd = random.Random(20260320889)
    out = []
    shapes = [(1, 1), (3, 1), (2, 2), (4, 2), (5, 3), (8, 3), (6, 4), (8, 4), (7, 4)]
    for m, n in shapes:
        while True:
            X = [[rnd.randint(-9, 9) for _ in range(n)] for _ in range(m)]
            try:
                R = exact.exact_r(X)
                break
            except ValueError:  # singular draw: try again
                continue
        out.append({"m": m, "n": n, "X_rows": X, "R_rows": R})
    return out


if __name__ == "__main__":
    data = {
        "source": "exact integer Gram + 60-digit decimal Cholesky (oracle/exact.py); "
                  "definition of R: Sec. 1 (X = QR, Q^T Q = I, R upper triangular, diag > 0)",
        "cases": cases(),
    }
    with open(os.path.join(HERE, "tiny_integer_r.json"), "w") as f:
        json.dump(data, f, indent=1)
    print("wrote", len(data["cases"]), "cases")
