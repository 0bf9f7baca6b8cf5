"""Write tests/golden/exact_small.json: small triangular systems with their
exact rational solutions, computed only by oracle/exact.py (Gauss-Jordan in
fractions).  Inputs come from the seeded generator; run from the repo root:
    python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import exact  # noqa: E402
from paper_2305_19917_gb300 import inputs  # noqa: E402

CASES = [
    # side, uplo, trans, diag, m, n, alpha, seed
    (0, 0, 0, 0, 4, 3, 1.0, 1),
    (0, 1, 1, 1, 5, 2, 1.5, 2),
    (1, 0, 1, 0, 3, 6, -2.0, 3),
    (1, 1, 0, 1, 6, 4, 0.5, 4),
]


def main():
    out = {"source": "oracle/exact.py (exact rational Gauss-Jordan); inputs from "
                     "paper_2305_19917_gb300/inputs.py make_problem(seed)",
           "cases": []}
    for side, uplo, trans, diag, m, n, alpha, seed in CASES:
        A, B = inputs.make_problem(side, uplo, trans, diag, m, n, seed)
        X = exact.exact_trsm(side, uplo, trans, diag, alpha, A.tolist(), B.tolist())
        out["cases"].append(dict(side=side, uplo=uplo, trans=trans, diag=diag, alpha=alpha,
                                 A=A.tolist(), B=B.tolist(),
                                 X_exact=[[str(v) for v in row] for row in X]))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "exact_small.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path)


if __name__ == "__main__":
    main()
