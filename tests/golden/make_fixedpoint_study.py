"""Writes tests/golden/fixedpoint_study.json: the fixed-point accuracy study of
Sec. IV.C (Fig. 1) run with oracle/fixedpoint.py, for stated word lengths.

    python tests/golden/make_fixedpoint_study.py

Calls only oracle/ (and the shared seeded input generators).
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import fixedpoint as fp  # noqa: E402

PARAMS = {"sizes": [4, 8, 16], "kappas": [10.0, 100.0, 1000.0], "frac_bits": [12, 16, 20, 24],
          "accumulate": ["round", "wide"], "count": 100, "seed": 2024}


def main():
    rows = fp.study(sizes=tuple(PARAMS["sizes"]), kappas=tuple(PARAMS["kappas"]),
                    frac_bits=tuple(PARAMS["frac_bits"]), accumulate=tuple(PARAMS["accumulate"]),
                    count=PARAMS["count"], seed=PARAMS["seed"])
    out = {"what": "mean relative Frobenius error of the upper half of X (against the binary64 inverse of "
                   "the quantised A) for A = Q diag(lambda) Q^T / kappa, lambda log-uniform on [1, kappa] with "
                   "lambda_1 = 1 and lambda_N = kappa, in signed Q(I.F) with I = ceil(log2 kappa) + 2; "
                   "'round' rounds every product, 'wide' accumulates exact products and rounds once",
           "citation": "Sec. IV.C and Fig. 1 (the figure and its word lengths are not in the text)",
           "params": PARAMS, "rows": rows}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fixedpoint_study.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(path, len(rows), "rows")


if __name__ == "__main__":
    main()
