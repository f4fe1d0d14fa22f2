"""Writes tests/golden/box_spectra.json from the oracle's closed form only.

Closed form: lumped P1 on the Kuhn split of a Dirichlet box reduces M^{-1} S to
the finite-difference Laplacian (oracle/spectra.py), so the eigenvalues of
eq. def:basisMatrixEVP inside a filter interval are known exactly. Run:
    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import spectra  # noqa: E402

CASES = [
    # name, cells, interval
    ("square64", (64, 64), (20.0, 30.0)),
    ("cube128", (128, 128, 128), (40.0, 45.0)),
    ("square32", (32, 32), (20.0, 30.0)),
]


def main():
    out = {}
    for name, cells, (a, b) in CASES:
        h = tuple(1.0 / c for c in cells)
        lam = spectra.eigenvalues_in(cells, h, a, b)
        vals, mult = spectra.distinct(lam)
        out[name] = dict(cells=list(cells), interval=[a, b], count=int(lam.size),
                         distinct=[float(v) for v in vals],
                         multiplicity=[int(k) for k in mult])
    with open(os.path.join(HERE, "box_spectra.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
