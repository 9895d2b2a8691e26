"""Writes singular_reference.json: reference values of P0 Galerkin entries
for triangle pairs that share a vertex, an edge or the whole panel.

The values come only from ``oracle.reference_entry``: closed-form inner
integrals (triangle potential for the single layer, Eq. (1); solid angle for
the double layer, Eq. (2); Green's function Eq. (5)) with adaptive outer
quadrature, plus nested adaptive quadrature of the bounded Helmholtz
remainder G_k - G_0.  None of this uses the Gauss or Sauter-Schwab rules
whose accuracy the tests then check (Sec. 3.2.3).

Run:  python tests/golden/make_singular_reference.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

P = {
    0: [0.0, 0.0, 0.0], 1: [1.0, 0.0, 0.0], 2: [0.3, 0.8, 0.0],
    3: [0.5, -0.6, 0.4], 4: [-0.7, 0.2, 0.3], 5: [-0.4, -0.8, -0.1],
    6: [1.6, 0.9, 0.5], 7: [2.4, 0.7, 0.2], 8: [1.9, 1.6, 0.9],
}
PAIRS = {
    "identical": ([0, 1, 2], [0, 1, 2]),
    "edge": ([0, 1, 2], [1, 0, 3]),
    "vertex": ([0, 1, 2], [0, 4, 5]),
    "regular": ([0, 1, 2], [6, 7, 8]),
}
CASES = [
    ("identical", 0, 0.0), ("edge", 0, 0.0), ("edge", 1, 0.0), ("vertex", 0, 0.0),
    ("vertex", 1, 0.0), ("regular", 0, 0.0), ("regular", 1, 0.0),
    ("edge", 0, 2.0), ("edge", 1, 2.0), ("vertex", 0, 2.0), ("vertex", 1, 2.0),
]


def main():
    out = {"citation": "Eq. (1)-(2) and (5), Sec. 2; singular pairs per Sec. 3.2.3",
           "recipe": "oracle.reference_entry(order=6, tol=1e-12, maxdepth=14) for k=0; "
                     "order=5, tol=1e-11, maxdepth=11 for k != 0",
           "points": P, "pairs": PAIRS, "values": []}
    for name, op, k in CASES:
        ia, ib = PAIRS[name]
        a9 = [c for v in ia for c in P[v]]
        b9 = [c for v in ib for c in P[v]]
        if k == 0.0:
            v = oracle.reference_entry(a9, b9, op, 0.0, order=6, tol=1e-12, maxdepth=14)
        else:
            v = oracle.reference_entry(a9, b9, op, k, order=5, tol=1e-11, maxdepth=11)
        out["values"].append({"pair": name, "op": op, "k": k, "re": v.real, "im": v.imag})
        print(name, op, k, v, flush=True)
    with open(os.path.join(HERE, "singular_reference.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
