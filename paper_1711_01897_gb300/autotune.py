"""Autotuner for the assembly launch configuration and for the regular
quadrature order per distance class of the admissible blocks.

For a representative mesh it times hmat_assemble (device time of the near
field plus the persistent ACA, from the library's own events) under each
candidate row threshold: blocks up to `warp_max_rows` rows are compressed by
one warp each, up to `lane_max_rows` by one lane each, larger ones by a whole
CTA.  A candidate is admissible only if its H-matrix product agrees with the
baseline candidate's to 2 * aca_eps (the thresholds change no arithmetic, but
ACA pivot near-ties may resolve differently).  The fastest admissible
candidate is written to a JSON tuning table that `apply()` loads.

With --quadrature it also searches the distance classes (bem_set_quadrature):
blocks with dist / h >= rho1 use the centroid rule, >= rho3 the 3-point
degree-2 rule, the rest the paper's 6-point rule.  A candidate is admissible
only if its H-matrix product stays within `accuracy` * aca_eps (default 0.5)
of the product with the 6-point rule everywhere, so the product's error bound
of 2 aca_eps against the dense matrix keeps its margin.  The fastest
admissible candidate goes to a separate table (quadrature.json) that
`apply_quadrature()` loads on request: the library's default stays the
paper's rule.

    python -m paper_1711_01897_gb300.autotune [--level 5] [--out tuning.json] [--quadrature]
"""
from __future__ import annotations

import argparse
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_TABLE = os.path.join(HERE, "tuning.json")
DEFAULT_QUAD_TABLE = os.path.join(HERE, "quadrature.json")

WARP_CANDIDATES = (160, 320, 640, 1280, 2560, 8192)
LANE_CANDIDATES = (0, 24, 48)
RHO3_CANDIDATES = (0.0, 4.0, 6.0, 8.0, 12.0)
RHO1_CANDIDATES = (0.0, 16.0, 24.0, 32.0, 48.0)


def choose(results, eps):
    """results: list of dicts with keys warp_max_rows, lane_max_rows,
    time_ms, rel_diff.  Returns the fastest admissible entry."""
    ok = [r for r in results if r["rel_diff"] <= 2.0 * eps]
    if not ok:
        raise RuntimeError("no candidate meets the accuracy constraint")
    return min(ok, key=lambda r: (r["time_ms"], -r["warp_max_rows"], r["lane_max_rows"]))


def shortlist(results, eps, n=3, default=(8192, 0)):
    """The n fastest admissible candidates and the library default, as
    (warp_max_rows, lane_max_rows) pairs, for a confirmation round with more
    repetitions (a single timing of a persistent launch varies by several
    percent between runs)."""
    ok = sorted((r for r in results if r["rel_diff"] <= 2.0 * eps), key=lambda r: r["time_ms"])
    pairs = [(r["warp_max_rows"], r["lane_max_rows"]) for r in ok[:n]]
    if default not in pairs:
        pairs.append(default)
    return pairs


def measure(V, T, ops=(0, 1), eps=1e-5, prec=1, reps=2, warp=WARP_CANDIDATES,
            lane=LANE_CANDIDATES, leaf=32, eta=1.2, k=0.0, pairs=None):
    """k != 0: the Helmholtz operators (complex entries and factors).  pairs:
    explicit (warp, lane) candidates instead of the product of warp and lane."""
    from . import bem
    mesh = bem.Mesh(V, T)
    x = np.random.default_rng(0).normal(size=T.shape[0])
    if k != 0.0:
        x = x + 0j
    base = {}
    results = []
    saved = bem.bem_get_tuning()
    try:
        cands = pairs if pairs is not None else [(w, l) for w in warp for l in lane]
        for w, l in cands:
            if l > w:
                continue
            bem.bem_set_tuning(w, l, 0)
            total, diffs = 0.0, []
            for op in ops:
                h = bem.HMatrix(mesh, leaf, eta)
                times = []
                for _ in range(reps):
                    h.assemble(op, k, eps, prec)
                    st = h.stats()
                    times.append(st["time_near_ms"] + st["time_far_ms"])
                y = h.matvec(x)
                h.close()
                if op not in base:
                    base[op] = y
                diffs.append(float(np.linalg.norm(y - base[op]) / np.linalg.norm(base[op])))
                total += min(times)
            results.append({"warp_max_rows": w, "lane_max_rows": l, "time_ms": total,
                            "rel_diff": max(diffs)})
    finally:
        bem.bem_set_tuning(saved["warp_max_rows"], saved["lane_max_rows"], saved["use_graphs"])
        mesh.close()
    return results


def choose_quadrature(results, eps, accuracy=0.5):
    """results: dicts with keys rho3, rho1, time_ms, rel_diff (product
    against the 6-point product).  Returns the fastest admissible entry; the
    6-point candidate (0, 0) is always admissible."""
    ok = [r for r in results if r["rel_diff"] <= accuracy * eps]
    if not ok:
        raise RuntimeError("no candidate meets the accuracy constraint")
    return min(ok, key=lambda r: (r["time_ms"], -r["rho3"] if r["rho3"] else 0.0,
                                  -r["rho1"] if r["rho1"] else 0.0))


def quadrature_candidates(rho3=RHO3_CANDIDATES, rho1=RHO1_CANDIDATES):
    """(rho3, rho1) pairs with the centroid class beyond the 3-point class."""
    return [(a, b) for a in rho3 for b in rho1 if b == 0.0 or a == 0.0 or b > a]


def measure_quadrature(V, T, ops=(0, 1), eps=1e-5, reps=2, candidates=None, leaf=32, eta=1.2):
    """Times the mixed Laplace assemblies (near field + ACA, from the
    library's events) of trees built under each pair of class thresholds, and
    the relative difference of their products from the 6-point products."""
    from . import bem
    cands = quadrature_candidates() if candidates is None else list(candidates)
    if (0.0, 0.0) not in cands:
        cands = [(0.0, 0.0)] + cands
    cands.sort(key=lambda c: (c != (0.0, 0.0), c))
    mesh = bem.Mesh(V, T)
    x = np.random.default_rng(1).normal(size=T.shape[0])
    base = {}
    results = []
    saved = bem.bem_get_quadrature()
    try:
        for r3, r1 in cands:
            bem.bem_set_quadrature(r3, r1)
            total, diffs, n3, n1 = 0.0, [], 0, 0
            for op in ops:
                h = bem.HMatrix(mesh, leaf, eta)
                times = []
                for _ in range(reps):
                    h.assemble(op, 0.0, eps, bem.MIXED)
                    st = h.stats()
                    times.append(st["time_near_ms"] + st["time_far_ms"])
                n3, n1 = st["n_blocks_rule3"], st["n_blocks_rule1"]
                y = h.matvec(x)
                h.close()
                if op not in base:
                    base[op] = y
                diffs.append(float(np.linalg.norm(y - base[op]) / np.linalg.norm(base[op])))
                total += min(times)
            results.append({"rho3": r3, "rho1": r1, "time_ms": total, "rel_diff": max(diffs),
                            "blocks_rule3": int(n3), "blocks_rule1": int(n1)})
    finally:
        bem.bem_set_quadrature(saved["rho3"], saved["rho1"])
        mesh.close()
    return results


def apply_quadrature(path: str = DEFAULT_QUAD_TABLE) -> bool:
    """Loads the distance classes of a quadrature table (if it exists); the
    trees built afterwards use them."""
    if not os.path.exists(path):
        return False
    from . import bem
    with open(path) as f:
        t = json.load(f)
    bem.bem_set_quadrature(float(t["rho3"]), float(t["rho1"]))
    return True


def apply(path: str = DEFAULT_TABLE) -> bool:
    """Loads a tuning table (if it exists) into the library."""
    if not os.path.exists(path):
        return False
    from . import bem
    with open(path) as f:
        t = json.load(f)
    bem.bem_set_tuning(t["warp_max_rows"], t["lane_max_rows"], t.get("use_graphs", 1))
    return True


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--level", type=int, default=5)
    ap.add_argument("--ellipsoid-nu", type=int, default=0,
                    help="tune on the 10 x 1 x 1 ellipsoid of this geodesic frequency instead of the "
                         "jittered sphere, Helmholtz single layer at 10 elements per wavelength")
    ap.add_argument("--eps", type=float, default=1e-5)
    ap.add_argument("--out", default=DEFAULT_TABLE)
    ap.add_argument("--quadrature", action="store_true",
                    help="also search the distance classes of the regular rule")
    ap.add_argument("--quad-out", default=DEFAULT_QUAD_TABLE)
    args = ap.parse_args()
    import torch
    from . import meshes
    torch.cuda.init()
    if args.ellipsoid_nu > 0:
        V, T = meshes.ellipsoid(args.ellipsoid_nu)
        k = meshes.helmholtz_k_10_per_wavelength(V, T)
        first = measure(V, T, ops=(0,), eps=args.eps, reps=1, k=k)
        res = measure(V, T, ops=(0,), eps=args.eps, reps=3, k=k,
                      pairs=shortlist(first, args.eps))
        what = (f"Helmholtz SLP, ellipsoid 10x1x1 nu {args.ellipsoid_nu} ({T.shape[0]} triangles), "
                f"k {k:.4g}, eps {args.eps}, mixed")
    else:
        V, T = meshes.icosphere_level(args.level)
        V = meshes.jitter(V, T, 0.05, 1001)
        first = measure(V, T, eps=args.eps)
        res = measure(V, T, eps=args.eps, reps=5, pairs=shortlist(first, args.eps))
        what = f"Laplace SLP+DLP, jittered icosphere level {args.level}, eps {args.eps}, mixed"
    best = choose(res, args.eps)
    table = {"warp_max_rows": best["warp_max_rows"], "lane_max_rows": best["lane_max_rows"],
             "use_graphs": 1, "time_ms": best["time_ms"], "workload": what, "candidates": first,
             "confirmation": res}
    with open(args.out, "w") as f:
        json.dump(table, f, indent=1)
    print(json.dumps({k: table[k] for k in ("warp_max_rows", "lane_max_rows", "time_ms")}))
    if args.quadrature and args.ellipsoid_nu == 0:
        apply(args.out)
        qres = measure_quadrature(V, T, eps=args.eps)
        qbest = choose_quadrature(qres, args.eps)
        qtable = {"rho3": qbest["rho3"], "rho1": qbest["rho1"], "time_ms": qbest["time_ms"],
                  "rel_diff": qbest["rel_diff"],
                  "workload": f"Laplace SLP+DLP, jittered icosphere level {args.level}, "
                              f"eps {args.eps}, mixed",
                  "candidates": qres}
        with open(args.quad_out, "w") as f:
            json.dump(qtable, f, indent=1)
        print(json.dumps({k: qtable[k] for k in ("rho3", "rho1", "time_ms", "rel_diff")}))


if __name__ == "__main__":
    main()
