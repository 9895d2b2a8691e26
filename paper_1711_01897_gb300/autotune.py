"""Autotuner for the assembly launch configuration.

For a representative mesh it times hmat_assemble (device time of the near
field plus the persistent ACA, from the library's own events) under each
candidate row threshold: blocks up to `warp_max_rows` rows are compressed by
one warp each, up to `lane_max_rows` by one lane each, larger ones by a whole
CTA.  A candidate is admissible only if its H-matrix product agrees with the
baseline candidate's to 2 * aca_eps (the thresholds change no arithmetic, but
ACA pivot near-ties may resolve differently).  The fastest admissible
candidate is written to a JSON tuning table that `apply()` loads.

    python -m paper_1711_01897_gb300.autotune [--level 5] [--out tuning.json]
"""
from __future__ import annotations

import argparse
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_TABLE = os.path.join(HERE, "tuning.json")

WARP_CANDIDATES = (160, 320, 640, 1280, 2560, 8192)
LANE_CANDIDATES = (0, 24, 48)


def choose(results, eps):
    """results: list of dicts with keys warp_max_rows, lane_max_rows,
    time_ms, rel_diff.  Returns the fastest admissible entry."""
    ok = [r for r in results if r["rel_diff"] <= 2.0 * eps]
    if not ok:
        raise RuntimeError("no candidate meets the accuracy constraint")
    return min(ok, key=lambda r: (r["time_ms"], -r["warp_max_rows"], r["lane_max_rows"]))


def measure(V, T, ops=(0, 1), eps=1e-5, prec=1, reps=2, warp=WARP_CANDIDATES,
            lane=LANE_CANDIDATES, leaf=32, eta=1.2):
    from . import bem
    mesh = bem.Mesh(V, T)
    x = np.random.default_rng(0).normal(size=T.shape[0])
    base = {}
    results = []
    saved = bem.bem_get_tuning()
    try:
        for w in warp:
            for l in lane:
                if l > w:
                    continue
                bem.bem_set_tuning(w, l, 0)
                total, diffs = 0.0, []
                for op in ops:
                    h = bem.HMatrix(mesh, leaf, eta)
                    times = []
                    for _ in range(reps):
                        h.assemble(op, 0.0, eps, prec)
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
    ap.add_argument("--eps", type=float, default=1e-5)
    ap.add_argument("--out", default=DEFAULT_TABLE)
    args = ap.parse_args()
    import torch
    from . import meshes
    torch.cuda.init()
    V, T = meshes.icosphere_level(args.level)
    V = meshes.jitter(V, T, 0.05, 1001)
    res = measure(V, T, eps=args.eps)
    best = choose(res, args.eps)
    table = {"warp_max_rows": best["warp_max_rows"], "lane_max_rows": best["lane_max_rows"],
             "use_graphs": 1, "time_ms": best["time_ms"],
             "workload": f"Laplace SLP+DLP, jittered icosphere level {args.level}, eps {args.eps}, mixed",
             "candidates": res}
    with open(args.out, "w") as f:
        json.dump(table, f, indent=1)
    print(json.dumps({k: table[k] for k in ("warp_max_rows", "lane_max_rows", "time_ms")}))


if __name__ == "__main__":
    main()
