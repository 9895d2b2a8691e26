"""CUDA-graph replay of the assembly and the tuning thresholds change no
results (GPU)."""
import numpy as np
import pytest

from paper_1711_01897_gb300 import autotune, bem, meshes

pytestmark = pytest.mark.gpu


def test_graph_replay_matches_eager_and_counts_launches():
    import torch
    torch.cuda.init()
    V, T = meshes.icosphere_level(4)
    V = meshes.jitter(V, T, 0.05, 3)
    m = bem.Mesh(V, T)
    saved = bem.bem_get_tuning()
    x = np.random.default_rng(1).normal(size=T.shape[0])
    try:
        bem.bem_set_tuning(saved["warp_max_rows"], saved["lane_max_rows"], 0)
        h0 = bem.HMatrix(m, 32, 1.2)
        h0.assemble(bem.DLP, 0.0, 1e-5, bem.MIXED)
        y0 = h0.matvec(x)
        bem.bem_set_tuning(saved["warp_max_rows"], saved["lane_max_rows"], 1)
        h = bem.HMatrix(m, 32, 1.2)
        ys, counts = [], []
        for _ in range(3):          # eager, capture + launch, replay
            c0 = bem.bem_kernel_launches()
            h.assemble(bem.DLP, 0.0, 1e-5, bem.MIXED)
            counts.append(bem.bem_kernel_launches() - c0)
            ys.append(h.matvec(x))
        for y in ys:
            assert np.array_equal(y, y0)
        assert counts[0] == counts[1] == counts[2] > 0
        h.assemble(bem.SLP, 0.0, 1e-5, bem.MIXED)   # new key: eager again
        assert h.stats()["op"] == bem.SLP
    finally:
        bem.bem_set_tuning(saved["warp_max_rows"], saved["lane_max_rows"], saved["use_graphs"])


def test_thresholds_keep_results_and_autotuner_runs():
    import torch
    torch.cuda.init()
    V, T = meshes.icosphere_level(4)
    V = meshes.jitter(V, T, 0.05, 4)
    res = autotune.measure(V, T, ops=(bem.SLP,), eps=1e-5, reps=1, warp=(160, 8192), lane=(0, 24))
    assert len(res) == 4
    for r in res:
        assert r["rel_diff"] <= 2e-5 and r["time_ms"] > 0
    best = autotune.choose(res, 1e-5)
    assert best in res
    q = autotune.measure_quadrature(V, T, ops=(bem.SLP,), eps=1e-5, reps=1,
                                    candidates=[(0.0, 0.0), (6.0, 0.0), (6.0, 12.0)])
    assert [(r["rho3"], r["rho1"]) for r in q] == [(0.0, 0.0), (6.0, 0.0), (6.0, 12.0)]
    assert q[0]["rel_diff"] == 0.0 and q[0]["blocks_rule3"] == 0
    assert q[1]["blocks_rule3"] > 0 and q[2]["blocks_rule1"] > 0
    assert all(r["rel_diff"] < 1e-4 for r in q)
    assert autotune.choose_quadrature(q, 1e-5) in q
    assert bem.bem_get_quadrature() == {"rho3": 0.0, "rho1": 0.0}
