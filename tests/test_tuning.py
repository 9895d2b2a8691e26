"""Tuning API validation and the autotuner's selection rule (host only)."""
import pytest

from paper_1711_01897_gb300 import autotune, bem
from paper_1711_01897_gb300 import build as bem_build


@pytest.fixture(scope="module")
def lib():
    bem_build.build()
    return bem.load()


def test_set_get_and_validation(lib):
    saved = bem.bem_get_tuning()
    try:
        bem.bem_set_tuning(640, 24, 0)
        assert bem.bem_get_tuning() == {"warp_max_rows": 640, "lane_max_rows": 24, "use_graphs": 0}
        for bad in [(0, 0, 1), (9000, 0, 1), (640, 65, 1), (16, 24, 1), (640, 0, 2)]:
            with pytest.raises(bem.BemError):
                bem.bem_set_tuning(*bad)
    finally:
        bem.bem_set_tuning(saved["warp_max_rows"], saved["lane_max_rows"], saved["use_graphs"])


def test_autotuner_picks_fastest_accurate_candidate():
    res = [
        {"warp_max_rows": 640, "lane_max_rows": 0, "time_ms": 10.0, "rel_diff": 0.0},
        {"warp_max_rows": 1280, "lane_max_rows": 0, "time_ms": 8.0, "rel_diff": 1e-3},   # inaccurate
        {"warp_max_rows": 2560, "lane_max_rows": 24, "time_ms": 9.0, "rel_diff": 1e-6},
    ]
    best = autotune.choose(res, eps=1e-5)
    assert best["warp_max_rows"] == 2560 and best["lane_max_rows"] == 24
    with pytest.raises(RuntimeError):
        autotune.choose([dict(res[1])], eps=1e-5)


def test_quadrature_autotuner_selection_rule():
    res = [
        {"rho3": 0.0, "rho1": 0.0, "time_ms": 10.0, "rel_diff": 0.0},
        {"rho3": 4.0, "rho1": 0.0, "time_ms": 9.0, "rel_diff": 4e-6},
        {"rho3": 4.0, "rho1": 16.0, "time_ms": 7.0, "rel_diff": 2e-5},   # beyond 0.5 eps
        {"rho3": 6.0, "rho1": 32.0, "time_ms": 8.0, "rel_diff": 1e-6},
    ]
    best = autotune.choose_quadrature(res, eps=1e-5)
    assert (best["rho3"], best["rho1"]) == (6.0, 32.0)
    assert autotune.choose_quadrature(res[:3], eps=1e-5)["rho3"] == 4.0
    with pytest.raises(RuntimeError):
        autotune.choose_quadrature([dict(res[2])], eps=1e-5)
    cands = autotune.quadrature_candidates((0.0, 4.0, 24.0), (0.0, 16.0))
    assert (0.0, 0.0) in cands and (4.0, 16.0) in cands and (24.0, 16.0) not in cands


def test_autotuner_shortlist_for_confirmation():
    res = [
        {"warp_max_rows": 160, "lane_max_rows": 0, "time_ms": 5.0, "rel_diff": 0.0},
        {"warp_max_rows": 320, "lane_max_rows": 24, "time_ms": 4.0, "rel_diff": 1e-3},  # inaccurate
        {"warp_max_rows": 640, "lane_max_rows": 0, "time_ms": 6.0, "rel_diff": 0.0},
        {"warp_max_rows": 8192, "lane_max_rows": 0, "time_ms": 9.0, "rel_diff": 0.0},
    ]
    assert autotune.shortlist(res, 1e-5, n=2) == [(160, 0), (640, 0), (8192, 0)]
    assert autotune.shortlist(res, 1e-5, n=3) == [(160, 0), (640, 0), (8192, 0)]
