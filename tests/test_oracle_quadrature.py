"""Pins of the oracle's quadrature rules and Sauter-Schwab maps against
exact polynomial integrals (Sec. 3.2.1 six-point degree-4 rule; Sec. 3.2.3
singular scheme)."""
from math import factorial

import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 8, 12])
def test_gauss_legendre_exact_to_degree_2n_minus_1(n):
    x, w = oracle.gauss_legendre01(n)
    assert np.all(np.diff(x) > 0) and np.all((x > 0) & (x < 1)) and np.all(w > 0)
    for d in range(2 * n):
        assert abs(np.sum(w * x ** d) - 1.0 / (d + 1)) < 1e-14
    # one degree higher is not exact (visible for small n)
    if n <= 5:
        assert abs(np.sum(w * x ** (2 * n)) - 1.0 / (2 * n + 1)) > 1e-9


def _tri_moment(a, b):
    """Normalised integral of s^a t^b over the unit right triangle."""
    return 2.0 * factorial(a) * factorial(b) / factorial(a + b + 2)


def test_six_point_rule_is_degree_four():
    s, t, w = oracle.triangle_rule_deg4()
    assert s.size == 6 and np.all(w > 0) and abs(w.sum() - 1) < 1e-15
    assert np.all((s > 0) & (t > 0) & (s + t < 1))
    for a in range(5):
        for b in range(5 - a):
            assert abs(np.sum(w * s ** a * t ** b) - _tri_moment(a, b)) < 1e-15
    worst = max(abs(np.sum(w * s ** a * t ** (5 - a)) - _tri_moment(a, 5 - a)) for a in range(6))
    assert worst > 1e-6
    # symmetric: two orbits of three points
    assert np.unique(np.round(w, 14)).size == 2


@pytest.mark.parametrize("n", [2, 4, 7])
def test_conical_rule_exactness(n):
    s, t, w = oracle.triangle_rule_conical(n)
    for a in range(2 * n - 1):
        for b in range(2 * n - 1 - a):
            assert abs(np.sum(w * s ** a * t ** b) - _tri_moment(a, b)) < 1e-14


def _that_moment(a, b):
    """Integral of x1^a x2^b over T^ = {0 <= x2 <= x1 <= 1}."""
    return 1.0 / ((b + 1) * (a + b + 2))


@pytest.mark.parametrize("ncase", [1, 2, 3])
def test_sauter_schwab_maps_cover_t_times_t(ncase):
    """Regions and Jacobians reproduce every moment of T^ x T^ (degree <= 3
    is integrated exactly by 4 GL points per axis after the maps)."""
    for a in range(4):
        for b in range(4 - a):
            for c in range(4 - a - b):
                for d in range(4 - a - b - c):
                    exact = _that_moment(a, b) * _that_moment(c, d)
                    got = oracle.ss_moment(ncase, 4, a, b, c, d)
                    assert abs(got - exact) <= 1e-13 * exact, (ncase, a, b, c, d)
