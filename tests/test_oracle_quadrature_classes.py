"""Pins of the oracle's per-distance-class regular rules (the 3-point degree-2
rule and the centroid rule beside the paper's 6-point degree-4 rule, Sec.
3.2.1) and of the class of each admissible block.

Fixed by mathematics, not by the oracle itself: polynomial exactness of each
rule on the reference triangle, the position of the points, the convergence
rate of each rule's error with the separation of a pair (an independent
high-order conical rule is the reference), and the class of every block
recomputed from the boxes and edge lengths with numpy.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1711_01897_gb300 import meshes


def _mean_monomial(i, j):
    # normalised integral of s^i t^j over {s, t >= 0, s + t <= 1}
    return 2.0 * math.factorial(i) * math.factorial(j) / math.factorial(i + j + 2)


@pytest.mark.parametrize("rule, degree", [("deg2", 2), ("deg1", 1), ("deg4", 4)])
def test_rule_polynomial_exactness(rule, degree):
    s, t, w = {"deg2": oracle.triangle_rule_deg2, "deg1": oracle.triangle_rule_deg1,
               "deg4": oracle.triangle_rule_deg4}[rule]()
    assert abs(w.sum() - 1.0) < 1e-15
    for tot in range(degree + 2):
        errs = [abs(np.sum(w * s**i * t**(tot - i)) - _mean_monomial(i, tot - i))
                for i in range(tot + 1)]
        if tot <= degree:
            assert max(errs) < 1e-14, (rule, tot, errs)
        else:
            assert max(errs) > 1e-4, (rule, tot, errs)  # the degree is exact, not higher


def test_rule_deg2_points_inside():
    """The interior degree-2 rule (barycentric 2/3, 1/6, 1/6), not the other
    root of its moment equation (the edge midpoints)."""
    s, t, w = oracle.triangle_rule_deg2()
    bary = np.stack([1.0 - s - t, s, t], axis=1)
    assert np.allclose(np.sort(bary, axis=1), [[1 / 6, 1 / 6, 2 / 3]] * 3, atol=1e-15)
    assert np.allclose(w, 1 / 3)
    s1, t1, w1 = oracle.triangle_rule_deg1()
    assert np.allclose([s1[0], t1[0], w1[0]], [1 / 3, 1 / 3, 1.0])


A9 = np.array([[0, 0, 0], [1, 0.1, 0], [0.2, 0.9, 0.1]], float)
B9 = np.array([[0, 0, 0], [0.8, -0.2, 0.3], [0.1, 0.7, -0.2]], float)
IA, IB = np.array([0, 1, 2], np.int32), np.array([3, 4, 5], np.int32)


def _rel_err(op, code, d):
    B = B9 + np.array([d, 0.3 * d, 0.2 * d])
    ref = oracle.pair_entry(A9.ravel(), B.ravel(), IA, IB, op, 0.0, regular_order=20)
    v = oracle.pair_entry(A9.ravel(), B.ravel(), IA, IB, op, 0.0, regular_order=code)
    return abs(v - ref) / abs(ref)


@pytest.mark.parametrize("op", [oracle.SLP, oracle.DLP])
@pytest.mark.parametrize("code, lo, hi", [(oracle.RULE3, 2.7, 3.6), (oracle.RULE1, 1.8, 2.4),
                                          (oracle.RULE6, 5.0, 7.0)])
def test_rule_error_decays_with_separation(op, code, lo, hi):
    """Relative error of a well-separated Laplace pair against a 20 x 20
    conical rule: O((h/d)^3) for the degree-2 rule (its first inexact Taylor
    terms are cubic), O((h/d)^2) for the centroid rule, O((h/d)^6) for the
    degree-4 rule (odd terms cancel by symmetry)."""
    e16, e32 = _rel_err(op, code, 16.0), _rel_err(op, code, 32.0)
    rate = math.log2(e16 / e32)
    assert lo <= rate <= hi, (op, code, rate, e16, e32)


@pytest.fixture(scope="module")
def l3():
    return meshes.icosphere_level(3)


def test_block_rules_brute_force(l3):
    V, T = l3
    rho3, rho1 = 5.0, 7.0
    ct = oracle.cluster_tree(V, T, 32)
    bt = oracle.block_tree(ct, 1.2)
    blocks = oracle.block_list(ct, bt)
    rules = oracle.block_rules(V, T, ct, bt, blocks, rho3, rho1)
    edge = np.sqrt(np.max([np.sum((V[T[:, a]] - V[T[:, (a + 1) % 3]]) ** 2, axis=1)
                           for a in range(3)], axis=0))
    counts = {}
    for b, (tb, te, sb, se, adm) in enumerate(blocks):
        if not adm:
            assert rules[b] == oracle.RULE6
            continue
        bx_t, bx_s = ct.box[bt.tau[b]], ct.box[bt.sigma[b]]
        gap = np.maximum(np.maximum(bx_s[:3] - bx_t[3:], bx_t[:3] - bx_s[3:]), 0.0)
        dist = float(np.sqrt(np.sum(gap ** 2)))
        h = max(edge[ct.perm[tb:te]].max(), edge[ct.perm[sb:se]].max())
        want = oracle.RULE1 if dist >= rho1 * h else (oracle.RULE3 if dist >= rho3 * h else oracle.RULE6)
        assert rules[b] == want, (b, dist / h)
        counts[want] = counts.get(want, 0) + 1
    assert all(counts.get(c, 0) > 0 for c in (oracle.RULE6, oracle.RULE3, oracle.RULE1)), counts
    assert np.all(oracle.block_rules(V, T, ct, bt, blocks, 0.0, 0.0) == oracle.RULE6)


@pytest.mark.parametrize("op", [oracle.SLP, oracle.DLP])
def test_hmatrix_blocks_use_their_class_rule(l3, op):
    """Each admissible block of the oracle H-matrix approximates the dense
    block of its own rule (to the ACA tolerance), and the rule changes the
    block by no more than its error bound for that separation."""
    V, T = l3
    eps = 1e-6
    hm = oracle.hmat_assemble(V, T, op, 0.0, 32, 1.2, eps, rho3=5.0, rho1=7.0)
    rng = np.random.default_rng(5)
    adm = [b for b in range(hm.blocks.shape[0]) if hm.blocks[b, 4]]
    seen = set()
    for b in rng.permutation(adm):
        code = int(hm.rules[b])
        if code in seen and len(seen) < 3:
            continue
        seen.add(code)
        tb, te, sb, se, _ = hm.blocks[b]
        rows, cols = hm.perm[tb:te], hm.perm[sb:se]
        own = oracle.entries(V, T, op, 0.0, rows, cols, regular_order=code).real
        ref6 = oracle.entries(V, T, op, 0.0, rows, cols).real
        got = hm.block_dense(b).real
        assert np.linalg.norm(got - own) <= 10 * eps * np.linalg.norm(own), (b, code)
        d6 = np.linalg.norm(own - ref6) / np.linalg.norm(ref6)
        if code == oracle.RULE6:
            assert d6 == 0.0
        else:
            assert 0.0 < d6 < 1e-2, (b, code, d6)
        if len(seen) == 3:
            break
    assert seen == {oracle.RULE6, oracle.RULE3, oracle.RULE1}


def test_classes_are_p0_only(l3):
    """The distance classes are defined for P0 (the library's DP1 and P1
    handles keep the 6-point rule); the oracle refuses them elsewhere."""
    V, T = l3
    with pytest.raises(ValueError):
        oracle.hmat_assemble(V, T, oracle.SLP, 0.0, 32, 1.2, 1e-4, space=oracle.DP1, rho3=5.0)
    hm = oracle.hmat_assemble(V, T, oracle.SLP, 0.0, 32, 1.2, 1e-4, block_ids=[0])
    assert np.all(hm.rules == oracle.RULE6)
