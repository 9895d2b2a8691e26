"""GPU parity of the per-distance-class regular rules (bem_set_quadrature)
against the FP64 oracle with the same classes.

Workload: Laplace SLP and DLP, P0, icosphere L3 (1,280 triangles), leaf 32,
eta 1.2, thresholds rho3 = 5, rho1 = 7 (all three classes occur).  Bars:
  class of every block: identical to the oracle's (integer decision, FP64 on
  both sides);
  admissible block vs the oracle's dense block of its own rule: the ACA
  yardstick as in test_gpu_parity (the oracle's ACA on the block and on copies
  perturbed at the mixed path's rounding level), and for blocks whose rule
  moves the entries by more than 5x that bar the result is nearer its own
  rule's block than the 6-point one (the class was applied);
  product vs the oracle H-matrix with the same classes: <= 2 aca_eps;
  FP64 and Helmholtz assemblies keep the 6-point rule: bitwise the products of
  a tree built without classes.
"""
import numpy as np
import pytest

import oracle
from paper_1711_01897_gb300 import bem, meshes

pytestmark = pytest.mark.gpu

RHO3, RHO1 = 5.0, 7.0
POINTS = {oracle.RULE6: 6, oracle.RULE3: 3, oracle.RULE1: 1}


def relf(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def aca_yardstick(truth, eps, draws=4, seed=0):
    """Largest error of the oracle's ACA on the block and on copies perturbed
    at the mixed path's rounding level (1e-7): the stopping rule is heuristic,
    and a near-tie decided by the last bit changes the rank."""
    rng = np.random.default_rng(seed)
    errs = []
    for d in range(draws + 1):
        B = truth if d == 0 else truth * (1 + 1e-7 * rng.normal(size=truth.shape))
        U, Vv = oracle.aca_dense(B, eps)
        errs.append(relf((U @ Vv.T).real, truth))
    return max(errs)


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    torch.cuda.init()
    return bem.load()


@pytest.fixture
def classes(lib):
    """Thresholds set for the trees built inside the test, restored after."""
    saved = bem.bem_get_quadrature()
    bem.bem_set_quadrature(RHO3, RHO1)
    yield
    bem.bem_set_quadrature(saved["rho3"], saved["rho1"])


@pytest.fixture(scope="module")
def l3():
    return meshes.icosphere_level(3)


def _tree(V, T):
    return bem.HMatrix(bem.Mesh(V, T), 32, 1.2)


def test_block_rules_match_oracle(l3, classes):
    V, T = l3
    h = _tree(V, T)
    got = h.block_rules()
    ct = oracle.cluster_tree(V, T, 32)
    bt = oracle.block_tree(ct, 1.2)
    blocks = oracle.block_list(ct, bt)
    want = oracle.block_rules(V, T, ct, bt, blocks, RHO3, RHO1)
    gb, _ = h.blocks()
    assert np.array_equal(gb, blocks)
    exp = np.array([POINTS[c] if a else 0 for c, a in zip(want, blocks[:, 4])])
    assert np.array_equal(got, exp)
    st = h.stats()
    assert st["n_blocks_rule3"] == int(np.sum(got == 3)) > 0
    assert st["n_blocks_rule1"] == int(np.sum(got == 1)) > 0
    assert (st["rho3"], st["rho1"]) == (RHO3, RHO1)


@pytest.mark.parametrize("op", [bem.SLP, bem.DLP])
def test_blocks_and_product_against_oracle(l3, classes, op):
    V, T = l3
    eps = 1e-5
    h = _tree(V, T)
    h.assemble(op, 0.0, eps, bem.MIXED)
    ohm = oracle.hmat_assemble(V, T, op, 0.0, 32, 1.2, eps, rho3=RHO3, rho1=RHO1)
    blocks, perm = h.blocks()
    rules = h.block_rules()
    applied = 0
    for b, (tb, te, sb, se, adm) in enumerate(blocks):
        if not adm:
            continue
        code = int(ohm.rules[b])
        assert rules[b] == POINTS[code]
        rows, cols = perm[tb:te], perm[sb:se]
        own = oracle.entries(V, T, op, 0.0, rows, cols, regular_order=code).real
        got, rank = h.block_dense(b, (te - tb, se - sb))
        bar = 2 * aca_yardstick(own, eps, seed=b) + 1e-5
        assert relf(got, own) <= bar, (b, code, rank)
        if code != oracle.RULE6:
            ref6 = oracle.entries(V, T, op, 0.0, rows, cols).real
            if relf(own, ref6) > 5 * bar:
                assert relf(got, own) < relf(got, ref6), b
                applied += 1
    assert applied > 0
    x = np.random.default_rng(11).normal(size=T.shape[0])
    y = h.matvec(x)
    assert relf(y, ohm.matvec(x).real) <= 2 * eps


def test_fp64_and_helmholtz_keep_the_six_point_rule(l3, lib):
    V, T = l3
    x = np.random.default_rng(2).normal(size=T.shape[0])
    out = {}
    for with_classes in (False, True):
        saved = bem.bem_get_quadrature()
        bem.bem_set_quadrature(RHO3 if with_classes else 0.0, RHO1 if with_classes else 0.0)
        try:
            h = _tree(V, T)
        finally:
            bem.bem_set_quadrature(saved["rho3"], saved["rho1"])
        assert (h.stats()["n_blocks_rule3"] > 0) == with_classes
        h.assemble(bem.SLP, 0.0, 1e-5, bem.FP64)
        y64 = h.matvec(x)
        h.assemble(bem.SLP, 2.0, 1e-5, bem.MIXED)
        yk = h.matvec(x + 0j)
        out[with_classes] = (y64, yk)
    assert np.array_equal(out[False][0], out[True][0])
    assert np.array_equal(out[False][1], out[True][1])
