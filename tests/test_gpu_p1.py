"""GPU parity of the piecewise linear spaces: DP1 local matrices
(bem_entries_dp1), DP1 H-matrices, continuous P1 operators (C^T A_DP1 C) and
the hypersingular operator applied through the DP1 single layer (Eq. (9)),
all through the C ABI, against the FP64 oracle (whose hypersingular operator
is assembled directly from the weak form, Eq. (4)).

Tolerances as for P0: FP64 <= 1e-6 (expected ~1e-13), mixed <= 1e-5
(expected ~1e-7) relative Frobenius per entry set; touching pairs are FP64
in both modes (elementwise <= 1e-11 relative to the set); H-matrix products
<= 2 aca_eps relative 2-norm.
"""
import numpy as np
import pytest

import oracle
from paper_1711_01897_gb300 import bem, meshes

pytestmark = pytest.mark.gpu

TOL = {bem.FP64: 1e-6, bem.MIXED: 1e-5}


def relf(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    torch.cuda.init()
    return bem.load()


@pytest.fixture(scope="module")
def l2j():
    V, T = meshes.icosphere_level(2)
    return meshes.jitter(V, T, 0.05, 1234), T


@pytest.fixture(scope="module")
def l2j_mesh(lib, l2j):
    return bem.Mesh(*l2j)


def _touching(T, seeds):
    ids = set()
    for s in seeds:
        ids |= set(np.nonzero(np.isin(T, T[s]).any(axis=1))[0].tolist())
    return np.array(sorted(ids), dtype=np.int32)


@pytest.mark.parametrize("op", [bem.SLP, bem.DLP, bem.ADLP])
@pytest.mark.parametrize("k", [0.0, 2.0])
@pytest.mark.parametrize("prec", [bem.FP64, bem.MIXED])
def test_dp1_entries_against_oracle(l2j, l2j_mesh, op, k, prec):
    V, T = l2j
    rng = np.random.default_rng(7 + op + 10 * int(k) + 100 * prec)
    test = np.concatenate([_touching(T, [3, 200]), rng.choice(T.shape[0], 17, replace=False)])
    trial = np.concatenate([_touching(T, [3, 201]), rng.choice(T.shape[0], 41, replace=False)])
    test, trial = test.astype(np.int32), trial.astype(np.int32)
    got = l2j_mesh.entries_dp1(op, k, prec, test, trial)
    ref = oracle.entries_dp1(V, T, op, k, test, trial)
    if k == 0:
        ref = ref.real
    assert got.shape == (3 * test.size, 3 * trial.size)
    err = relf(got, ref)
    assert err <= TOL[prec], err
    if prec == bem.FP64:
        assert err < 1e-11, err
    # touching pairs: FP64 Sauter-Schwab in both modes, against the oracle's
    # rule (the 4-point rule is exact in xi for the Laplace integrands, so the
    # two agree to rounding)
    touch = np.array([[np.isin(T[a], T[b]).any() for b in trial] for a in test])
    mask = np.kron(touch, np.ones((3, 3), dtype=bool))
    scale = np.abs(ref).max()
    assert np.abs(got[mask] - ref[mask]).max() <= 1e-11 * scale


def test_dp1_entries_ragged_and_errors(l2j, l2j_mesh):
    V, T = l2j
    test = np.arange(0, T.shape[0], 7, dtype=np.int32)       # 46 rows
    trial = np.arange(1, T.shape[0], 3, dtype=np.int32)      # 107 columns
    got = l2j_mesh.entries_dp1(bem.SLP, 0.0, bem.MIXED, test, trial)
    ref = oracle.entries_dp1(V, T, bem.SLP, 0.0, test, trial).real
    assert relf(got, ref) <= 1e-5
    bad = np.array([0, T.shape[0]], dtype=np.int32)
    with pytest.raises(bem.BemError):
        l2j_mesh.entries_dp1(bem.SLP, 0.0, bem.FP64, bad, trial)
    empty = l2j_mesh.entries_dp1(bem.SLP, 0.0, bem.FP64, np.zeros(0, np.int32), trial)
    assert empty.shape == (0, 3 * trial.size)


@pytest.mark.parametrize("op", [bem.SLP, bem.DLP])
@pytest.mark.parametrize("prec", [bem.FP64, bem.MIXED])
def test_dp1_hmatrix_blocks_and_product(l2j, l2j_mesh, op, prec):
    V, T = l2j
    eps = 1e-6
    h = bem.HMatrix(l2j_mesh, 16, 1.2, space=bem.DP1)
    assert h.n == 3 * T.shape[0]
    h.assemble(op, 0.0, eps, prec)
    A = oracle.dense_matrix_dp1(V, T, op, 0.0).real
    blocks, perm = h.blocks()
    dperm = (3 * perm[:, None] + np.arange(3)[None, :]).reshape(-1)
    Ap = A[np.ix_(dperm, dperm)]
    n_far = 0
    for b, (tb, te, sb, se, adm) in enumerate(blocks):
        ref = Ap[tb:te, sb:se]
        got, rank = h.block_dense(b, (te - tb, se - sb))
        err = relf(got, ref)
        if adm:
            n_far += 1
            U, Vv = oracle.aca_dense(ref, eps)
            assert err <= 2 * relf((U @ Vv.T).real, ref) + 10 * eps + TOL[prec], (b, err)
        else:
            assert err <= TOL[prec], (b, err)
    assert n_far > 0
    x = np.random.default_rng(3).normal(size=h.n)
    y = h.matvec(x)
    assert relf(y, A @ x) <= 2 * eps + TOL[prec]
    st = h.stats()
    assert st["space"] == bem.DP1 and st["n_dofs"] == h.n
    h.close()


@pytest.mark.parametrize("op", [bem.SLP, bem.DLP, bem.ADLP])
@pytest.mark.parametrize("k", [0.0, 2.0])
def test_p1_products_against_oracle(l2j, l2j_mesh, op, k):
    V, T = l2j
    eps = 1e-5
    h = bem.HMatrix(l2j_mesh, 16, 1.2, space=bem.P1)
    assert h.n == V.shape[0]
    h.assemble(op, k, eps, bem.MIXED)
    A = oracle.dense_matrix_p1(V, T, op, k)
    rng = np.random.default_rng(11)
    x = rng.normal(size=h.n) + (1j * rng.normal(size=h.n) if k else 0)
    y = h.matvec(x)
    ref = A @ x if k else (A.real @ x)
    assert relf(y, ref) <= 2 * eps, relf(y, ref)
    h.close()


@pytest.mark.parametrize("k", [0.0, 2.0])
@pytest.mark.parametrize("prec", [bem.FP64, bem.MIXED])
def test_hypersingular_against_weak_form(l2j, l2j_mesh, k, prec):
    V, T = l2j
    eps = 1e-6
    h = bem.HMatrix(l2j_mesh, 16, 1.2, space=bem.P1)
    h.assemble(bem.HYPS, k, eps, prec)
    D = oracle.hypersingular_p1(V, T, k)
    rng = np.random.default_rng(5)
    x = rng.normal(size=h.n) + (1j * rng.normal(size=h.n) if k else 0)
    y = h.matvec(x)
    ref = D @ x if k else (D.real @ x)
    # the curl part's products cancel (D 1 = 0): the error is relative to the
    # size of the terms, so compare against |D| |x|
    err = np.linalg.norm(y - ref) / (np.linalg.norm(D, 2) * np.linalg.norm(x))
    assert err <= 2 * eps + TOL[prec], err
    if k == 0:
        one = h.matvec(np.ones(h.n))
        assert np.abs(one).max() <= 1e-10 * np.abs(D).max()


def test_p1_batch_and_device_vectors(l2j, l2j_mesh):
    import torch
    V, T = l2j
    h = bem.HMatrix(l2j_mesh, 16, 1.2, space=bem.P1)
    h.assemble(bem.SLP, 0.0, 1e-6, bem.FP64)
    rng = np.random.default_rng(2)
    X = rng.normal(size=(2, h.n))
    Y = h.matvec(X.copy(), np.zeros_like(X), batch=2)
    xd = torch.from_numpy(X).cuda()
    yd = torch.zeros_like(xd)
    bem.hmat_matvec(h.handle, xd, yd, 2)
    torch.cuda.synchronize()
    assert np.abs(yd.cpu().numpy() - Y).max() <= 1e-14 * np.abs(Y).max()
    A = oracle.dense_matrix_p1(V, T, bem.SLP, 0.0).real
    assert relf(Y[1], A @ X[1]) <= 2e-6
    with pytest.raises(bem.BemError):
        bem.HMatrix(l2j_mesh, 16, 1.2, space=bem.DP1).assemble(bem.HYPS, 0.0, 1e-4, bem.FP64)


def test_p1_helmholtz_sampled_rows_l4(lib):
    """A larger case: jittered L4 sphere (2,562 vertices), Helmholtz k = 3,
    single layer and hypersingular operator in mixed precision, against exact
    rows of the oracle's P1 matrices."""
    V, T = meshes.icosphere_level(4)
    V = meshes.jitter(V, T, 0.05, 77)
    mesh = bem.Mesh(V, T)
    k, eps = 3.0, 1e-5
    rng = np.random.default_rng(9)
    x = rng.normal(size=V.shape[0]) + 1j * rng.normal(size=V.shape[0])
    rows = np.sort(rng.choice(V.shape[0], 6, replace=False))
    for op in (bem.SLP, bem.HYPS):
        h = bem.HMatrix(mesh, 32, 1.2, space=bem.P1)
        h.assemble(op, k, eps, bem.MIXED)
        y = h.matvec(x)
        if op == bem.SLP:
            R = oracle.p1_rows(V, T, oracle.SLP, k, rows)
            scale = np.linalg.norm(R @ x)
        else:
            R = oracle.hypersingular_p1_rows(V, T, k, rows)
            scale = np.linalg.norm(np.abs(R) @ np.abs(x))
        err = np.linalg.norm(y[rows] - R @ x) / scale
        assert err <= 2 * eps, (op, err)
        h.close()
    mesh.close()


def test_p1_icosahedron_all_near_field(lib):
    """20 triangles: the H-matrix is (almost) all dense blocks."""
    V, T = meshes.icosphere(1)
    mesh = bem.Mesh(V, T)
    for op, k in ((bem.SLP, 0.0), (bem.DLP, 1.0), (bem.HYPS, 0.0), (bem.HYPS, 1.0)):
        h = bem.HMatrix(mesh, 4, 1.2, space=bem.P1)
        h.assemble(op, k, 1e-12, bem.FP64)
        x = np.arange(V.shape[0], dtype=np.float64) - 5.0
        if k:
            x = x + 0.5j
        y = h.matvec(x)
        A = oracle.hypersingular_p1(V, T, k) if op == bem.HYPS else oracle.dense_matrix_p1(V, T, op, k)
        ref = A @ x if k else A.real @ x
        assert np.linalg.norm(y - ref) <= 1e-9 * np.linalg.norm(np.abs(A) @ np.abs(x)), op
        h.close()
    mesh.close()


def test_dp1_helmholtz_hmatrix_blocks(l2j, l2j_mesh):
    V, T = l2j
    k, eps = 2.0, 1e-6
    h = bem.HMatrix(l2j_mesh, 16, 1.2, space=bem.DP1)
    h.assemble(bem.SLP, k, eps, bem.MIXED)
    A = oracle.dense_matrix_dp1(V, T, bem.SLP, k)
    blocks, perm = h.blocks()
    dperm = (3 * perm[:, None] + np.arange(3)[None, :]).reshape(-1)
    Ap = A[np.ix_(dperm, dperm)]
    for b, (tb, te, sb, se, adm) in enumerate(blocks):
        ref = Ap[tb:te, sb:se]
        got, _ = h.block_dense(b, (te - tb, se - sb))
        err = relf(got, ref)
        if adm:
            U, Vv = oracle.aca_dense(ref, eps)
            assert err <= 2 * relf(U @ Vv.T, ref) + 10 * eps + TOL[bem.MIXED], (b, err)
        else:
            assert err <= TOL[bem.MIXED], (b, err)
    x = np.random.default_rng(4).normal(size=h.n) * (1 + 0.3j)
    assert relf(h.matvec(x), A @ x) <= 2 * eps + TOL[bem.MIXED]
    h.close()


def test_p1_graph_replay_matches_eager(l2j, l2j_mesh):
    """The DP1 assembly sequence captured into a CUDA graph and replayed gives
    the eager result bit for bit (hypersingular, Helmholtz, mixed)."""
    V, T = l2j
    saved = bem.bem_get_tuning()
    x = np.random.default_rng(8).normal(size=V.shape[0]) + 0.25j
    try:
        bem.bem_set_tuning(saved["warp_max_rows"], saved["lane_max_rows"], 0)
        h0 = bem.HMatrix(l2j_mesh, 16, 1.2, space=bem.P1)
        h0.assemble(bem.HYPS, 1.5, 1e-5, bem.MIXED)
        y0 = h0.matvec(x)
        bem.bem_set_tuning(saved["warp_max_rows"], saved["lane_max_rows"], 1)
        h = bem.HMatrix(l2j_mesh, 16, 1.2, space=bem.P1)
        for _ in range(3):          # eager, capture + launch, replay
            h.assemble(bem.HYPS, 1.5, 1e-5, bem.MIXED)
            assert np.array_equal(h.matvec(x), y0)
        h.close()
        h0.close()
    finally:
        bem.bem_set_tuning(saved["warp_max_rows"], saved["lane_max_rows"], saved["use_graphs"])
