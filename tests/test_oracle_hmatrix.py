"""Pins of the oracle's block partition, ACA and H-matrix product
(Sec. 2.1, Eq. (6)-(7), Algorithm ACA, Algorithm "H-Matrix Assembly")."""
import numpy as np
import pytest

import oracle
from paper_1711_01897_gb300 import meshes


@pytest.fixture(scope="module")
def l3():
    return meshes.icosphere_level(3)


def test_cluster_tree_invariants(l3):
    V, T = l3
    ct = oracle.cluster_tree(V, T, 32)
    n = T.shape[0]
    assert np.array_equal(np.sort(ct.perm), np.arange(n))
    assert ct.begin[0] == 0 and ct.end[0] == n
    for c in range(ct.n_clusters):
        b, e = ct.begin[c], ct.end[c]
        if ct.left[c] < 0:
            assert e - b <= 32
        else:
            l, r = ct.left[c], ct.right[c]
            assert ct.begin[l] == b and ct.end[l] == ct.begin[r] and ct.end[r] == e
            assert ct.end[l] - ct.begin[l] == (e - b) // 2
            # the split is at the median along the longest axis
            box = ct.box[c]
            ax = int(np.argmax(box[3:] - box[:3]))
            cen = V[T[ct.perm]].mean(axis=1)[:, ax]
            assert cen[b:ct.end[l]].max() <= cen[ct.begin[r]:e].min() + 1e-15
        pts = V[T[ct.perm[b:e]]].reshape(-1, 3)
        assert np.all(pts >= ct.box[c, :3]) and np.all(pts <= ct.box[c, 3:])
        assert np.allclose(pts.min(0), ct.box[c, :3]) and np.allclose(pts.max(0), ct.box[c, 3:])


def test_block_tree_tiles_index_square_once(l3):
    V, T = l3
    ct = oracle.cluster_tree(V, T, 32)
    bt = oracle.block_tree(ct, 1.2)
    blocks = oracle.block_list(ct, bt)
    n = T.shape[0]
    cover = np.zeros((n, n), dtype=np.int32)
    for tb, te, sb, se, _ in blocks:
        cover[tb:te, sb:se] += 1
    assert np.all(cover == 1)
    assert blocks[:, 4].sum() > 0 and (1 - blocks[:, 4]).sum() > 0
    perm = ct.perm
    for tb, te, sb, se, adm in blocks:
        if adm:
            # admissible clusters share no vertex, so no singular pair
            assert not np.intersect1d(T[perm[tb:te]].ravel(), T[perm[sb:se]].ravel()).size
    # every pair of triangles sharing a vertex lies in a near block
    near = np.zeros((n, n), dtype=bool)
    for tb, te, sb, se, adm in blocks:
        if not adm:
            near[tb:te, sb:se] = True
    inv = np.empty(n, dtype=np.int64)
    inv[perm] = np.arange(n)
    shared = (T[:, None, :, None] == T[None, :, None, :]).any(axis=(2, 3))
    i, j = np.nonzero(shared)
    assert np.all(near[inv[i], inv[j]])


def test_admissibility_condition(l3):
    V, T = l3
    ct = oracle.cluster_tree(V, T, 32)
    bt = oracle.block_tree(ct, 1.2)
    for t, s, adm in zip(bt.tau, bt.sigma, bt.adm):
        bx, by = ct.box[t], ct.box[s]
        diam = lambda b: np.linalg.norm(b[3:] - b[:3])
        gap = np.maximum(0, np.maximum(by[:3] - bx[3:], bx[:3] - by[3:]))
        dist = np.linalg.norm(gap)
        expect = dist > 0 and min(diam(bx), diam(by)) <= 1.2 * dist
        assert bool(adm) == bool(expect)


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("r", [1, 3, 7])
def test_aca_recovers_exact_rank(cplx, r):
    rng = np.random.default_rng(r + 10 * cplx)
    m, n = 40, 33
    X = rng.normal(size=(m, r)) + (1j * rng.normal(size=(m, r)) if cplx else 0)
    Y = rng.normal(size=(n, r)) + (1j * rng.normal(size=(n, r)) if cplx else 0)
    A = X @ Y.T
    U, Vv = oracle.aca_dense(A, 1e-12)
    assert U.shape[1] == r
    assert np.linalg.norm(U @ Vv.T - A) <= 1e-11 * np.linalg.norm(A)


def test_aca_zero_block_and_pivot_rule():
    A = np.zeros((5, 4))
    U, Vv = oracle.aca_dense(A, 1e-6)
    assert U.shape[1] == 0
    # rank-1 with a vanishing first row: the first row is skipped
    A = np.outer([0, 2.0, 1.0], [1.0, -3.0, 0.5])
    U, Vv = oracle.aca_dense(A, 1e-12)
    assert U.shape[1] == 1 and np.allclose(U @ Vv.T, A)
    # column pivot is the largest |entry| of the row (Eq. (7)): v is scaled so
    # that v[j_k] = 1
    assert np.isclose(Vv[1, 0], 1.0)


def _rows_reproduced(A, kcap):
    U, Vv = oracle.aca_dense(A, 1e-14, kcap=kcap)
    R = U @ Vv.T
    return [i for i in range(A.shape[0]) if np.allclose(R[i], A[i], rtol=0.0, atol=1e-13)]


@pytest.mark.parametrize("cplx", [False, True])
def test_aca_row_pivot_rule(cplx):
    """Reading R1 (the paper leaves the row pivot to Bebendorf's rule): the
    first row is row 0, the next the unused row with the largest modulus in
    the last column of the residual, the lowest index on ties.  A cross
    approximation reproduces its pivot rows exactly, so the rows that the
    rank-2 approximant reproduces name the two row pivots."""
    rng = np.random.default_rng(21 + cplx)
    m, n = 7, 6
    A = rng.uniform(0.1, 0.5, size=(m, n)) + (1j * rng.uniform(0.1, 0.5, size=(m, n)) if cplx else 0)
    # j1 = 3, the largest modulus of row 0; the first column of the residual
    # is column 3 itself, whose largest modulus outside row 0 is in row 4
    A[:, 3] = np.array([2.0, 0.2, 0.3, 0.1, 0.9, 0.4, 0.25]) * (1j if cplx else 1.0)
    assert _rows_reproduced(A, 2) == [0, 4]
    # a tie in modulus between rows 2 and 4: the lower index
    A[2, 3] = -A[4, 3]
    assert _rows_reproduced(A, 2) == [0, 2]
    # one step reproduces row 0 alone
    assert _rows_reproduced(A, 1) == [0]


@pytest.mark.parametrize("scale", [1.0, 1e10, 1e-10])
def test_aca_vanishing_row_threshold(scale):
    """Reading R2: a residual row counts as vanished when its largest modulus
    is at most 1e-14 of the largest pivot so far.  On diag(1, d) the second
    row's residual is (0, d): d = 1e-13 is a second pivot (rank 2), d = 1e-15
    vanishes (rank 1), whatever the matrix's scale."""
    for d, rank in ((1e-13, 2), (1e-15, 1)):
        A = scale * np.diag([1.0, d])
        U, Vv = oracle.aca_dense(A, 1e-30)
        assert U.shape[1] == rank, (d, scale)


@pytest.mark.parametrize("k", [0.0, 25.0])
def test_aca_stopping_rule(k):
    """Reading R3: ACA stops after the first step k with ||u_k|| ||v_k|| <=
    eps ||S_k||_F, where the oracle updates ||S_k||_F^2 incrementally (cross
    terms 2 Re <u_k, u_l><v_k, v_l>).  Here ||S_l||_F is recomputed from the
    returned factors by numpy for every prefix, so the run must stop at the
    first step that meets the criterion.  On this kernel matrix a missing
    cross term, a wrong sign of the cross terms or unconjugated inner
    products (k = 25) move the stopping step for some of the tolerances."""
    x = np.linspace(0.0, 1.0, 50)
    y = np.linspace(1.3, 2.2, 40)
    r = np.abs(x[:, None] - y[None, :])
    A = np.exp(1j * k * r) / r if k else 1.0 / r
    for eps in (1e-2, 1e-3, 1e-4, 1e-5, 1e-6, 1e-7, 1e-8):
        U, Vv = oracle.aca_dense(A, eps)
        rank = U.shape[1]
        assert 0 < rank < min(A.shape)

        def ratio(l):
            uv = np.linalg.norm(U[:, l - 1]) * np.linalg.norm(Vv[:, l - 1])
            return uv / (eps * np.linalg.norm(U[:, :l] @ Vv[:, :l].T))

        assert ratio(rank) <= 1.0 + 1e-9, (eps, rank)
        assert all(ratio(l) > 1.0 - 1e-9 for l in range(1, rank)), (eps, rank)


def test_aca_error_decreases_with_eps():
    """Smooth kernel matrix: the ACA error tracks the requested accuracy."""
    x = np.linspace(0, 1, 60)
    y = np.linspace(3, 4, 50)
    A = 1.0 / np.abs(x[:, None] - y[None, :])
    errs = []
    for eps in (1e-3, 1e-6, 1e-9):
        U, Vv = oracle.aca_dense(A, eps)
        errs.append(np.linalg.norm(U @ Vv.T - A) / np.linalg.norm(A))
        assert errs[-1] < 30 * eps
    assert errs[0] > errs[1] > errs[2]


@pytest.fixture(scope="module")
def hm_l3(l3):
    V, T = l3
    return oracle.hmat_assemble(V, T, oracle.SLP, 0.0, 32, 1.2, 1e-4)


@pytest.fixture(scope="module")
def dense_l3(l3):
    V, T = l3
    return oracle.dense_matrix(V, T, oracle.SLP, 0.0)


def test_hmatrix_blocks_against_dense(l3, hm_l3, dense_l3):
    A = dense_l3
    perm = hm_l3.perm
    Ap = A[np.ix_(perm, perm)]
    worst = 0.0
    for b, (tb, te, sb, se, adm) in enumerate(hm_l3.blocks):
        blk = Ap[tb:te, sb:se]
        got = hm_l3.block_dense(b)
        e = np.linalg.norm(got - blk) / np.linalg.norm(blk)
        if adm:
            worst = max(worst, e)
            assert hm_l3.ranks[b] < min(te - tb, se - sb)
        else:
            assert e < 1e-14
    assert worst < 30 * 1e-4, worst  # heuristic criterion (Sec. 2.1): error tracks eps, not bounded by it


def test_hmatrix_matvec_against_dense(l3, hm_l3, dense_l3):
    rng = np.random.default_rng(1)
    x = rng.normal(size=dense_l3.shape[0])
    y = hm_l3.matvec(x)
    yd = dense_l3 @ x
    assert np.linalg.norm(y - yd) / np.linalg.norm(yd) < 2e-4


def test_hmatrix_helmholtz_matvec(l3):
    V, T = meshes.icosphere_level(2)
    hm = oracle.hmat_assemble(V, T, oracle.SLP, 3.0, 16, 1.2, 1e-6)
    A = oracle.dense_matrix(V, T, oracle.SLP, 3.0)
    x = np.random.default_rng(2).normal(size=A.shape[0])
    assert any(hm.blocks[:, 4])
    assert np.linalg.norm(hm.matvec(x) - A @ x) / np.linalg.norm(A @ x) < 2e-6
