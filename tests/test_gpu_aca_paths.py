"""Every ACA work shape against the oracle (GPU, through the C ABI).

The persistent ACA kernel compresses an admissible block on one of three
work shapes, chosen per block by max(m, n) against the thresholds of
bem_set_tuning when the tree is built: a whole CTA, a warp (which may hold
several small blocks at once), or a single lane (32 blocks per warp).  The
default thresholds put every block of the benchmark meshes on warps, so these
tests force each shape in turn and compare every admissible block with the
oracle's dense block (Sec. 2.1, Algorithm ACA; the yardstick of
test_gpu_parity: the oracle ACA's own error on the exact and on rounding-level
perturbed copies of the block), and the product with the dense product
(<= 2 eps).  Laplace single and double layer and the complex Helmholtz single
layer (k = 2), both precisions.  Each case also asserts, from hmat_stats,
that the shapes it is meant to exercise really held blocks.

Also here: the FP64 reciprocal that scales every pivot (Eq. (7)), against
IEEE division over the whole exponent range its seed accepts and beyond."""
import numpy as np
import pytest

import oracle
from paper_1711_01897_gb300 import bem, meshes

pytestmark = pytest.mark.gpu

TOL = {bem.FP64: 1e-6, bem.MIXED: 1e-5, bem.MIXED_SP: 1e-5}
NOISE = {bem.FP64: 1e-15, bem.MIXED: 1e-7, bem.MIXED_SP: 1e-7}

# (warp_max_rows, lane_max_rows): the shapes each puts blocks on, for the L3
# mesh (blocks of 20 and 40 rows) and the L4 mesh (20 to 160 rows).  "warp"
# counts every block on warps; "quarter" (at most 40 rows, four blocks per
# warp on 8 lanes each) and "half" (at most 80 rows, two per warp) are parts
# of it, asserted where the mesh has such blocks
SHAPES = {
    "cta_warp": ((32, 0), {"cta", "warp", "quarter"}),
    "lane_warp": ((160, 24), {"lane", "warp", "quarter"}),
    "lane_only": ((8192, 64), {"lane"}),
    "cta_only": ((16, 0), {"cta"}),
    "default": ((8192, 0), {"warp", "quarter"}),
}
CASES = [(bem.SLP, 0.0), (bem.DLP, 0.0), (bem.SLP, 2.0)]


def relf(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def yardstick(truth, eps, prec, draws=3, seed=0):
    """Largest error of the oracle's ACA on the block and on copies
    perturbed at the rounding level of the path under test: the stopping
    rule is heuristic and a near-tie decided by the last bits can change the
    pivot sequence and the rank (several correct results, Sec. 2.1).  A
    block that fails the first bound gets a 64-draw sample before it is
    judged: some alternative sequences occur in about 1 % of draws (one L3
    double-layer block stops at rank 10 with error 1.7e-5 instead of rank 12
    with 1.5e-6 under 1e-7 noise)."""
    rng = np.random.default_rng(seed)
    errs = []
    for d in range(draws + 1):
        B = truth if d == 0 else truth * (1 + NOISE[prec] * rng.normal(size=truth.shape))
        U, Vv = oracle.aca_dense(B, eps)
        R = U @ Vv.T
        errs.append(relf(R.real if np.isrealobj(truth) else R, truth))
    return max(errs)


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    torch.cuda.init()
    return bem.load()


@pytest.fixture(scope="module")
def l3():
    V, T = meshes.icosphere_level(3)
    return meshes.jitter(V, T, 0.05, 31), T


@pytest.fixture(scope="module")
def l3_dense(l3):
    V, T = l3
    out = {}
    for op, k in CASES:
        A = oracle.dense_matrix(V, T, op, k)
        out[(op, k)] = A.real if k == 0 else A
    return out


_yard = {}


def _with_shape(shape, fn):
    saved = bem.bem_get_tuning()
    try:
        bem.bem_set_tuning(shape[0], shape[1], saved["use_graphs"])
        return fn()
    finally:
        bem.bem_set_tuning(saved["warp_max_rows"], saved["lane_max_rows"], saved["use_graphs"])


def _check_shapes(stats, want, l4=False):
    got = {"cta": stats["n_blocks_cta"], "warp": stats["n_blocks_warp"],
           "lane": stats["n_blocks_lane"], "half": stats["n_blocks_half_warp"],
           "quarter": stats["n_blocks_quarter_warp"]}
    assert got["cta"] + got["warp"] + got["lane"] == stats["n_blocks_far"]
    assert got["half"] + got["quarter"] <= got["warp"]
    want = set(want)
    if l4 and "warp" in want and "lane" not in want:
        want.add("half")          # the L4 mesh has 80-row blocks
    for s in ("cta", "warp", "lane", "quarter", "half"):
        if s in want:
            assert got[s] > 0, (s, got)
        elif s in ("cta", "warp", "lane"):
            assert got[s] == 0, (s, got)


@pytest.mark.parametrize("shape", sorted(SHAPES))
@pytest.mark.parametrize("case", CASES, ids=["slp", "dlp", "helmholtz_slp_k2"])
@pytest.mark.parametrize("prec", [bem.FP64, bem.MIXED, bem.MIXED_SP], ids=["fp64", "mixed", "mixed_sp"])
def test_every_block_every_shape_l3(lib, l3, l3_dense, shape, case, prec):
    """Jittered L3 (1,280 triangles), leaf 32, eta 1.2, eps 1e-5: every
    admissible block and the product."""
    V, T = l3
    op, k = case
    eps = 1e-5
    (wmax, lmax), want = SHAPES[shape]
    m = bem.Mesh(V, T)

    def build():
        h = bem.HMatrix(m, 32, 1.2)
        h.assemble(op, k, eps, prec)
        return h

    h = _with_shape((wmax, lmax), build)
    s = h.stats()
    _check_shapes(s, want)
    assert s["rank_capped_blocks"] == 0
    blocks, perm = h.blocks()
    A = l3_dense[case]
    Ap = A[np.ix_(perm, perm)]
    worst = 0.0
    for b, (tb, te, sb, se, adm) in enumerate(blocks):
        if not adm:
            continue
        got, rank = h.block_dense(b, (te - tb, se - sb))
        truth = Ap[tb:te, sb:se]
        key = (case, prec, b)
        if key not in _yard:
            _yard[key] = yardstick(truth, eps, prec, seed=b)
        e = relf(got, truth)
        worst = max(worst, e)
        if e > 2 * _yard[key] + TOL[prec]:
            # a rarer pivot sequence: widen the yardstick's sample
            _yard[key] = max(_yard[key], yardstick(truth, eps, prec, draws=64, seed=1000 + b))
        assert e <= 2 * _yard[key] + TOL[prec], (shape, b, e, _yard[key], rank)
        assert 0 < rank <= min(te - tb, se - sb)
    x = np.random.default_rng(5).normal(size=T.shape[0])
    if k != 0:
        x = x + 1j * np.random.default_rng(6).normal(size=T.shape[0])
    y = h.matvec(x)
    assert relf(y, A @ x) <= 2 * eps
    print(f"{shape} op={op} k={k} prec={prec}: worst block {worst:.2e}, "
          f"shapes cta/warp/lane {s['n_blocks_cta']}/{s['n_blocks_warp']}/{s['n_blocks_lane']}")


@pytest.mark.parametrize("prec", [bem.MIXED, bem.MIXED_SP], ids=["mixed", "mixed_sp"])
@pytest.mark.parametrize("shape", ["cta_warp", "lane_warp", "default"])
@pytest.mark.parametrize("case", CASES, ids=["slp", "dlp", "helmholtz_slp_k2"])
def test_sampled_blocks_every_shape_l4(lib, shape, case, prec):
    """Jittered L4 (5,120 triangles; blocks of 20 to 160 rows), both mixed
    modes: the largest blocks of every shape plus random ones against the
    oracle's dense blocks, and 24 exact rows of the product."""
    V, T = meshes.icosphere_level(4)
    V = meshes.jitter(V, T, 0.05, 41)
    op, k = case
    eps = 1e-5
    (wmax, lmax), want = SHAPES[shape]
    m = bem.Mesh(V, T)

    def build():
        h = bem.HMatrix(m, 32, 1.2)
        h.assemble(op, k, eps, prec)
        return h

    h = _with_shape((wmax, lmax), build)
    s = h.stats()
    _check_shapes(s, want, l4=shape != "cta_warp")
    blocks, perm = h.blocks()
    far = np.nonzero(blocks[:, 4] == 1)[0]
    mx = np.maximum(blocks[far, 1] - blocks[far, 0], blocks[far, 3] - blocks[far, 2])
    rng = np.random.default_rng(17 + op)
    pick = []
    # every shape's largest blocks and random ones: lane, quarter, half, warp, CTA
    cuts = sorted({0, lmax, min(40, wmax), min(80, wmax), wmax, 10 ** 9})
    for lo, hi in zip(cuts, cuts[1:]):
        cls = far[(mx > lo) & (mx <= hi)]
        if cls.size:
            order = cls[np.argsort(-mx[np.isin(far, cls)], kind="stable")]
            pick += list(order[:3]) + list(rng.choice(cls, min(6, cls.size), replace=False))
    for b in sorted(set(pick)):
        tb, te, sb, se, _ = blocks[b]
        truth = oracle.entries(V, T, op, k, perm[tb:te], perm[sb:se])
        if k == 0:
            truth = truth.real
        got, rank = h.block_dense(b, (te - tb, se - sb))
        e_or = yardstick(truth, eps, prec, draws=2, seed=int(b))
        if relf(got, truth) > 2 * e_or + TOL[prec]:
            e_or = max(e_or, yardstick(truth, eps, prec, draws=64, seed=1000 + int(b)))
        assert relf(got, truth) <= 2 * e_or + TOL[prec], (shape, b, relf(got, truth), e_or, rank)
    rows = rng.choice(T.shape[0], 24, replace=False).astype(np.int32)
    Arows = oracle.entries(V, T, op, k, rows, np.arange(T.shape[0], dtype=np.int32))
    if k == 0:
        Arows = Arows.real
    x = rng.normal(size=T.shape[0])
    y = h.matvec(x + 0j if k else x)
    assert relf(y[rows], Arows @ x) <= 2 * eps


def test_work_shapes_give_the_same_product(lib):
    """The shape decides which lanes evaluate an entry, not its value: in
    FP64 the products of every shape agree to rounding with the default's
    (ranks may differ only through near-ties decided by the last bit)."""
    V, T = meshes.icosphere_level(4)
    V = meshes.jitter(V, T, 0.05, 43)
    m = bem.Mesh(V, T)
    x = np.random.default_rng(9).normal(size=T.shape[0])
    ys = {}
    for name, (shape, _) in SHAPES.items():
        def run():
            h = bem.HMatrix(m, 32, 1.2)
            h.assemble(bem.DLP, 0.0, 1e-6, bem.FP64)
            return h.matvec(x)
        ys[name] = _with_shape(shape, run)
    ref = ys["cta_warp"]
    for name, y in ys.items():
        assert relf(y, ref) < 4e-6, name


def test_entries_repeated_trial_ids(lib):
    """bem_entries with a trial list that repeats a touching triangle more
    often than the singular-pair bound counts (n_test times the most
    triangles touching one triangle): the second, exactly sized pass gives
    the oracle's values."""
    V, T = meshes.icosphere_level(2)
    m = bem.Mesh(V, T)
    test = np.array([0, 7], dtype=np.int32)
    trial = np.array([0] * 40 + [1, 2, 3] * 10 + [7] * 25, dtype=np.int32)
    for prec in (bem.FP64, bem.MIXED, bem.MIXED_SP):
        got = m.entries(bem.SLP, 0.0, prec, test, trial)
        ref = oracle.entries(V, T, bem.SLP, 0.0, test, trial).real
        assert relf(got, ref) < (1e-11 if prec == bem.FP64 else 1e-5)


def test_pivot_reciprocal_against_division(lib):
    """recip(a): Newton-Raphson from a single-precision seed for exponents
    within +-120 of the bias, IEEE division outside.  Checked against 1/a
    (numpy, correctly rounded) to within one unit in the last place, at
    random mantissas and signs over exponents -140 .. 140, at both edges of
    the seed's window (2^-120, 2^120 and their neighbours) and at values
    whose FP32 seed rounds up (mantissas of all ones)."""
    import torch
    rng = np.random.default_rng(3)
    ex = rng.integers(-140, 141, size=20000)
    x = rng.uniform(1.0, 2.0, size=ex.size) * np.ldexp(1.0, ex)
    x *= rng.choice([-1.0, 1.0], size=x.size)
    edges = []
    for e in (-121, -120, -119, 119, 120, 121):
        for mant in (1.0, np.nextafter(1.0, 2.0), np.nextafter(2.0, 1.0), 1.5):
            edges += [mant * np.ldexp(1.0, e), -mant * np.ldexp(1.0, e)]
    x = np.concatenate([x, edges, [1.0, -1.0, 3.0, 1.0 / 3.0, 1e-300, 1e300, 3e-308]])
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    bem.bem_debug_recip(xd, yd)
    y = yd.cpu().numpy()
    ref = 1.0 / x
    ulp = np.abs(np.spacing(ref))
    err = np.abs(y - ref)
    assert np.all(err <= ulp), (x[np.argmax(err / ulp)], np.max(err / ulp))
    # in the seed's window the result is at most one ulp from the correctly
    # rounded quotient, and most are exact
    inwin = (np.abs(np.frexp(x)[1] - 1) <= 120)
    assert np.mean(y[inwin] == ref[inwin]) > 0.9
    # outside the window the division is exact IEEE
    out = ~inwin
    assert np.array_equal(y[out], ref[out])
