"""The FP64 reciprocal square root of the FP64 quadratures (singular pairs,
Sec. 3.2.3; FP64 regular pairs), checked directly against numpy's correctly
rounded 1/sqrt(x) over the whole normal range.  The entries built from it are
checked against the oracle in the parity tests."""
import numpy as np
import pytest

from paper_1711_01897_gb300 import bem

pytestmark = pytest.mark.gpu

# one Newton step from a seed with relative error below 2^-22.3 leaves
# 1.5 e^2 plus the rounding of three FP64 operations
BOUND = 2.0 ** -43.7


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    torch.cuda.init()
    return bem.load()


def _run(x):
    import torch
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    bem.bem_debug_rsqrt(xd, yd)
    return yd.cpu().numpy()


def test_rsqrt_random_mantissas_all_exponents(lib):
    """Random mantissas at every exponent of the normal range (odd and even,
    since the reduction moves an even power of two out of the argument)."""
    rng = np.random.default_rng(11)
    ex = np.repeat(np.arange(-1022, 1024), 24)
    x = rng.uniform(1.0, 2.0, size=ex.size) * np.ldexp(1.0, ex)
    x = x[np.isfinite(x)]
    y = _run(x)
    ref = 1.0 / np.sqrt(x)
    rel = np.abs(y - ref) / ref
    assert np.all(np.isfinite(y))
    assert rel.max() < BOUND, (x[np.argmax(rel)], rel.max())


def test_rsqrt_edges(lib):
    """Mantissa edges (1, the largest below 2, below 4 after the reduction),
    exact squares, and the extreme normals."""
    vals = []
    for e in (-1022, -1021, -2, -1, 0, 1, 2, 3, 1020, 1021, 1022, 1023):
        for m in (1.0, np.nextafter(1.0, 2.0), np.nextafter(2.0, 1.0), 1.5):
            v = m * np.ldexp(1.0, e)
            if np.isfinite(v):
                vals.append(v)
    vals += [4.0, 9.0, 0.25, 1e-300, 1e300, np.finfo(np.float64).tiny, np.finfo(np.float64).max]
    x = np.array(vals)
    y = _run(x)
    ref = 1.0 / np.sqrt(x)
    rel = np.abs(y - ref) / ref
    assert rel.max() < BOUND, (x[np.argmax(rel)], rel.max())
    # the geometry's range: most results are within a few ulps
    ulp = np.abs(np.spacing(ref))
    assert np.median(np.abs(y - ref) / ulp) < 64
