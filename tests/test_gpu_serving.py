"""Request server on the GPU: results are identical alone and in a mix of
concurrent requests (each request's arithmetic does not depend on what runs
beside it, even when its blocks share one persistent ACA launch with other
requests' blocks), the HBM budget is respected, products match the oracle,
and product-only requests against resident matrices give the same result
as the assembly that left the matrix there."""
import numpy as np
import pytest

import oracle
from paper_1711_01897_gb300 import bem, meshes

pytestmark = pytest.mark.gpu


def _requests():
    rng = np.random.default_rng(17)
    reqs = []
    for i, (nu, kind, k, eps) in enumerate([(4, "sphere", 0.0, 1e-4), (6, "ellipsoid", 2.0, 1e-6),
                                             (8, "sphere", 5.0, 1e-4), (5, "sphere", 0.0, 1e-6),
                                             (10, "ellipsoid", 0.0, 1e-4), (7, "sphere", 1.0, 1e-4),
                                             (12, "sphere", 0.0, 1e-4), (9, "ellipsoid", 3.0, 1e-6)]):
        V, T = meshes.icosphere(nu)
        if kind == "ellipsoid":
            V = V * np.array([1.5, 1.0, 0.6])
        else:
            V = meshes.jitter(V, T, 0.05, 500 + i)
        x = rng.normal(size=T.shape[0])
        if k != 0:
            x = x + 1j * rng.normal(size=T.shape[0])
        reqs.append(dict(V=V, T=T, x=x, k=k, eps=eps))
    return reqs


def _run(reqs, slots, budget, reuse=False):
    srv = bem.Server(budget, max_slots=slots)
    ids = [srv.submit(r["V"], r["T"], r["x"], op=bem.SLP, k=r["k"], aca_eps=r["eps"],
                      prec=bem.MIXED, leaf_size=16, eta=1.2) for r in reqs]
    out = []
    for i in ids:
        rc, info, y = srv.wait(i)
        assert rc == 0, bem.bem_last_error()
        out.append((y, info))
    again = []
    if reuse:
        # the same vectors again, as products against the resident matrices
        for i, r in zip(ids, reqs):
            p = srv.submit_product(i, r["x"])
            rc, info, y = srv.wait(p)
            assert rc == 0, bem.bem_last_error()
            assert info.reused == 1
            again.append(y)
    st = srv.stats()
    srv.close()
    return out, st, again


def test_alone_and_mixed_identical_and_budget():
    import torch
    assert torch.cuda.is_available()
    torch.cuda.init()
    reqs = _requests()
    alone, st1, again = _run(reqs, 1, 64 << 30, reuse=True)
    assert st1["max_launch_requests"] == 1 and st1["reuse_hits"] == len(reqs)
    for (ya, _), yr in zip(alone, again):
        assert np.array_equal(ya, yr)
    budget = 3 * max(info.reserved_bytes for _, info in alone)
    mixed, st, _ = _run(reqs, 4, budget)
    assert st["peak_reserved_bytes"] <= budget
    assert st["completed"] == len(reqs)
    # requests of the same kind shared ACA launches
    assert st["max_launch_requests"] >= 2, st
    assert any(info.launch_requests >= 2 for _, info in mixed)
    for (ya, ia), (ym, im) in zip(alone, mixed):
        assert np.array_equal(ya, ym)
        assert ia.integrals == im.integrals and ia.integrals > 0
    # overlap: some request was admitted before an earlier one finished
    overl = any(mixed[j][1].t_admit_ms < mixed[i][1].t_done_ms
                for i in range(len(mixed)) for j in range(i + 1, len(mixed)))
    assert overl
    # two products against the oracle's dense matrix
    for idx in (0, 2):
        r = reqs[idx]
        A = oracle.dense_matrix(r["V"], r["T"], oracle.SLP, r["k"])
        if r["k"] == 0:
            A = A.real
        ref = A @ r["x"]
        assert np.linalg.norm(alone[idx][0] - ref) / np.linalg.norm(ref) < 2 * r["eps"] + 1e-5
