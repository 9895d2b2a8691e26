"""Request server on the GPU: results are identical alone and in a mix of
concurrent requests (each request's arithmetic does not depend on what runs
beside it), the HBM budget is respected, and products match the oracle."""
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


def _run(reqs, slots, budget):
    srv = bem.Server(budget, max_slots=slots)
    ids = [srv.submit(r["V"], r["T"], r["x"], op=bem.SLP, k=r["k"], aca_eps=r["eps"],
                      prec=bem.MIXED, leaf_size=16, eta=1.2) for r in reqs]
    out = []
    for i in ids:
        rc, info, y = srv.wait(i)
        assert rc == 0, bem.bem_last_error()
        out.append((y, info))
    st = srv.stats()
    srv.close()
    return out, st


def test_alone_and_mixed_identical_and_budget():
    import torch
    assert torch.cuda.is_available()
    torch.cuda.init()
    reqs = _requests()
    alone, _ = _run(reqs, 1, 64 << 30)
    budget = 3 * max(info.reserved_bytes for _, info in alone)
    mixed, st = _run(reqs, 4, budget)
    assert st["peak_reserved_bytes"] <= budget
    assert st["completed"] == len(reqs)
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
