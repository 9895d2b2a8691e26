"""Host logic of the request server, run without a GPU (dry-run servers:
no CUDA call, simulated device work, reserved bytes = 1024 per triangle)."""
import time

import numpy as np
import pytest

from paper_1711_01897_gb300 import bem, meshes
from paper_1711_01897_gb300 import build as bem_build


@pytest.fixture(scope="module")
def lib():
    bem_build.build()
    return bem.load()


def _mesh(nu):
    return meshes.icosphere(nu)


def test_budget_never_exceeded_and_all_complete(lib):
    budget = 3 * 1024 * 1280          # room for three L3-sized requests
    srv = bem.Server(budget, max_slots=6, dry_run=True)
    V, T = _mesh(8)                   # 1,280 triangles -> 1.25 MiB each
    ids = [srv.submit(V, T, np.arange(T.shape[0], dtype=float), dry_run_ms=30) for _ in range(12)]
    peak_running = 0
    while srv.stats()["completed"] < len(ids):
        peak_running = max(peak_running, srv.stats()["running"])
        time.sleep(0.005)
    st = srv.stats()
    assert st["peak_reserved_bytes"] <= budget
    assert st["peak_reserved_bytes"] == budget      # three ran together
    assert peak_running <= 3
    for i in ids:
        rc, info, y = srv.wait(i)
        assert rc == 0 and info.state == bem.DONE
        assert np.array_equal(y, np.arange(T.shape[0], dtype=float))
        assert info.t_submit_ms <= info.t_admit_ms <= info.t_done_ms
    srv.close()


def test_admission_in_arrival_order(lib):
    V, T = _mesh(8)
    srv = bem.Server(1024 * 1280, max_slots=4, dry_run=True)   # one at a time
    ids = [srv.submit(V, T, np.zeros(T.shape[0]), dry_run_ms=10) for _ in range(6)]
    infos = [srv.wait(i)[1] for i in ids]
    admits = [inf.t_admit_ms for inf in infos]
    assert admits == sorted(admits)
    for a, b in zip(infos, infos[1:]):
        assert b.t_admit_ms >= a.t_done_ms - 1e-6   # never two at once
    srv.close()


def test_oversized_request_fails_alone(lib):
    V, T = _mesh(8)
    srv = bem.Server(1024 * 100, max_slots=2, dry_run=True)
    rid = srv.submit(V, T, np.zeros(T.shape[0]), dry_run_ms=1)
    rc, info, _ = srv.wait(rid)
    assert rc == 3 and info.state == bem.FAILED
    srv.close()


def test_cancel_timeout_and_shutdown(lib):
    V, T = _mesh(8)
    srv = bem.Server(1024 * 1280, max_slots=1, dry_run=True)
    a = srv.submit(V, T, np.zeros(T.shape[0]), dry_run_ms=300)
    b = srv.submit(V, T, np.zeros(T.shape[0]), dry_run_ms=1)
    c = srv.submit(V, T, np.zeros(T.shape[0]), dry_run_ms=1)
    time.sleep(0.05)
    assert srv.cancel(b) == 0
    rc, info, _ = srv.wait(a, timeout_ms=20)          # still running: bounded wait ends
    assert rc == 5 and info.state in (bem.PREPARING, bem.RUNNING)
    rc, info, _ = srv.wait(b)
    assert info.state == bem.CANCELLED
    assert srv.cancel(a) == 6                          # already started
    rc, _, _ = srv.wait(a)
    assert rc == 0
    srv.close()                                        # c is done or cancelled, no hang
    assert c > a


def test_bad_requests_rejected(lib):
    srv = bem.Server(1 << 20, max_slots=1, dry_run=True)
    V, T = _mesh(2)
    with pytest.raises(bem.BemError):
        srv.submit(V, T, np.zeros(T.shape[0]), aca_eps=-1.0)
    with pytest.raises(bem.BemError):
        srv.submit(V, T, np.zeros(T.shape[0]), op=5)
    srv.close()


def test_batches_share_launches(lib):
    """Requests admitted while a batch runs go into the next batch together:
    one (simulated) ACA launch holds several requests."""
    V, T = _mesh(8)
    srv = bem.Server(16 * 1024 * 1280, max_slots=8, dry_run=True)
    ids = [srv.submit(V, T, np.full(T.shape[0], float(i)), dry_run_ms=60) for i in range(8)]
    for i, rid in enumerate(ids):
        rc, info, y = srv.wait(rid)
        assert rc == 0 and np.all(y == float(i))
        assert info.launch_requests >= 1 and info.reused == 0
    st = srv.stats()
    assert st["max_launch_requests"] >= 2
    assert st["aca_launch_requests"] == len(ids)
    assert st["aca_launches"] < len(ids)
    srv.close()


def test_resident_reuse_and_eviction(lib):
    """A finished request's matrix stays resident (its bytes stay reserved);
    a product-only request naming it runs without assembling; admissions that
    need the bytes evict it, after which naming it fails with BEM_E_STATE."""
    V, T = _mesh(8)
    per = 1024 * T.shape[0]
    srv = bem.Server(2 * per, max_slots=2, dry_run=True)
    a = srv.submit(V, T, np.ones(T.shape[0]), dry_run_ms=5)
    rc, info, _ = srv.wait(a)
    assert rc == 0
    st = srv.stats()
    assert st["resident"] == 1 and st["resident_bytes"] == per and st["reserved_bytes"] == per
    p = srv.submit_product(a, np.arange(T.shape[0], dtype=float))
    rc, info, y = srv.wait(p)
    assert rc == 0 and info.reused == 1 and info.launch_requests == 0
    assert np.array_equal(y, np.arange(T.shape[0], dtype=float))
    assert srv.stats()["reuse_hits"] == 1
    # two more requests need the whole budget: the idle resident one goes
    b = srv.submit(V, T, np.zeros(T.shape[0]), dry_run_ms=5)
    c = srv.submit(V, T, np.zeros(T.shape[0]), dry_run_ms=5)
    assert srv.wait(b)[0] == 0 and srv.wait(c)[0] == 0
    st = srv.stats()
    assert st["evictions"] >= 1 and st["peak_reserved_bytes"] <= 2 * per
    with pytest.raises(bem.BemError) as e:
        srv.submit_product(a, np.zeros(T.shape[0]))
    assert e.value.status == 6
    srv.close()


def test_product_waits_for_its_assembly(lib):
    """A product request submitted while the assembly it names is still
    running waits for it and then reuses it."""
    V, T = _mesh(8)
    srv = bem.Server(4 * 1024 * T.shape[0], max_slots=2, dry_run=True)
    a = srv.submit(V, T, np.ones(T.shape[0]), dry_run_ms=80)
    p = srv.submit_product(a, np.full(T.shape[0], 2.0))
    rc, info, y = srv.wait(p)
    assert rc == 0 and info.reused == 1 and np.all(y == 2.0)
    assert srv.poll(a).state == bem.DONE
    srv.close()


def test_small_requests_pass_a_waiting_large_one(lib):
    """A large request that must wait for budget lets small requests that
    fit start before it (for a bounded time), so that they do not queue
    behind it; it still starts once the budget allows."""
    VL, TL = _mesh(45)                 # 40,500 triangles: a large request
    VS, TS = _mesh(8)
    per_large = 1024 * TL.shape[0]
    srv = bem.Server(int(1.2 * per_large), max_slots=6, dry_run=True)
    l1 = srv.submit(VL, TL, np.zeros(TL.shape[0]), dry_run_ms=250)
    time.sleep(0.02)
    l2 = srv.submit(VL, TL, np.zeros(TL.shape[0]), dry_run_ms=50)
    time.sleep(0.02)
    small = [srv.submit(VS, TS, np.zeros(TS.shape[0]), dry_run_ms=5) for _ in range(3)]
    infos = {rid: srv.wait(rid)[1] for rid in [l1, l2] + small}
    for rid in small:
        assert infos[rid].t_done_ms < infos[l2].t_admit_ms        # passed the waiting one
        assert infos[rid].t_done_ms - infos[rid].t_submit_ms < 200
    assert infos[l2].t_admit_ms >= infos[l1].t_done_ms - 1e-6       # budget: one large at a time
    assert srv.stats()["peak_reserved_bytes"] <= int(1.2 * per_large)
    srv.close()
