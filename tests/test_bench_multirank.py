"""The N > 1 path of bench.py on CPU: two gloo ranks (no GPU, no data-path
collective besides the final figures).  Each rank solves an independent
problem (its own jitter seed); the job's time is the slowest rank's and its
integrals are the sum over ranks.  The reference arm does no work on ranks
other than 0."""
import contextlib
import io
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t, e = bench.reduce_over_ranks(10.0 + 3.0 * rank, 100 * (rank + 1), dist, "cpu")
        q.put((rank, t, e, bench.rank_jitter_seed(rank)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_max_and_integrals_sum():
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get() for _ in range(2))
    for rank, t, e, seed in got:
        assert t == 13.0 and e == 300.0
    assert got[0][3] != got[1][3] and got[0][3] == 1001


def test_reference_arm_only_on_rank_zero(monkeypatch):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")

    class Args:
        warmup, steps, ref_seconds, gpus = 1, 1, 1.0, 2

    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        assert bench.run_reference(Args()) == 0
    assert buf.getvalue() == ""
