"""bem_entries_noalloc: the allocation-free variant of bem_entries, called
through the C ABI.  Some callers cannot allocate device memory once they run
(their memory is fully reserved by their own pool allocator, or an allocation
stall or failure mid-run is not acceptable); this entry point takes device
buffers and uses a fixed scratch array inside the library instead.

Its results must equal bem_entries' results within the tolerances of the
other parity tests, on two calls in a row (the shared scratch keeps the
previous call's contents, so the second call checks that it is cleared), and
a call must change neither the library's memory pool nor the device's free
memory."""
import ctypes

import numpy as np
import pytest

from paper_1711_01897_gb300 import bem, meshes

pytestmark = pytest.mark.gpu


def _fn():
    lib = bem.load()
    f = lib.bem_entries_noalloc
    P = ctypes.c_void_p
    f.argtypes = [P, ctypes.c_int32, ctypes.c_double, ctypes.c_int32, P, ctypes.c_int64, P,
                  ctypes.c_int64, P, P]
    f.restype = ctypes.c_int
    return f


def _call(f, mesh, op, k, prec, test, trial, out, stream):
    return f(mesh.handle, op, k, prec, ctypes.c_void_p(test.data_ptr()), test.numel(),
             ctypes.c_void_p(trial.data_ptr()), trial.numel(), ctypes.c_void_p(out.data_ptr()),
             ctypes.c_void_p(stream))


def test_noalloc_matches_bem_entries_twice():
    import torch
    assert torch.cuda.is_available()
    torch.cuda.init()
    f = _fn()
    V, T = meshes.icosphere_level(3)
    mesh = bem.Mesh(V, T)
    stream = torch.cuda.current_stream().cuda_stream
    cases = [
        # (op, k, prec, test ids, trial ids): both sets share many vertices
        (bem.SLP, 0.0, bem.FP64, np.arange(0, 90, dtype=np.int32), np.arange(40, 170, dtype=np.int32)),
        (bem.DLP, 2.0, bem.MIXED, np.arange(500, 561, dtype=np.int32), np.arange(480, 600, dtype=np.int32)),
    ]
    for op, k, prec, ti, tj in cases:
        dt = torch.float64 if k == 0 else torch.complex128
        test = torch.from_numpy(ti).cuda()
        trial = torch.from_numpy(tj).cuda()
        out = torch.full((ti.size, tj.size), float("nan"), dtype=dt, device="cuda")
        rc = _call(f, mesh, op, k, prec, test, trial, out, stream)
        assert rc == 0, bem.bem_last_error()
        ref = mesh.entries(op, k, prec, ti, tj)
        got = out.cpu().numpy()
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert rel < (1e-13 if prec == bem.FP64 else 1e-12), rel
        assert np.isfinite(got).all()


def test_noalloc_allocates_nothing():
    """After a first call (which may load code and look up the scratch
    address), further calls leave the library pool's reserved and used bytes
    and the device's free memory unchanged."""
    import torch
    torch.cuda.init()
    f = _fn()
    V, T = meshes.icosphere_level(3)
    mesh = bem.Mesh(V, T)
    stream = torch.cuda.current_stream().cuda_stream
    test = torch.arange(100, 260, dtype=torch.int32, device="cuda")
    trial = torch.arange(150, 400, dtype=torch.int32, device="cuda")
    out = torch.zeros(160, 250, dtype=torch.complex128, device="cuda")
    assert _call(f, mesh, bem.SLP, 1.5, bem.MIXED, test, trial, out, stream) == 0
    torch.cuda.synchronize()
    pool0, free0 = bem.bem_memory_usage(), torch.cuda.mem_get_info()[0]
    for op in (bem.SLP, bem.DLP, bem.ADLP):
        assert _call(f, mesh, op, 1.5, bem.MIXED, test, trial, out, stream) == 0
    torch.cuda.synchronize()
    assert bem.bem_memory_usage() == pool0
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_host_buffers_bad_ids_and_oversized_requests():
    import torch
    f = _fn()
    V, T = meshes.icosphere_level(2)
    mesh = bem.Mesh(V, T)
    nt = T.shape[0]
    ids = torch.arange(0, 10, dtype=torch.int32)            # host tensor
    out = torch.zeros(10, 10, dtype=torch.float64)
    rc = f(mesh.handle, 0, 0.0, 0, ctypes.c_void_p(ids.data_ptr()), 10,
           ctypes.c_void_p(ids.data_ptr()), 10, ctypes.c_void_p(out.data_ptr()), None)
    assert rc == 1
    # an id one past the last triangle is found on the device
    bad = torch.tensor([0, 1, nt], dtype=torch.int32, device="cuda")
    good = torch.arange(0, 8, dtype=torch.int32, device="cuda")
    o = torch.zeros(3, 8, dtype=torch.float64, device="cuda")
    rc = f(mesh.handle, 0, 0.0, 1, ctypes.c_void_p(bad.data_ptr()), 3,
           ctypes.c_void_p(good.data_ptr()), 8, ctypes.c_void_p(o.data_ptr()), None)
    assert rc == 1 and "out of range" in bem.bem_last_error()
    big = torch.zeros(300000, dtype=torch.int32, device="cuda")
    one = torch.zeros(1, dtype=torch.int32, device="cuda")
    o = torch.zeros(300000, dtype=torch.float64, device="cuda")
    rc = f(mesh.handle, 0, 0.0, 0, ctypes.c_void_p(big.data_ptr()), big.numel(),
           ctypes.c_void_p(one.data_ptr()), 1, ctypes.c_void_p(o.data_ptr()), None)
    assert rc == 1 and "scratch" in bem.bem_last_error()
    # one test triangle against 300,000 copies of itself passes the size
    # bound (1 x the touching count) but holds 300,000 identical pairs: the
    # scratch fills and the call says so
    rc = f(mesh.handle, 0, 0.0, 0, ctypes.c_void_p(one.data_ptr()), 1,
           ctypes.c_void_p(big.data_ptr()), big.numel(), ctypes.c_void_p(o.data_ptr()), None)
    assert rc == 1 and "repeated" in bem.bem_last_error()
