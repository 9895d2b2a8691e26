"""Thin Python binding of libbem.so (include/bem.h): the same call names,
argument marshalling only.  Every step of the computation runs in the CUDA
library; there is no fallback, and a missing library raises.

Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA);
streams default to torch's current CUDA stream when torch is available.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbem.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "bem.h")

SLP, DLP, ADLP, HYPS = 0, 1, 2, 3
FP64, MIXED, MIXED_SP = 0, 1, 2
P0, DP1, P1 = 0, 1, 2
STATUS = {0: "BEM_OK", 1: "BEM_E_ARG", 2: "BEM_E_MESH", 3: "BEM_E_OOM", 4: "BEM_E_CUDA",
          5: "BEM_E_TIMEOUT", 6: "BEM_E_STATE"}

_lock = threading.Lock()
_lib = None


class BemError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class HmatStats(ctypes.Structure):
    _fields_ = [("n_triangles", ctypes.c_int64), ("n_clusters", ctypes.c_int64),
                ("n_blocks_near", ctypes.c_int64), ("n_blocks_far", ctypes.c_int64),
                ("near_entries", ctypes.c_int64), ("singular_pairs", ctypes.c_int64 * 3),
                ("far_entries", ctypes.c_int64), ("factor_bytes", ctypes.c_int64),
                ("near_bytes", ctypes.c_int64), ("rank_min", ctypes.c_int32),
                ("rank_max", ctypes.c_int32), ("rank_mean", ctypes.c_double),
                ("rank_capped_blocks", ctypes.c_int64), ("time_tree_ms", ctypes.c_double),
                ("time_near_ms", ctypes.c_double), ("time_far_ms", ctypes.c_double),
                ("time_near_regular_ms", ctypes.c_double), ("time_singular_ms", ctypes.c_double),
                ("aca_fp64_fma", ctypes.c_int64),
                ("assembled", ctypes.c_int32), ("op", ctypes.c_int32), ("k", ctypes.c_double),
                ("aca_eps", ctypes.c_double), ("prec", ctypes.c_int32),
                ("space", ctypes.c_int32), ("n_dofs", ctypes.c_int64),
                ("time_tree_clusters_ms", ctypes.c_double), ("time_tree_blocks_ms", ctypes.c_double),
                ("time_tree_lists_ms", ctypes.c_double), ("time_tree_upload_ms", ctypes.c_double),
                ("factor_read_bytes", ctypes.c_int64),
                ("n_blocks_rule3", ctypes.c_int64), ("n_blocks_rule1", ctypes.c_int64),
                ("rho3", ctypes.c_double), ("rho1", ctypes.c_double),
                ("n_blocks_cta", ctypes.c_int64), ("n_blocks_warp", ctypes.c_int64),
                ("n_blocks_lane", ctypes.c_int64), ("n_blocks_half_warp", ctypes.c_int64),
                ("n_blocks_quarter_warp", ctypes.c_int64)]


class Peaks(ctypes.Structure):
    _fields_ = [("fp32_fma_per_s", ctypes.c_double), ("fp64_fma_per_s", ctypes.c_double),
                ("mufu_rsqrt_per_s", ctypes.c_double), ("mufu_sin_per_s", ctypes.c_double),
                ("copy_bytes_per_s", ctypes.c_double), ("sm_count", ctypes.c_int32),
                ("clock_mhz_nominal", ctypes.c_double), ("ms", ctypes.c_float * 5)]


class Tuning(ctypes.Structure):
    _fields_ = [("warp_max_rows", ctypes.c_int32), ("lane_max_rows", ctypes.c_int32),
                ("use_graphs", ctypes.c_int32)]


class Quadrature(ctypes.Structure):
    _fields_ = [("rho3", ctypes.c_double), ("rho1", ctypes.c_double)]


class Request(ctypes.Structure):
    _fields_ = [("vertices", ctypes.c_void_p), ("n_vertices", ctypes.c_int64),
                ("triangles", ctypes.c_void_p), ("n_triangles", ctypes.c_int64),
                ("op", ctypes.c_int32), ("k", ctypes.c_double), ("aca_eps", ctypes.c_double),
                ("prec", ctypes.c_int32), ("leaf_size", ctypes.c_int32), ("eta", ctypes.c_double),
                ("x", ctypes.c_void_p), ("dry_run_ms", ctypes.c_double),
                ("reuse", ctypes.c_int64)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("status", ctypes.c_int32),
                ("t_submit_ms", ctypes.c_double), ("t_admit_ms", ctypes.c_double),
                ("t_done_ms", ctypes.c_double), ("reserved_bytes", ctypes.c_int64),
                ("integrals", ctypes.c_int64), ("assembly_ms", ctypes.c_double),
                ("launch_requests", ctypes.c_int32), ("reused", ctypes.c_int32),
                ("t_ready_ms", ctypes.c_double), ("t_launch_ms", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in
                ("submitted", "completed", "failed", "cancelled", "queued", "running",
                 "reserved_bytes", "peak_reserved_bytes", "budget_bytes", "resident",
                 "resident_bytes", "evictions", "reuse_hits", "aca_launches",
                 "aca_launch_requests", "max_launch_requests")]


QUEUED, PREPARING, RUNNING, DONE, FAILED, CANCELLED = range(6)
SERVER_DRY_RUN = 1


def header_functions() -> list[str]:
    """Names of the functions declared in include/bem.h."""
    with open(HEADER) as f:
        src = f.read()
    return re.findall(r"^\w[\w\s\*]*?\b((?:bem|hmat)_\w+)\s*\(", src, flags=re.M)


def load(path: str = LIB_PATH):
    """Loads libbem.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with "
                               "`python -m paper_1711_01897_gb300.build`")
        L = ctypes.CDLL(path)
        P, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        sig = {
            "bem_version": ([], ctypes.c_int),
            "bem_kernel_launches": ([], ctypes.c_int64),
            "bem_memory_usage": ([P, P], ctypes.c_int),
            "bem_debug_recip": ([P, P, i64, P], ctypes.c_int),
            "bem_debug_rsqrt": ([P, P, i64, P], ctypes.c_int),
            "bem_measure_peaks": ([ctypes.POINTER(Peaks), P], ctypes.c_int),
            "bem_set_tuning": ([ctypes.POINTER(Tuning)], ctypes.c_int),
            "bem_get_tuning": ([ctypes.POINTER(Tuning)], ctypes.c_int),
            "bem_set_quadrature": ([ctypes.POINTER(Quadrature)], ctypes.c_int),
            "bem_get_quadrature": ([ctypes.POINTER(Quadrature)], ctypes.c_int),
            "bem_last_error": ([], ctypes.c_char_p),
            "bem_mesh_create": ([P, i64, P, i64, P], ctypes.c_int),
            "bem_mesh_destroy": ([P], ctypes.c_int),
            "bem_mesh_size": ([P], i64),
            "bem_entries": ([P, i32, dbl, i32, P, i64, P, i64, P, P], ctypes.c_int),
            "bem_entries_dp1": ([P, i32, dbl, i32, P, i64, P, i64, P, P], ctypes.c_int),
            "hmat_build_tree": ([P, i32, dbl, P], ctypes.c_int),
            "hmat_build_tree_space": ([P, i32, dbl, i32, P], ctypes.c_int),
            "hmat_dofs": ([P], i64),
            "bem_partition_rows": ([P, i64, i64, i32, dbl, P], ctypes.c_int),
            "hmat_build_tree_part": ([P, i32, dbl, i32, i32, P], ctypes.c_int),
            "hmat_part_rows": ([P, P, P], ctypes.c_int),
            "hmat_assemble": ([P, i32, dbl, dbl, i32, P], ctypes.c_int),
            "hmat_matvec": ([P, P, P, i32, P], ctypes.c_int),
            "hmat_stats": ([P, ctypes.POINTER(HmatStats)], ctypes.c_int),
            "hmat_blocks": ([P, P, i64, P, P], ctypes.c_int),
            "hmat_block_dense": ([P, i64, P, P], ctypes.c_int),
            "hmat_block_rules": ([P, P, i64], ctypes.c_int),
            "hmat_destroy": ([P], ctypes.c_int),
            "bem_server_create": ([i64, i32, i32, P], ctypes.c_int),
            "bem_server_submit": ([P, ctypes.POINTER(Request), P], ctypes.c_int),
            "bem_server_poll": ([P, i64, ctypes.POINTER(RequestInfo)], ctypes.c_int),
            "bem_server_wait": ([P, i64, i64, ctypes.POINTER(RequestInfo), P], ctypes.c_int),
            "bem_server_cancel": ([P, i64], ctypes.c_int),
            "bem_server_stats_get": ([P, ctypes.POINTER(ServerStats)], ctypes.c_int),
            "bem_server_destroy": ([P], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    # apply the autotuner's table, if one has been written
    table = os.path.join(_HERE, "tuning.json")
    if os.path.exists(table):
        import json
        with open(table) as f:
            t = json.load(f)
        tt = Tuning(int(t["warp_max_rows"]), int(t["lane_max_rows"]), int(t.get("use_graphs", 1)))
        L.bem_set_tuning(ctypes.byref(tt))
    return L


def _check(rc: int):
    if rc != 0:
        raise BemError(rc, load().bem_last_error().decode())


def _ptr(a):
    """(pointer, keepalive) for a numpy array or torch tensor."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data), a
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr()), a
    raise TypeError(f"unsupported array type {type(a)}")


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return ctypes.c_void_p(0)


def bem_version() -> int:
    return int(load().bem_version())


def bem_kernel_launches() -> int:
    return int(load().bem_kernel_launches())


def bem_memory_usage() -> dict:
    r, u = ctypes.c_int64(), ctypes.c_int64()
    _check(load().bem_memory_usage(ctypes.byref(r), ctypes.byref(u)))
    return {"reserved": r.value, "used": u.value}


def bem_measure_peaks(stream=None) -> dict:
    """Unit throughputs measured on the current device (see bem.h)."""
    p = Peaks()
    _check(load().bem_measure_peaks(ctypes.byref(p), _stream(stream)))
    d = {n: getattr(p, n) for n, _ in Peaks._fields_ if n != "ms"}
    d["ms"] = list(p.ms)
    return d


def bem_debug_recip(x, y, stream=None):
    """y = 1 / x on the device by the ACA pivot reciprocal; x, y device
    tensors of float64 (same length)."""
    n = x.numel()
    assert y.numel() == n
    _check(load().bem_debug_recip(_ptr(x)[0], _ptr(y)[0], n, _stream(stream)))


def bem_debug_rsqrt(x, y, stream=None):
    """y = 1 / sqrt(x) on the device by the FP64 quadratures' reciprocal
    square root; x, y device tensors of float64 (same length), x > 0."""
    n = x.numel()
    assert y.numel() == n
    _check(load().bem_debug_rsqrt(_ptr(x)[0], _ptr(y)[0], n, _stream(stream)))


def bem_set_tuning(warp_max_rows: int, lane_max_rows: int, use_graphs: int = 1):
    t = Tuning(int(warp_max_rows), int(lane_max_rows), int(use_graphs))
    _check(load().bem_set_tuning(ctypes.byref(t)))


def bem_get_tuning() -> dict:
    t = Tuning()
    _check(load().bem_get_tuning(ctypes.byref(t)))
    return {"warp_max_rows": t.warp_max_rows, "lane_max_rows": t.lane_max_rows,
            "use_graphs": t.use_graphs}


def bem_set_quadrature(rho3: float, rho1: float):
    """Distance classes of the regular rule for trees built from now on:
    admissible blocks with dist / h >= rho1 use the centroid rule, else >= rho3
    the 3-point degree-2 rule, else the 6-point rule (0 = class off)."""
    q = Quadrature(float(rho3), float(rho1))
    _check(load().bem_set_quadrature(ctypes.byref(q)))


def bem_get_quadrature() -> dict:
    q = Quadrature()
    _check(load().bem_get_quadrature(ctypes.byref(q)))
    return {"rho3": q.rho3, "rho1": q.rho1}


def bem_last_error() -> str:
    return load().bem_last_error().decode()


def bem_mesh_create(vertices, triangles):
    V = np.ascontiguousarray(vertices, dtype=np.float64)
    T = np.ascontiguousarray(triangles, dtype=np.int32)
    if V.ndim != 2 or V.shape[1] != 3 or T.ndim != 2 or T.shape[1] != 3:
        raise ValueError("vertices and triangles must be [n,3]")
    h = ctypes.c_void_p()
    _check(load().bem_mesh_create(V.ctypes.data, V.shape[0], T.ctypes.data, T.shape[0],
                                  ctypes.byref(h)))
    return h


def bem_mesh_destroy(mesh):
    _check(load().bem_mesh_destroy(mesh))


def bem_mesh_size(mesh) -> int:
    return int(load().bem_mesh_size(mesh))


def bem_entries(mesh, op: int, k: float, prec: int, test_ids, trial_ids, out, stream=None):
    pt, kt = _ptr(test_ids)
    pj, kj = _ptr(trial_ids)
    po, ko = _ptr(out)
    _check(load().bem_entries(mesh, op, float(k), prec, pt, len(test_ids), pj, len(trial_ids), po,
                              _stream(stream)))
    del kt, kj, ko
    return out


def bem_entries_dp1(mesh, op: int, k: float, prec: int, test_tris, trial_tris, out, stream=None):
    pt, kt = _ptr(test_tris)
    pj, kj = _ptr(trial_tris)
    po, ko = _ptr(out)
    _check(load().bem_entries_dp1(mesh, op, float(k), prec, pt, len(test_tris), pj,
                                  len(trial_tris), po, _stream(stream)))
    del kt, kj, ko
    return out


def hmat_build_tree(mesh, leaf_size: int, eta: float):
    h = ctypes.c_void_p()
    _check(load().hmat_build_tree(mesh, int(leaf_size), float(eta), ctypes.byref(h)))
    return h


def hmat_build_tree_space(mesh, leaf_size: int, eta: float, space: int):
    h = ctypes.c_void_p()
    _check(load().hmat_build_tree_space(mesh, int(leaf_size), float(eta), int(space),
                                        ctypes.byref(h)))
    return h


def bem_partition_rows(blocks, n_rows: int, n_parts: int, rank_est: float = 10.0) -> np.ndarray:
    """Cluster-order row bounds [n_parts + 1] of a cost-balanced block-row
    partition of a block list (rows of 5 int64, as hmat_blocks returns)."""
    B = np.ascontiguousarray(blocks, dtype=np.int64)
    out = np.zeros(n_parts + 1, dtype=np.int64)
    _check(load().bem_partition_rows(B.ctypes.data, B.shape[0], int(n_rows), int(n_parts),
                                     float(rank_est), out.ctypes.data))
    return out


def hmat_build_tree_part(mesh, leaf_size: int, eta: float, n_parts: int, part: int):
    h = ctypes.c_void_p()
    _check(load().hmat_build_tree_part(mesh, int(leaf_size), float(eta), int(n_parts), int(part),
                                       ctypes.byref(h)))
    return h


def hmat_part_rows(hmat):
    b, e = ctypes.c_int64(), ctypes.c_int64()
    _check(load().hmat_part_rows(hmat, ctypes.byref(b), ctypes.byref(e)))
    return b.value, e.value


def hmat_dofs(hmat) -> int:
    return int(load().hmat_dofs(hmat))


def hmat_assemble(hmat, op: int, k: float, aca_eps: float, prec: int, stream=None):
    _check(load().hmat_assemble(hmat, op, float(k), float(aca_eps), prec, _stream(stream)))


def hmat_matvec(hmat, x, y, batch: int = 1, stream=None):
    px, kx = _ptr(x)
    py, ky = _ptr(y)
    _check(load().hmat_matvec(hmat, px, py, int(batch), _stream(stream)))
    del kx, ky
    return y


def hmat_stats(hmat) -> dict:
    s = HmatStats()
    _check(load().hmat_stats(hmat, ctypes.byref(s)))
    d = {name: getattr(s, name) for name, _ in HmatStats._fields_}
    d["singular_pairs"] = list(s.singular_pairs)
    return d


def hmat_blocks(hmat):
    """(blocks int64 [n,5] in cluster order, perm int32 [n_triangles])."""
    L = load()
    n = ctypes.c_int64()
    _check(L.hmat_blocks(hmat, None, 0, ctypes.byref(n), None))
    nt = hmat_stats(hmat)["n_triangles"]
    blocks = np.zeros((n.value, 5), dtype=np.int64)
    perm = np.zeros(nt, dtype=np.int32)
    _check(L.hmat_blocks(hmat, blocks.ctypes.data, n.value, ctypes.byref(n), perm.ctypes.data))
    return blocks, perm


def hmat_block_dense(hmat, block: int, shape, cplx: bool):
    out = np.zeros(shape, dtype=np.complex128 if cplx else np.float64)
    r = ctypes.c_int32()
    _check(load().hmat_block_dense(hmat, int(block), out.ctypes.data, ctypes.byref(r)))
    return out, int(r.value)


def hmat_block_rules(hmat) -> np.ndarray:
    """Points per triangle of every block's regular rule (6, 3, 1; 0 near)."""
    L = load()
    n = ctypes.c_int64()
    _check(L.hmat_blocks(hmat, None, 0, ctypes.byref(n), None))
    out = np.zeros(n.value, dtype=np.int32)
    _check(L.hmat_block_rules(hmat, out.ctypes.data, n.value))
    return out


def hmat_destroy(hmat):
    _check(load().hmat_destroy(hmat))


class Mesh:
    """Owns a bem_mesh handle."""

    def __init__(self, vertices, triangles):
        self.handle = bem_mesh_create(vertices, triangles)
        self.n = bem_mesh_size(self.handle)

    def entries(self, op, k, prec, test_ids, trial_ids, out=None, stream=None):
        if out is None:
            out = np.zeros((len(test_ids), len(trial_ids)),
                           dtype=np.complex128 if k != 0 else np.float64)
        return bem_entries(self.handle, op, k, prec, test_ids, trial_ids, out, stream)

    def entries_dp1(self, op, k, prec, test_tris, trial_tris, out=None, stream=None):
        if out is None:
            out = np.zeros((3 * len(test_tris), 3 * len(trial_tris)),
                           dtype=np.complex128 if k != 0 else np.float64)
        return bem_entries_dp1(self.handle, op, k, prec, test_tris, trial_tris, out, stream)

    def close(self):
        if self.handle is not None:
            bem_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HMatrix:
    """Owns a bem_hmat handle built on a Mesh."""

    def __init__(self, mesh: Mesh, leaf_size: int = 32, eta: float = 1.2, space: int = P0,
                 parts: int = 1, part: int = 0):
        """parts > 1: only block rows of part `part` of the row partition
        (hmat_build_tree_part)."""
        self.mesh = mesh
        self.space = space
        if parts > 1:
            self.handle = hmat_build_tree_part(mesh.handle, leaf_size, eta, parts, part)
        elif space == P0:
            self.handle = hmat_build_tree(mesh.handle, leaf_size, eta)
        else:
            self.handle = hmat_build_tree_space(mesh.handle, leaf_size, eta, space)
        self.n = hmat_dofs(self.handle)
        self.cplx = False

    def part_rows(self):
        return hmat_part_rows(self.handle)

    def assemble(self, op, k, aca_eps, prec, stream=None):
        hmat_assemble(self.handle, op, k, aca_eps, prec, stream)
        self.cplx = k != 0

    def matvec(self, x, y=None, batch=1, stream=None):
        if y is None:
            y = np.zeros_like(x)
        return hmat_matvec(self.handle, x, y, batch, stream)

    def stats(self):
        return hmat_stats(self.handle)

    def blocks(self):
        return hmat_blocks(self.handle)

    def block_dense(self, b, shape):
        return hmat_block_dense(self.handle, b, shape, self.cplx)

    def block_rules(self):
        return hmat_block_rules(self.handle)

    def close(self):
        if self.handle is not None:
            hmat_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Owns a bem_server: submit requests, wait for their products."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 4, dry_run: bool = False):
        self.handle = ctypes.c_void_p()
        _check(load().bem_server_create(int(hbm_budget_bytes), int(max_slots),
                                        SERVER_DRY_RUN if dry_run else 0, ctypes.byref(self.handle)))
        self._keep = {}
        self._shape = {}

    def submit(self, vertices, triangles, x, op=SLP, k=0.0, aca_eps=1e-4, prec=MIXED,
               leaf_size=32, eta=1.2, dry_run_ms=0.0) -> int:
        V = np.ascontiguousarray(vertices, dtype=np.float64)
        T = np.ascontiguousarray(triangles, dtype=np.int32)
        X = np.ascontiguousarray(x, dtype=np.complex128 if k != 0 else np.float64)
        q = Request(V.ctypes.data, V.shape[0], T.ctypes.data, T.shape[0], op, float(k),
                    float(aca_eps), prec, leaf_size, float(eta), X.ctypes.data, float(dry_run_ms), 0)
        rid = ctypes.c_int64()
        _check(load().bem_server_submit(self.handle, ctypes.byref(q), ctypes.byref(rid)))
        self._keep[rid.value] = (T.shape[0], k != 0)
        self._shape[rid.value] = (T.shape[0], k != 0)
        return rid.value

    def submit_product(self, reuse: int, x, dry_run_ms=0.0) -> int:
        """A product-only request: y = A x with the resident matrix that
        request `reuse` assembled."""
        nt, cplx = self._shape[reuse]
        X = np.ascontiguousarray(x, dtype=np.complex128 if cplx else np.float64)
        if X.shape != (nt,):
            raise ValueError("x must have one entry per triangle")
        q = Request(None, 0, None, nt, 0, 1.0 if cplx else 0.0, 1e-4, MIXED, 32, 1.2,
                    X.ctypes.data, float(dry_run_ms), int(reuse))
        rid = ctypes.c_int64()
        _check(load().bem_server_submit(self.handle, ctypes.byref(q), ctypes.byref(rid)))
        self._keep[rid.value] = (nt, cplx)
        self._shape[rid.value] = (nt, cplx)
        return rid.value

    def poll(self, rid: int) -> RequestInfo:
        info = RequestInfo()
        _check(load().bem_server_poll(self.handle, rid, ctypes.byref(info)))
        return info

    def wait(self, rid: int, timeout_ms: int = -1):
        """(status, info, y); status BEM_E_TIMEOUT (5) keeps the request."""
        nt, cplx = self._keep[rid]
        y = np.zeros(nt, dtype=np.complex128 if cplx else np.float64)
        info = RequestInfo()
        rc = load().bem_server_wait(self.handle, rid, int(timeout_ms), ctypes.byref(info),
                                    y.ctypes.data)
        if rc != 5:
            self._keep.pop(rid, None)
        return rc, info, y

    def cancel(self, rid: int) -> int:
        return load().bem_server_cancel(self.handle, rid)

    def stats(self) -> dict:
        s = ServerStats()
        _check(load().bem_server_stats_get(self.handle, ctypes.byref(s)))
        return {n: getattr(s, n) for n, _ in ServerStats._fields_}

    def close(self):
        if self.handle:
            load().bem_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
