"""FP64 CPU oracle for P0 Galerkin BEM entries, the block partition, ACA and
the H-matrix product (Vater, Betcke, Dilba, arXiv 1711.01897).

TEST INFRASTRUCTURE ONLY.  This package checks the CUDA path; it is not part
of it.  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import it.  It shares no code with the product library:
the arithmetic lives in ``bem_oracle.c`` (plain C, FP64), this module only
marshals numpy arrays and strings the per-block results together.

Every function cites the passage it follows.  Pins live in
``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bem_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")

SLP, DLP, ADLP = 0, 1, 2
# regular-rule codes (``regular_order``): the 6-point degree-4 rule, the
# 3-point degree-2 rule and the centroid rule; points per triangle of each
RULE6, RULE3, RULE1 = 0, -3, -1
RULE_POINTS = {RULE6: 6, RULE3: 3, RULE1: 1}
P0, DP1, P1 = 0, 1, 2
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            P = ctypes.c_void_p
            i32, i64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
            L.orc_gauss_legendre01.argtypes = [ctypes.c_int, P, P]
            L.orc_triangle_rule_deg4.argtypes = [P, P, P]
            L.orc_triangle_rule_conical.argtypes = [ctypes.c_int, P, P, P]
            L.orc_ss_moment.argtypes = [ctypes.c_int] * 6
            L.orc_ss_moment.restype = dbl
            L.orc_entries.argtypes = [P, P, i64, ctypes.c_int, dbl, P, i64, P, i64, ctypes.c_int,
                                      ctypes.c_int, P, ctypes.c_int]
            L.orc_pair_entry.argtypes = [P, P, P, P, ctypes.c_int, dbl, ctypes.c_int, ctypes.c_int,
                                         P, P]
            L.orc_triangle_potential.argtypes = [P, P]
            L.orc_triangle_potential.restype = dbl
            L.orc_triangle_solid_angle.argtypes = [P, P]
            L.orc_triangle_solid_angle.restype = dbl
            L.orc_reference_entry.argtypes = [P, P, ctypes.c_int, dbl, ctypes.c_int, dbl,
                                              ctypes.c_int, P, P]
            L.orc_cluster_tree.argtypes = [P, P, i64, ctypes.c_int, P, P, P, P, P, P, P]
            L.orc_block_tree.argtypes = [P, P, P, dbl, P, P, P, i64, P]
            L.orc_aca_blocks.argtypes = [P, P, P, ctypes.c_int, i64, P, P, P, P, ctypes.c_int, dbl,
                                         dbl, P, P, P, P, P, P, P, P, P, ctypes.c_int]
            L.orc_block_rules.argtypes = [P, P, P, i64, P, P, P, P, P, P, dbl, dbl, P]
            L.orc_triangle_rule_deg2.argtypes = [P, P, P]
            L.orc_triangle_rule_deg1.argtypes = [P, P, P]
            L.orc_entries_dp1.argtypes = [P, P, i64, ctypes.c_int, dbl, P, i64, P, i64,
                                          ctypes.c_int, ctypes.c_int, P, ctypes.c_int]
            L.orc_pair_local.argtypes = [P, P, P, P, ctypes.c_int, dbl, ctypes.c_int, ctypes.c_int,
                                         P]
            L.orc_aca_dense.argtypes = [P, i64, i64, dbl, ctypes.c_int, P, P, P]
            L.orc_num_threads.restype = ctypes.c_int
            _lib = L
            del i32
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(lib().orc_num_threads())


# --------------------------------------------------------------------------
# Quadrature (Sec. 3.2.1: six-point symmetric Gauss triangle rule of order 4;
# Sec. 3.2.3: Erichsen-Sauter scheme, Gauss-Legendre factors)
# --------------------------------------------------------------------------

def gauss_legendre01(n: int):
    x, w = np.zeros(n), np.zeros(n)
    if lib().orc_gauss_legendre01(n, _p(x), _p(w)):
        raise ValueError("n out of range")
    return x, w


def triangle_rule_deg4():
    s, t, w = np.zeros(6), np.zeros(6), np.zeros(6)
    lib().orc_triangle_rule_deg4(_p(s), _p(t), _p(w))
    return s, t, w


def triangle_rule_deg2():
    """The 3-point degree-2 rule (s, t, w) of the middle distance class."""
    s, t, w = (np.zeros(3) for _ in range(3))
    lib().orc_triangle_rule_deg2(_p(s), _p(t), _p(w))
    return s, t, w


def triangle_rule_deg1():
    """The centroid rule (s, t, w) of the farthest distance class."""
    s, t, w = (np.zeros(1) for _ in range(3))
    lib().orc_triangle_rule_deg1(_p(s), _p(t), _p(w))
    return s, t, w


def triangle_rule_conical(n: int):
    s, t, w = np.zeros(n * n), np.zeros(n * n), np.zeros(n * n)
    lib().orc_triangle_rule_conical(n, _p(s), _p(t), _p(w))
    return s, t, w


def ss_moment(ncase: int, n: int, a: int, b: int, c: int, d: int) -> float:
    """Sum over Sauter-Schwab regions of the [0,1]^4 GL integral of
    J * x1^a x2^b y1^c y2^d (ncase: 3 identical, 2 edge, 1 vertex)."""
    return float(lib().orc_ss_moment(ncase, n, a, b, c, d))


# --------------------------------------------------------------------------
# Entries (Eq. (1)-(3), Eq. (5); Sec. 3.2.3)
# --------------------------------------------------------------------------

def _mesh_arrays(V, T):
    V = np.ascontiguousarray(V, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.int32)
    return V, T


def entries(V, T, op: int, k: float, test_ids, trial_ids, n_gl: int = 4,
            regular_order: int = 0, nthreads: int = 0) -> np.ndarray:
    """Dense sub-block A[test_ids][:, trial_ids] (complex128).  Regular pairs
    use the 6-point rule (regular_order <= 0) or a conical n x n rule; pairs
    sharing a vertex use Sauter-Schwab with n_gl GL points per axis."""
    V, T = _mesh_arrays(V, T)
    ti = np.ascontiguousarray(test_ids, dtype=np.int32)
    tj = np.ascontiguousarray(trial_ids, dtype=np.int32)
    out = np.zeros((ti.size, tj.size), dtype=np.complex128)
    if ti.size and tj.size:
        lib().orc_entries(_p(V), _p(T), T.shape[0], op, float(k), _p(ti), ti.size, _p(tj),
                          tj.size, n_gl, regular_order, _p(out), nthreads)
    return out


def dense_matrix(V, T, op: int, k: float, **kw) -> np.ndarray:
    n = np.asarray(T).shape[0]
    ids = np.arange(n, dtype=np.int32)
    return entries(V, T, op, k, ids, ids, **kw)


def pair_entry(a9, b9, ia, ib, op: int, k: float, n_gl: int = 4, regular_order: int = 0) -> complex:
    a9 = np.ascontiguousarray(a9, dtype=np.float64).reshape(9)
    b9 = np.ascontiguousarray(b9, dtype=np.float64).reshape(9)
    ia = np.ascontiguousarray(ia, dtype=np.int32)
    ib = np.ascontiguousarray(ib, dtype=np.int32)
    re, im = ctypes.c_double(), ctypes.c_double()
    lib().orc_pair_entry(_p(a9), _p(b9), _p(ia), _p(ib), op, float(k), n_gl, regular_order,
                         ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


# --------------------------------------------------------------------------
# Piecewise linear spaces (Sec. 3.3: local dofs of each element pair; Sec.
# 3.2.3 "Global matrix assembly": contributions summed into global dofs)
# --------------------------------------------------------------------------

def entries_dp1(V, T, op: int, k: float, test_tris, trial_tris, n_gl: int = 4,
                regular_order: int = 0, nthreads: int = 0) -> np.ndarray:
    """DP1 sub-block (complex128, 3 n_test x 3 n_trial): row 3a + alpha, column
    3b + beta holds the local entry (alpha, beta) of the pair (test_tris[a],
    trial_tris[b]); local basis functions are the barycentric coordinates of
    the stored vertices."""
    V, T = _mesh_arrays(V, T)
    ti = np.ascontiguousarray(test_tris, dtype=np.int32)
    tj = np.ascontiguousarray(trial_tris, dtype=np.int32)
    out = np.zeros((3 * ti.size, 3 * tj.size), dtype=np.complex128)
    if ti.size and tj.size:
        lib().orc_entries_dp1(_p(V), _p(T), T.shape[0], op, float(k), _p(ti), ti.size, _p(tj),
                              tj.size, n_gl, regular_order, _p(out), nthreads)
    return out


def dense_matrix_dp1(V, T, op: int, k: float, **kw) -> np.ndarray:
    n = np.asarray(T).shape[0]
    ids = np.arange(n, dtype=np.int32)
    return entries_dp1(V, T, op, k, ids, ids, **kw)


def pair_local(a9, b9, ia, ib, op: int, k: float, n_gl: int = 4,
               regular_order: int = 0) -> np.ndarray:
    """3 x 3 local matrix of an explicit triangle pair."""
    a9 = np.ascontiguousarray(a9, dtype=np.float64).reshape(9)
    b9 = np.ascontiguousarray(b9, dtype=np.float64).reshape(9)
    ia = np.ascontiguousarray(ia, dtype=np.int32)
    ib = np.ascontiguousarray(ib, dtype=np.int32)
    out = np.zeros(9, dtype=np.complex128)
    lib().orc_pair_local(_p(a9), _p(b9), _p(ia), _p(ib), op, float(k), n_gl, regular_order,
                         _p(out))
    return out.reshape(3, 3)


def assemble_p1(T, n_vertices: int, local: np.ndarray) -> np.ndarray:
    """Global assembly of element-pair contributions into continuous P1 dofs:
    A[u, v] = sum over pairs (i, j), local a, b with T[i, a] = u, T[j, b] = v
    of local[3i + a, 3j + b] (Sec. 3.2.3, "Global matrix assembly": the raw
    element results are added to the global degrees of freedom)."""
    T = np.asarray(T)
    dof = T.reshape(-1)
    A = np.zeros((n_vertices, n_vertices), dtype=local.dtype)
    for a in range(dof.size):
        np.add.at(A[dof[a]], dof, local[a])
    return A


def dense_matrix_p1(V, T, op: int, k: float, **kw) -> np.ndarray:
    """Continuous piecewise linear Galerkin matrix of op (Eq. (1)-(3) with
    hat functions as test and trial basis)."""
    return assemble_p1(T, np.asarray(V).shape[0], dense_matrix_dp1(V, T, op, k, **kw))


def surface_curls(V, T) -> np.ndarray:
    """curl_Gamma of each local basis function on its triangle, [nt, 3, 3]
    (triangle, local vertex, component): n x grad_Gamma lambda_a, with the
    surface gradient from the 2 x 2 metric of the edge vectors (the gradient
    g in the plane with g.(v1 - v0) = lambda_a(v1) - lambda_a(v0) and
    g.(v2 - v0) = lambda_a(v2) - lambda_a(v0))."""
    V = np.asarray(V, dtype=np.float64)
    T = np.asarray(T)
    P = V[T]
    E1, E2 = P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]
    n = np.cross(E1, E2)
    n /= np.linalg.norm(n, axis=1)[:, None]
    G = np.stack([np.einsum("ij,ij->i", E1, E1), np.einsum("ij,ij->i", E1, E2),
                  np.einsum("ij,ij->i", E2, E1), np.einsum("ij,ij->i", E2, E2)], 1).reshape(-1, 2, 2)
    Ginv = np.linalg.inv(G)
    # differences lambda_a(v1) - lambda_a(v0), lambda_a(v2) - lambda_a(v0)
    dl = np.array([[-1.0, -1.0], [1.0, 0.0], [0.0, 1.0]])
    out = np.zeros((T.shape[0], 3, 3))
    for a in range(3):
        c = np.einsum("tij,j->ti", Ginv, dl[a])          # coefficients on E1, E2
        grad = c[:, 0:1] * E1 + c[:, 1:2] * E2
        out[:, a] = np.cross(n, grad)
    return out


def hypersingular_p1(V, T, k: float, **kw) -> np.ndarray:
    """Hypersingular operator on continuous P1 by its weak form, Eq. (4):
    D[u, v] = sum over element pairs of
        curl phi_u . curl phi_v  int int g  -  k^2 n_x . n_y  int int phi_u g phi_v,
    the first integral the P0 single-layer entry of the pair (the curls are
    constant per triangle), the second the local P1 single-layer entry."""
    V = np.asarray(V, dtype=np.float64)
    T = np.asarray(T)
    nt = T.shape[0]
    ids = np.arange(nt, dtype=np.int32)
    S0 = entries(V, T, SLP, k, ids, ids, **kw)                  # [nt, nt]
    S1 = dense_matrix_dp1(V, T, SLP, k, **kw)                    # [3nt, 3nt]
    C = surface_curls(V, T).reshape(3 * nt, 3)                   # row 3t + a
    P = V[T]
    n = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    n /= np.linalg.norm(n, axis=1)[:, None]
    tri = np.repeat(np.arange(nt), 3)
    local = (C @ C.T) * S0[np.ix_(tri, tri)]
    if k != 0.0:
        local = local - k * k * (n[tri] @ n[tri].T) * S1
    return assemble_p1(T, V.shape[0], local)


def _vertex_dofs(T, verts):
    """For each vertex, the (triangle, local index) pairs of its DP1 dofs."""
    T = np.asarray(T)
    out = []
    for v in verts:
        t, a = np.nonzero(T == v)
        out.append((t.astype(np.int32), a))
    return out


def p1_rows(V, T, op: int, k: float, verts, **kw) -> np.ndarray:
    """Rows `verts` of the continuous P1 matrix of op (global assembly of the
    local matrices, Sec. 3.2.3), [len(verts), n_vertices] complex128."""
    V = np.asarray(V, dtype=np.float64)
    T = np.asarray(T)
    nt, nv = T.shape[0], V.shape[0]
    allt = np.arange(nt, dtype=np.int32)
    cols = T.reshape(-1)                      # DP1 dof 3t + b -> vertex
    out = np.zeros((len(verts), nv), dtype=np.complex128)
    for r, (tris, loc) in enumerate(_vertex_dofs(T, verts)):
        A = entries_dp1(V, T, op, k, tris, allt, **kw)       # [3 len(tris), 3 nt]
        row = A[3 * np.arange(tris.size) + loc].sum(axis=0)
        np.add.at(out[r], cols, row)
    return out


def hypersingular_p1_rows(V, T, k: float, verts, **kw) -> np.ndarray:
    """Rows `verts` of the hypersingular P1 matrix by the weak form, Eq. (4)
    (as hypersingular_p1), [len(verts), n_vertices] complex128."""
    V = np.asarray(V, dtype=np.float64)
    T = np.asarray(T)
    nt, nv = T.shape[0], V.shape[0]
    allt = np.arange(nt, dtype=np.int32)
    C = surface_curls(V, T)                                   # [nt, 3, 3]
    P = V[T]
    n = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    n /= np.linalg.norm(n, axis=1)[:, None]
    cols = T.reshape(-1)
    out = np.zeros((len(verts), nv), dtype=np.complex128)
    for r, (tris, loc) in enumerate(_vertex_dofs(T, verts)):
        S0 = entries(V, T, SLP, k, tris, allt, **kw)          # [len(tris), nt]
        row = np.zeros(3 * nt, dtype=np.complex128)
        for q in range(tris.size):
            cu = C[tris[q], loc[q]]                          # curl of phi_u on this triangle
            row += (np.repeat(S0[q], 3) * (C.reshape(3 * nt, 3) @ cu))
        if k != 0.0:
            S1 = entries_dp1(V, T, SLP, k, tris, allt, **kw)
            for q in range(tris.size):
                nn = np.repeat(n @ n[tris[q]], 3)
                row -= k * k * nn * S1[3 * q + loc[q]]
        np.add.at(out[r], cols, row)
    return out


def mass_p1(V, T) -> np.ndarray:
    """P1 mass matrix M[u, v] = int phi_u phi_v (exact: |T|/12 (1 + delta_ab))."""
    V = np.asarray(V, dtype=np.float64)
    T = np.asarray(T)
    P = V[T]
    area = 0.5 * np.linalg.norm(np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), axis=1)
    M = np.zeros((V.shape[0], V.shape[0]))
    loc = (np.ones((3, 3)) + np.eye(3)) / 12.0
    for a in range(3):
        for b in range(3):
            np.add.at(M, (T[:, a], T[:, b]), area * loc[a, b])
    return M


def triangle_potential(tri9, x) -> float:
    tri9 = np.ascontiguousarray(tri9, dtype=np.float64).reshape(9)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(3)
    return float(lib().orc_triangle_potential(_p(tri9), _p(x)))


def triangle_solid_angle(tri9, x) -> float:
    tri9 = np.ascontiguousarray(tri9, dtype=np.float64).reshape(9)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(3)
    return float(lib().orc_triangle_solid_angle(_p(tri9), _p(x)))


def reference_entry(a9, b9, op: int, k: float = 0.0, order: int = 6, tol: float = 1e-12,
                    maxdepth: int = 12) -> complex:
    """Entry by closed-form inner integral plus adaptive outer quadrature
    (and nested adaptive quadrature of the bounded Helmholtz remainder).
    Independent of the Gauss and Sauter-Schwab rules; for the pins only."""
    a9 = np.ascontiguousarray(a9, dtype=np.float64).reshape(9)
    b9 = np.ascontiguousarray(b9, dtype=np.float64).reshape(9)
    re, im = ctypes.c_double(), ctypes.c_double()
    r = lib().orc_reference_entry(_p(a9), _p(b9), op, float(k), order, tol, maxdepth,
                                  ctypes.byref(re), ctypes.byref(im))
    if r:
        raise ValueError("reference_entry supports SLP and DLP")
    return complex(re.value, im.value)


# --------------------------------------------------------------------------
# Cluster tree, block tree (Sec. 2.1; Algorithm "H-Matrix Assembly", Sec. 4.1)
# --------------------------------------------------------------------------

@dataclass
class ClusterTree:
    perm: np.ndarray
    begin: np.ndarray
    end: np.ndarray
    left: np.ndarray
    right: np.ndarray
    box: np.ndarray

    @property
    def n_clusters(self) -> int:
        return self.begin.size


def cluster_tree(V, T, leaf_size: int) -> ClusterTree:
    V, T = _mesh_arrays(V, T)
    nt = T.shape[0]
    cap = 2 * nt + 1
    perm = np.zeros(nt, dtype=np.int32)
    b, e, l, r = (np.zeros(cap, dtype=np.int64) for _ in range(4))
    box = np.zeros((cap, 6))
    nc = ctypes.c_int64()
    if lib().orc_cluster_tree(_p(V), _p(T), nt, leaf_size, _p(perm), _p(b), _p(e), _p(l), _p(r),
                              _p(box), ctypes.byref(nc)):
        raise ValueError("bad cluster tree arguments")
    n = nc.value
    return ClusterTree(perm, b[:n].copy(), e[:n].copy(), l[:n].copy(), r[:n].copy(),
                       box[:n].copy())


@dataclass
class BlockTree:
    tau: np.ndarray
    sigma: np.ndarray
    adm: np.ndarray


def block_tree(ct: ClusterTree, eta: float) -> BlockTree:
    cap = 4 * ct.n_clusters * 8 + 64
    while True:
        bt, bs = np.zeros(cap, dtype=np.int64), np.zeros(cap, dtype=np.int64)
        ba = np.zeros(cap, dtype=np.int8)
        nb = ctypes.c_int64()
        r = lib().orc_block_tree(_p(ct.left), _p(ct.right), _p(np.ascontiguousarray(ct.box)),
                                 float(eta), _p(bt), _p(bs), _p(ba), cap, ctypes.byref(nb))
        if r == 0:
            n = nb.value
            return BlockTree(bt[:n].copy(), bs[:n].copy(), ba[:n].astype(bool))
        cap *= 4


# --------------------------------------------------------------------------
# ACA (Sec. 2.1, Eq. (6)-(7), Algorithm ACA)
# --------------------------------------------------------------------------

def aca_dense(A: np.ndarray, eps: float, kcap: int | None = None):
    """ACA with partial pivoting on an explicit matrix; returns U (m x k),
    V (n x k) with A ~ U V^T."""
    A = np.asarray(A, dtype=np.complex128)
    m, n = A.shape
    kcap = min(m, n) if kcap is None else kcap
    Af = np.asfortranarray(A)
    U = np.zeros((kcap, m), dtype=np.complex128)
    Vf = np.zeros((kcap, n), dtype=np.complex128)
    rank = ctypes.c_int()
    lib().orc_aca_dense(_p(Af), m, n, float(eps), kcap, _p(U), _p(Vf), ctypes.byref(rank))
    k = rank.value
    return U[:k].T.copy(), Vf[:k].T.copy()


@dataclass
class HMatrix:
    """Oracle H-matrix: near blocks dense, admissible blocks as U V^T, all in
    cluster order.  ``blocks`` rows: (tau_begin, tau_end, sig_begin, sig_end,
    admissible)."""
    n: int
    perm: np.ndarray
    blocks: np.ndarray
    near: dict = field(default_factory=dict)
    far: dict = field(default_factory=dict)
    ranks: dict = field(default_factory=dict)
    entries_evaluated: int = 0
    rules: np.ndarray | None = None

    def matvec(self, x: np.ndarray) -> np.ndarray:
        """y = P (Near x~ + sum_b U_b (V_b^T x~_sigma)), x~ = x in cluster
        order (the product the assembled H-matrix represents)."""
        x = np.asarray(x)
        xt = x[self.perm]
        yt = np.zeros(self.n, dtype=np.complex128)
        for b, (tb, te, sb, se, adm) in enumerate(self.blocks):
            if adm:
                U, Vv = self.far[b]
                if U.shape[1]:
                    yt[tb:te] += U @ (Vv.T @ xt[sb:se])
            else:
                yt[tb:te] += self.near[b] @ xt[sb:se]
        y = np.zeros_like(yt)
        y[self.perm] = yt
        return y

    def block_dense(self, b: int) -> np.ndarray:
        tb, te, sb, se, adm = self.blocks[b]
        if adm:
            U, Vv = self.far[b]
            return U @ Vv.T
        return self.near[b]


def block_list(ct: ClusterTree, bt: BlockTree) -> np.ndarray:
    return np.stack([ct.begin[bt.tau], ct.end[bt.tau], ct.begin[bt.sigma], ct.end[bt.sigma],
                     bt.adm.astype(np.int64)], axis=1)


def block_rules(V, T, ct: ClusterTree, bt: BlockTree, blocks: np.ndarray, rho3: float,
                rho1: float) -> np.ndarray:
    """Regular-rule code of every block (quadrature order per block distance
    class): admissible blocks by rho = dist(tau, sigma) / h (box distance over
    the longest triangle edge in tau or sigma) against the thresholds (0 =
    class unused), near blocks RULE6."""
    V, T = _mesh_arrays(V, T)
    n = blocks.shape[0]
    rules = np.zeros(n, dtype=np.int32)
    adm = np.flatnonzero(blocks[:, 4])
    if adm.size and (rho3 > 0 or rho1 > 0):
        tb, te, sb, se = (np.ascontiguousarray(blocks[adm, c]) for c in range(4))
        bx_t = np.ascontiguousarray(ct.box[bt.tau[adm]])
        bx_s = np.ascontiguousarray(ct.box[bt.sigma[adm]])
        out = np.zeros(adm.size, dtype=np.int32)
        lib().orc_block_rules(_p(V), _p(T), _p(ct.perm), adm.size, _p(tb), _p(te), _p(sb), _p(se),
                              _p(bx_t), _p(bx_s), float(rho3), float(rho1), _p(out))
        rules[adm] = out
    return rules


def hmat_assemble(V, T, op: int, k: float, leaf_size: int, eta: float, eps: float,
                  n_gl: int = 4, kcap_max: int = 256, nthreads: int = 0,
                  block_ids=None, space: int = P0, rho3: float = 0.0,
                  rho1: float = 0.0) -> HMatrix:
    """Algorithm "H-Matrix Assembly" (Sec. 4.1): generate the block cluster
    tree, evaluate inadmissible blocks densely, approximate admissible blocks
    by ACA.  block_ids restricts the work to a subset of leaf blocks.

    space=DP1: the same triangle cluster and block trees, each triangle
    carrying its three local dofs (cluster position t -> dofs 3t, 3t+1,
    3t+2), so every block is the tripled dof block; ``perm`` and ``blocks``
    are then in dof units.

    rho3, rho1 > 0 (P0 only): admissible blocks with dist / h >= rho1 use
    the centroid rule, else >= rho3 the 3-point rule, else the 6-point rule
    (``block_rules``); ``rules`` records the code of every block."""
    V, T = _mesh_arrays(V, T)
    ct = cluster_tree(V, T, leaf_size)
    bt = block_tree(ct, eta)
    blocks = block_list(ct, bt)
    perm = ct.perm
    if space != P0 and (rho3 > 0 or rho1 > 0):
        raise ValueError("per-class regular rules are defined for P0 only")
    rules = block_rules(V, T, ct, bt, blocks, rho3, rho1)
    if space == DP1:
        dof_perm = (3 * perm[:, None] + np.arange(3)[None, :]).reshape(-1).astype(np.int32)
        dblocks = blocks.copy()
        dblocks[:, :4] *= 3
        hm = HMatrix(n=3 * T.shape[0], perm=dof_perm, blocks=dblocks)
    else:
        hm = HMatrix(n=T.shape[0], perm=perm, blocks=blocks)
    hm.rules = rules
    sel = np.arange(blocks.shape[0]) if block_ids is None else np.asarray(block_ids)
    far_ids = [b for b in sel if blocks[b, 4]]
    near_ids = [b for b in sel if not blocks[b, 4]]
    for b in near_ids:
        tb, te, sb, se, _ = blocks[b]
        if space == DP1:
            hm.near[b] = entries_dp1(V, T, op, k, perm[tb:te], perm[sb:se], n_gl=n_gl,
                                     nthreads=nthreads)
            hm.entries_evaluated += 9 * (te - tb) * (se - sb)
        else:
            hm.near[b] = entries(V, T, op, k, perm[tb:te], perm[sb:se], n_gl=n_gl,
                                 nthreads=nthreads)
            hm.entries_evaluated += (te - tb) * (se - sb)
    chunk = 2048
    for c0 in range(0, len(far_ids), chunk):
        ids = np.array(far_ids[c0:c0 + chunk], dtype=np.int64)
        tb, te, sb, se = (np.ascontiguousarray(hm.blocks[ids, c]) for c in range(4))
        m, n = te - tb, se - sb
        kc = np.minimum(np.minimum(m, n), kcap_max).astype(np.int32)
        uoff = np.concatenate([[0], np.cumsum(m * kc)[:-1]]).astype(np.int64)
        voff = np.concatenate([[0], np.cumsum(n * kc)[:-1]]).astype(np.int64)
        U = np.zeros(int((m * kc).sum()), dtype=np.complex128)
        Vf = np.zeros(int((n * kc).sum()), dtype=np.complex128)
        rank = np.zeros(ids.size, dtype=np.int32)
        status = np.zeros(ids.size, dtype=np.int32)
        ev = np.zeros(ids.size, dtype=np.int64)
        rl = np.ascontiguousarray(rules[ids])
        lib().orc_aca_blocks(_p(V), _p(T), _p(perm), int(space), ids.size, _p(tb), _p(te), _p(sb), _p(se), op,
                             float(k), float(eps), _p(kc), _p(rl), _p(uoff), _p(voff), _p(U), _p(Vf),
                             _p(rank), _p(status), _p(ev), nthreads)
        if np.any(status == 3):
            raise MemoryError("oracle ACA allocation failed")
        for q, b in enumerate(ids):
            r = int(rank[q])
            Ub = U[uoff[q]:uoff[q] + m[q] * r].reshape(r, m[q]).T.copy()
            Vb = Vf[voff[q]:voff[q] + n[q] * r].reshape(r, n[q]).T.copy()
            hm.far[int(b)] = (Ub, Vb)
            hm.ranks[int(b)] = r
        hm.entries_evaluated += int(ev.sum())
    return hm
