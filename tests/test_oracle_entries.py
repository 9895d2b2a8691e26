"""Pins of the oracle's Galerkin entries (Eq. (1)-(3), (5); Sec. 3.2.3)
against closed forms, stored semi-analytic references and identities that
hold for the exact integrals."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1711_01897_gb300 import meshes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "singular_reference.json")


def _areas(V, T):
    a, b, c = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    return 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)


def test_triangle_potential_and_solid_angle_match_quadrature():
    rng = np.random.default_rng(5)
    s, t, w = oracle.triangle_rule_conical(40)
    for _ in range(5):
        tri = rng.normal(size=(3, 3))
        x = rng.normal(size=3) * 4.0
        e1, e2 = tri[1] - tri[0], tri[2] - tri[0]
        nn = np.cross(e1, e2)
        area = 0.5 * np.linalg.norm(nn)
        n = nn / np.linalg.norm(nn)
        y = tri[0] + s[:, None] * e1 + t[:, None] * e2
        d = x - y
        r = np.linalg.norm(d, axis=1)
        if r.min() < 1.0:
            continue
        assert abs(oracle.triangle_potential(tri, x) - area * np.sum(w / r)) < 1e-12
        assert abs(oracle.triangle_solid_angle(tri, x) - area * np.sum(w * (d @ n) / r ** 3)) < 1e-12


def test_solid_angle_of_closed_surface_is_minus_4pi_inside():
    """Sum of the solid-angle integrals over a closed outward mesh is 4 pi
    for an interior point and 0 outside (sign convention of Eq. (2))."""
    V, T = meshes.icosphere_level(1)
    tot_in = sum(oracle.triangle_solid_angle(V[t].reshape(9), [0.1, -0.2, 0.05]) for t in T)
    tot_out = sum(oracle.triangle_solid_angle(V[t].reshape(9), [1.5, 0.3, 0.2]) for t in T)
    # (x - y).n_y < 0 for x inside and outward n_y, so the integral is -4 pi
    assert abs(tot_in + 4 * np.pi) < 1e-12
    assert abs(tot_out) < 1e-12


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


@pytest.mark.parametrize("idx", range(11))
def test_singular_and_regular_entries_against_stored_references(idx):
    g = _golden()
    rec = g["values"][idx]
    ia, ib = g["pairs"][rec["pair"]]
    P = {int(k): v for k, v in g["points"].items()}
    a9 = [c for v in ia for c in P[v]]
    b9 = [c for v in ib for c in P[v]]
    ref = complex(rec["re"], rec["im"])
    # converged rule (12 GL points per axis, or a 20x20 regular rule)
    hi = oracle.pair_entry(a9, b9, ia, ib, rec["op"], rec["k"], n_gl=12, regular_order=20)
    assert abs(hi - ref) <= 2e-9 * abs(ref), (rec, hi)
    # the production rule (4 GL points per axis / 6-point Gauss) is accurate
    # to the level of a 4-point Gauss rule, and not better than 1e-12
    lo = oracle.pair_entry(a9, b9, ia, ib, rec["op"], rec["k"], n_gl=4, regular_order=0)
    rel = abs(lo - ref) / abs(ref)
    assert 1e-12 < rel < 1e-3, (rec, rel)


def test_reference_entry_live_vertex_pair():
    """One reference recomputed live (closed form + adaptive outer rule)."""
    g = _golden()
    rec = next(r for r in g["values"] if r["pair"] == "vertex" and r["op"] == 0 and r["k"] == 0)
    P = {int(k): v for k, v in g["points"].items()}
    ia, ib = g["pairs"]["vertex"]
    a9 = [c for v in ia for c in P[v]]
    b9 = [c for v in ib for c in P[v]]
    v = oracle.reference_entry(a9, b9, 0, 0.0, order=6, tol=1e-12, maxdepth=14)
    assert abs(v - complex(rec["re"], rec["im"])) < 1e-13


def test_coincident_double_layer_vanishes_on_flat_panels():
    V, T = meshes.icosphere_level(2)
    ids = np.arange(0, T.shape[0], 7, dtype=np.int32)
    for op in (oracle.DLP, oracle.ADLP):
        for k in (0.0, 3.0):
            d = np.array([oracle.entries(V, T, op, k, [i], [i])[0, 0] for i in ids])
            assert np.max(np.abs(d)) < 1e-25  # rounding of (y - x).n_y only


@pytest.fixture(scope="module")
def sphere_l3():
    return meshes.icosphere_level(3)


def test_single_layer_sphere_identity(sphere_l3):
    """On the unit sphere the single layer of the constant density 1 equals 1,
    so sum_j V_ij = |T_i| up to the flat-panel geometry error O(h^2)."""
    errs = []
    for level in (2, 3):
        V, T = meshes.icosphere_level(level)
        A = oracle.dense_matrix(V, T, oracle.SLP, 0.0)
        area = _areas(V, T)
        errs.append(np.max(np.abs(A.sum(1).real / area - 1.0)))
        assert np.max(np.abs(A.imag)) == 0.0
    assert errs[1] < 0.02 and errs[1] < errs[0] / 3.0, errs


@pytest.mark.parametrize("jit", [False, True])
def test_double_layer_jump_minus_half(jit):
    """For any closed flat polyhedron with outward normals the double layer
    of the constant 1 equals -1/2 on the faces, so sum_j K_ij = -|T_i|/2 up
    to quadrature error (row sums; column sums do not satisfy it)."""
    V, T = meshes.icosphere_level(2)
    if jit:
        V = meshes.jitter(V, T, 0.05, 7)
    area = _areas(V, T)
    K = oracle.dense_matrix(V, T, oracle.DLP, 0.0, n_gl=8, regular_order=8)
    assert np.max(np.abs(K.sum(1).real + area / 2) / area) < 1e-8
    assert np.max(np.abs(K.sum(0).real + area / 2) / area) > 1e-3
    K4 = oracle.dense_matrix(V, T, oracle.DLP, 0.0)
    assert np.max(np.abs(K4.sum(1).real + area / 2) / area) < 5e-5


def test_symmetry_and_adjoint(sphere_l3):
    V, T = meshes.icosphere_level(2)
    for k in (0.0, 2.5):
        S = oracle.dense_matrix(V, T, oracle.SLP, k)
        K = oracle.dense_matrix(V, T, oracle.DLP, k)
        Kp = oracle.dense_matrix(V, T, oracle.ADLP, k)
        # exact up to quadrature error for singular pairs, rounding otherwise
        assert np.max(np.abs(S - S.T)) <= 1e-4 * np.max(np.abs(S))
        assert np.max(np.abs(Kp - K.T)) <= 1e-4 * np.max(np.abs(K))
        # regular pairs: the tensor rule is symmetric up to rounding
        ids = np.arange(T.shape[0])
        shared = (T[:, None, :, None] == T[None, :, None, :]).any(axis=(2, 3))
        reg = ~shared
        assert np.max(np.abs((S - S.T)[reg])) <= 1e-15 * np.max(np.abs(S))
        assert np.max(np.abs((Kp - K.T)[reg])) <= 1e-14 * np.max(np.abs(K))
        del ids


def test_helmholtz_to_laplace_limit():
    """V_k - V_0 = i k |T_i||T_j| / (4 pi) + O(k^2) for every pair."""
    V, T = meshes.icosphere_level(1)
    area = _areas(V, T)
    ids = np.arange(T.shape[0], dtype=np.int32)
    S0 = oracle.entries(V, T, oracle.SLP, 0.0, ids, ids)
    lead = np.outer(area, area) / (4 * np.pi)
    res = []
    for k in (1e-3, 2e-3):
        Sk = oracle.entries(V, T, oracle.SLP, k, ids, ids)
        res.append(np.max(np.abs(Sk - S0 - 1j * k * lead)))
        assert np.max(np.abs((Sk - S0).imag / (k * lead) - 1.0)) < 1e-2
    assert 3.5 < res[1] / res[0] < 4.5


def test_helmholtz_sphere_eigenvalues(sphere_l3):
    """On the unit sphere the constant density is an eigenfunction:
    V_k 1 = e^{ik} sin(k)/k and K_k 1 = (i k^2/2)(j0 h0' + j0' h0)(k) with
    h0(z) = e^{iz}/(iz); the sums of the discrete rows match up to O(h^2)."""
    V, T = sphere_l3
    area = _areas(V, T)
    k = 1.5
    ids = np.arange(0, T.shape[0], 37, dtype=np.int32)
    allj = np.arange(T.shape[0], dtype=np.int32)
    S = oracle.entries(V, T, oracle.SLP, k, ids, allj)
    K = oracle.entries(V, T, oracle.DLP, k, ids, allj)
    lam_s = np.exp(1j * k) * np.sin(k) / k
    j0 = np.sin(k) / k
    j0p = np.cos(k) / k - np.sin(k) / k ** 2
    h0 = np.exp(1j * k) / (1j * k)
    h0p = np.exp(1j * k) / k - np.exp(1j * k) / (1j * k ** 2)
    lam_k = 0.5j * k ** 2 * (j0 * h0p + j0p * h0)
    es = np.abs(S.sum(1) / area[ids] - lam_s) / abs(lam_s)
    ek = np.abs(K.sum(1) / area[ids] - lam_k) / abs(lam_k)
    assert es.max() < 1e-2 and ek.max() < 2e-2, (es.max(), ek.max())
    # wrong-sign phase fails badly
    lam_bad = np.exp(-1j * k) * np.sin(k) / k
    assert np.min(np.abs(S.sum(1) / area[ids] - lam_bad)) / abs(lam_s) > 0.5
