"""Seeded synthetic surface meshes: the inputs of every test and benchmark.

This module generates inputs only.  It holds none of the boundary-element
arithmetic, so both the product library and the test oracle can be fed from
it.  The paper benchmarks on a unit sphere of flat triangles (Sec. 5.2);
these generators stand in for its meshes:

* ``icosphere(nu)``: class-I geodesic sphere of frequency ``nu`` (20 nu^2
  triangles): each icosahedron face is cut into a nu x nu triangular grid and
  every grid point is projected onto the unit sphere.  "Level L" means
  ``nu = 2**L`` (L3 = 1,280 triangles, L6 = 81,920, L9 = 5,242,880).
* ``ellipsoid(nu, axes)``: the same sphere scaled by the semi-axes.
* ``jitter(V, T, frac, seed)``: every vertex coordinate gets an independent
  offset, uniform in [-frac*h, +frac*h], h the mean edge length before
  jitter; the offsets come from the counter-based splitmix64 generator.

Triangles are counter-clockwise seen from outside, so the right-hand normal
points outwards.
"""
from __future__ import annotations

import numpy as np

_MASK = np.uint64(0xFFFFFFFFFFFFFFFF)


def _icosahedron():
    t = (1.0 + 5.0 ** 0.5) / 2.0
    V = np.array([(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t),
                  (0, -1, -t), (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)],
                 dtype=np.float64)
    V /= np.linalg.norm(V, axis=1)[:, None]
    F = np.array([(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9),
                  (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2),
                  (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10),
                  (8, 6, 7), (9, 8, 1)], dtype=np.int64)
    # orient every face outwards (right-hand normal along the centroid)
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    flip = np.einsum("ij,ij->i", np.cross(b - a, c - a), a + b + c) < 0
    F[flip] = F[flip][:, [0, 2, 1]]
    return V, F


def icosphere(nu: int):
    """Geodesic unit sphere of frequency nu; returns (vertices f64 [n_v,3],
    triangles i32 [20 nu^2, 3])."""
    if nu < 1 or nu > 2047:
        raise ValueError("nu must be in [1, 2047]")
    C, F = _icosahedron()
    # grid points (i, j) of one face, weights (nu-i-j, i, j) on corners (A, B, C)
    ii, jj = np.meshgrid(np.arange(nu + 1), np.arange(nu + 1), indexing="ij")
    keep = ii + jj <= nu
    gi, gj = ii[keep], jj[keep]
    gw = np.stack([nu - gi - gj, gi, gj], axis=1)                     # [P, 3]
    loc = -np.ones((nu + 1, nu + 1), dtype=np.int64)
    loc[gi, gj] = np.arange(gi.size)
    P = gi.size
    corners = np.repeat(F[:, None, :], P, axis=1)                     # [20, P, 3]
    weights = np.broadcast_to(gw[None], (20, P, 3)).copy()
    # canonical key: (corner, weight) pairs sorted by corner, zero weights last
    cs = np.where(weights > 0, corners, 99)
    order = np.argsort(cs, axis=2, kind="stable")
    cs = np.take_along_axis(cs, order, axis=2)
    ws = np.take_along_axis(weights, order, axis=2)
    code = np.where(ws > 0, (cs + 1) * 4096 + ws, 0).astype(np.int64)  # 16+12 bits per slot
    key = (code[..., 0] << 34) | (code[..., 1] << 17) | code[..., 2]
    uniq, first, inv = np.unique(key.ravel(), return_index=True, return_inverse=True)
    cflat, wflat = cs.reshape(-1, 3)[first], ws.reshape(-1, 3)[first]
    pos = np.zeros((uniq.size, 3))
    for s in range(3):                       # sum in canonical (sorted) order
        valid = wflat[:, s] > 0
        pos[valid] += wflat[valid, s, None] * C[cflat[valid, s]]
    pos /= nu
    pos /= np.linalg.norm(pos, axis=1)[:, None]
    gid = inv.reshape(20, P)
    # triangles of one face in local grid indices
    up_i, up_j = np.nonzero((ii + jj <= nu - 1))
    tri_up = np.stack([loc[up_i, up_j], loc[up_i + 1, up_j], loc[up_i, up_j + 1]], axis=1)
    dn_i, dn_j = np.nonzero((ii + jj <= nu - 2))
    tri_dn = np.stack([loc[dn_i + 1, dn_j], loc[dn_i + 1, dn_j + 1], loc[dn_i, dn_j + 1]], axis=1)
    local = np.concatenate([tri_up, tri_dn], axis=0)                  # [nu^2, 3]
    T = gid[:, local].reshape(-1, 3)
    return pos, T.astype(np.int32)


def icosphere_level(level: int):
    return icosphere(2 ** level)


def ellipsoid(nu: int, semi_axes=(5.0, 0.5, 0.5)):
    V, T = icosphere(nu)
    return V * np.asarray(semi_axes, dtype=np.float64)[None, :], T


def edges(T) -> np.ndarray:
    T = np.asarray(T, dtype=np.int64)
    e = np.concatenate([T[:, [0, 1]], T[:, [1, 2]], T[:, [2, 0]]], axis=0)
    e.sort(axis=1)
    return np.unique(e, axis=0)


def mean_edge_length(V, T) -> float:
    e = edges(T)
    return float(np.linalg.norm(V[e[:, 0]] - V[e[:, 1]], axis=1).mean())


def mean_longest_edge(V, T) -> float:
    T = np.asarray(T, dtype=np.int64)
    a, b, c = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    L = np.stack([np.linalg.norm(b - a, axis=1), np.linalg.norm(c - b, axis=1),
                  np.linalg.norm(a - c, axis=1)], axis=1)
    return float(L.max(axis=1).mean())


def splitmix64(counter) -> np.ndarray:
    """splitmix64 output for each 64-bit counter value (Steele, Lea, Flood 2014)."""
    z = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z + np.uint64(0x9E3779B97F4A7C15)) & _MASK
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _MASK
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _MASK
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int) -> np.ndarray:
    """n uniforms in [0,1) from counters seed * 2^32 + 0..n-1."""
    ctr = np.uint64(seed) * np.uint64(1 << 32) + np.arange(n, dtype=np.uint64)
    return (splitmix64(ctr) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def jitter(V, T, frac: float, seed: int):
    """Offsets every vertex coordinate by U[-frac*h, frac*h], h = mean edge
    length of the unjittered mesh."""
    h = mean_edge_length(V, T)
    u = uniform01(seed, V.size).reshape(V.shape)
    return V + (2.0 * u - 1.0) * frac * h


def workload_mesh(name: str):
    """Meshes of the benchmark workloads (seed = 1000 + workload index)."""
    if name == "sphere_l3":
        return icosphere_level(3)
    if name == "sphere_l6_jitter":
        V, T = icosphere_level(6)
        return jitter(V, T, 0.05, 1001), T
    if name == "ellipsoid_nu158":
        return ellipsoid(158)
    if name == "sphere_l9":
        return icosphere_level(9)
    raise KeyError(name)


def helmholtz_k_10_per_wavelength(V, T) -> float:
    """k = 2 pi / (10 h) with h the mean longest triangle edge."""
    return 2.0 * np.pi / (10.0 * mean_longest_edge(V, T))
