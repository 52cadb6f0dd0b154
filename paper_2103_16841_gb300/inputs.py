"""Seeded synthetic inputs: space-time meshes and Dirichlet-data parameters.

This module holds no arithmetic of the boundary element method itself. It
produces plain arrays (vertex coordinates, connectivity, time nodes, data
parameters) that are handed unchanged both to the CUDA path and to the CPU
oracle, so the two never share code beyond their inputs.

Meshes follow the setting of Sec. 3 of the paper: the lateral boundary
Sigma = (0,T) x Gamma is split into open tetrahedra ("panels"), each flat in
Gamma_K x R for a flat spatial triangle K. The paper builds such meshes with an
algorithm it does not print; here every prism K x [t_n, t_{n+1}] is split
into three tetrahedra by the sorted-vertex-id rule, which makes neighbouring
prisms conforming (each quadrilateral side is cut along the diagonal that
joins the upper node of the smaller id to the lower node of the larger id).

Random numbers come from SplitMix64 (Steele, Lea, Flood 2014), used as a
counter-based generator: draw k of stream `seed` is mix(seed + (k+1)*gamma).
Seeds: 1 mesh time jitter, 2 data directions and centres, 3 ellipsoid axes,
4 serving traces.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Draws offset..offset+n-1 of the SplitMix64 stream `seed` (uint64)."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed) + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def gaussian(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Standard normal samples by Box-Muller on pairs of uniforms."""
    u = uniform(seed, 2 * n, 2 * offset)
    u1 = 1.0 - u[0::2]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


# ---------------------------------------------------------------------------
# spatial surfaces
# ---------------------------------------------------------------------------

def icosahedron():
    p = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array([[-1, p, 0], [1, p, 0], [-1, -p, 0], [1, -p, 0],
                  [0, -1, p], [0, 1, p], [0, -1, -p], [0, 1, -p],
                  [p, 0, -1], [p, 0, 1], [-p, 0, -1], [-p, 0, 1]], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                  [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                  [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                  [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int32)
    return v, f


def icosphere(level: int):
    """Unit icosphere: 20*4^level flat triangles, 10*4^level+2 vertices on S^2."""
    v, f = icosahedron()
    verts = [tuple(x) for x in v]
    for _ in range(level):
        cache = {}
        nf = []

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                m = (np.array(verts[a]) + np.array(verts[b])) * 0.5
                m /= np.linalg.norm(m)
                cache[key] = len(verts)
                verts.append(tuple(m))
            return cache[key]

        for a, b, c in f:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        f = np.array(nf, dtype=np.int32)
    return np.array(verts, dtype=np.float64), f


def ellipsoid(level: int, axes):
    v, f = icosphere(level)
    return v * np.asarray(axes, dtype=np.float64)[None, :], f


# ---------------------------------------------------------------------------
# space-time prism meshes
# ---------------------------------------------------------------------------

def time_nodes(n_vtx: int, n_slabs: int, T: float, jitter: float = 0.0, seed: int = 1):
    """Per-vertex time nodes t[v, n], n = 0..n_slabs.

    t[v, n] = n*dt + U(-jitter, jitter)*dt for interior n; t[v,0]=0 and
    t[v,n_slabs]=T are not jittered.
    """
    dt = T / n_slabs
    n = np.arange(n_slabs + 1, dtype=np.float64)
    t = np.tile(n * dt, (n_vtx, 1))
    if jitter > 0.0 and n_slabs > 1:
        u = uniform(seed, n_vtx * (n_slabs + 1)).reshape(n_vtx, n_slabs + 1)
        t[:, 1:n_slabs] += (2.0 * u[:, 1:n_slabs] - 1.0) * jitter * dt
    t[:, 0] = 0.0
    t[:, n_slabs] = T
    return t


class SpaceTimeMesh:
    """Plain arrays of a space-time tetrahedral mesh of Gamma x [0, T].

    svert   [n_sv, 3]  spatial vertices
    stv_sv  [n_stv]    spatial vertex of each space-time vertex
    stv_t   [n_stv]    time of each space-time vertex
    tets    [n_tet, 4] space-time vertex ids
    tri     [n_tri, 3] spatial triangles (for reference only)
    n_slabs, T
    """

    def __init__(self, svert, tri, tnodes, T):
        self.svert = np.ascontiguousarray(svert, dtype=np.float64)
        self.tri = np.ascontiguousarray(tri, dtype=np.int32)
        n_sv = self.svert.shape[0]
        ns = tnodes.shape[1] - 1
        self.n_slabs = ns
        self.T = float(T)
        self.tnodes = np.ascontiguousarray(tnodes, dtype=np.float64)
        self.stv_sv = np.repeat(np.arange(n_sv, dtype=np.int32), ns + 1)
        self.stv_t = self.tnodes.reshape(-1).copy()
        tets = []
        for a, b, c in np.sort(self.tri, axis=1):
            for n in range(ns):
                A0, B0, C0 = a * (ns + 1) + n, b * (ns + 1) + n, c * (ns + 1) + n
                A1, B1, C1 = A0 + 1, B0 + 1, C0 + 1
                tets += [(A0, B0, C0, A1), (B0, C0, A1, B1), (C0, A1, B1, C1)]
        self.tets = np.array(tets, dtype=np.int32).reshape(-1, 4)

    @property
    def n_tet(self):
        return self.tets.shape[0]

    def stv_xyzt(self):
        """[n_stv, 4] array of (t, x, y, z)."""
        out = np.empty((self.stv_t.shape[0], 4))
        out[:, 0] = self.stv_t
        out[:, 1:] = self.svert[self.stv_sv]
        return out


def prism_mesh(svert, tri, n_slabs, T, jitter=0.0, seed=1):
    t = time_nodes(svert.shape[0], n_slabs, T, jitter, seed)
    return SpaceTimeMesh(svert, tri, t, T)


def sphere_mesh(level, n_slabs, T, jitter=0.0, seed=1):
    v, f = icosphere(level)
    return prism_mesh(v, f, n_slabs, T, jitter, seed)


# ---------------------------------------------------------------------------
# Dirichlet data parameters
# ---------------------------------------------------------------------------

# Data families understood by both the library and the oracle:
#   0  SIN2_UNIFORM : g(t, x) = sin^2(pi t / 2) for 0 < t < 2, else 0
#   1  PULSE        : g(t, x) = exp(-((t - <x, d> - c) / w)^2), params (d0, d1, d2, c, w)
DATA_SIN2_UNIFORM = 0
DATA_PULSE = 1


def pulse_params(nrhs: int, seed: int = 2, c_range=(1.0, 2.0), width=0.25, fixed_c=None):
    """[nrhs, 5] rows (d0, d1, d2, c, w): seeded unit directions, centres U[c_range]."""
    g = gaussian(seed, 3 * nrhs).reshape(nrhs, 3)
    d = g / np.linalg.norm(g, axis=1, keepdims=True)
    if fixed_c is None:
        c = c_range[0] + (c_range[1] - c_range[0]) * uniform(seed + 100, nrhs)
    else:
        c = np.full(nrhs, float(fixed_c))
    out = np.empty((nrhs, 5))
    out[:, :3] = d
    out[:, 3] = c
    out[:, 4] = width
    return out


# ---------------------------------------------------------------------------
# the five workload shapes
# ---------------------------------------------------------------------------

def workload_c1():
    """Unit sphere, icosphere level 1, T=2, 4 uniform slabs: 960 tetrahedra."""
    return sphere_mesh(1, 4, 2.0, 0.0)


def workload_c2(seed=1):
    """Icosphere level 3, T=4, 32 slabs, +-20% interior jitter: 122,880 tetrahedra."""
    return sphere_mesh(3, 32, 4.0, 0.2, seed)


def scatterer_meshes(n, T=4.0, jitter=0.2, seed=3, only=None):
    """Space-time meshes and pulse parameters of n small ellipsoid scatterers
    (icosphere level 1 or 2 scaled by semi-axes in [0.5, 1.5], 8-16 slabs,
    1-4 pulse right-hand sides each); `only`: the indices to build."""
    out = []
    for k, (level, axes, slabs, nrhs) in enumerate(small_scatterers(n, seed)):
        if only is not None and k not in only:
            continue
        v, f = ellipsoid(level, axes)
        m = prism_mesh(v, f, slabs, T, jitter, seed=seed * 100003 + k)
        out.append((m, pulse_params(nrhs, seed=seed * 100019 + k)))
    return out


def small_scatterers(n, seed=3):
    """Shapes of n small ellipsoid scatterers: (level, axes, slabs, nrhs) each."""
    u = uniform(seed, 6 * n).reshape(n, 6)
    out = []
    for k in range(n):
        level = 1 + int(u[k, 0] * 2.0)
        axes = 0.5 + u[k, 1:4]
        slabs = 8 + int(u[k, 4] * 9.0)
        nrhs = 1 + int(u[k, 5] * 4.0)
        out.append((level, axes, slabs, nrhs))
    return out
