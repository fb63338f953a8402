"""Seeded synthetic inputs shared by the CUDA path, its tests and the benchmark.

This module generates *inputs only*: tetrahedral meshes of the cube [-1/2, 1/2]^3,
per-element materials, source and receiver locations and random states.  It holds none
of the Bernstein-Bezier DG arithmetic (no basis, operator, flux or time-stepping code),
so both the CUDA path and the CPU oracle may consume what it produces.

Mesh recipe (the paper's experiments run on tetrahedral meshes of the cube
[-.5, .5]^3, Section 4.1, with K = 1536 and K = 98304 elements, Section 4.3):
  * n^3 hexahedra of width h = 1/n, each split into 6 tetrahedra along the main
    diagonal (0,0,0)->(1,1,1) (Kuhn/Freudenthal split; the same diagonal in every hex
    makes the mesh conforming);
  * each tetrahedron is listed with a positive orientation (det > 0);
  * optional jitter moves every vertex strictly inside the cube by an independent
    U[-j h, j h] offset per coordinate; boundary vertices stay put, so the domain
    boundary stays planar.
"""
from __future__ import annotations

import itertools

import numpy as np

# Seeds of the synthetic workloads (numpy PCG64 ``default_rng``).
SEED_JITTER = 1
SEED_WAVESPEED = 2
SEED_SOURCES = 3
SEED_FD_ELEMENTS = 4
SEED_CTRUE = 5
SEED_STATE = 6


def kuhn_cube_mesh(n: int, jitter: float = 0.0, seed: int = SEED_JITTER):
    """Return (VX [Nv,3] float64, EToV [K,4] int32) for an n^3 x 6 Kuhn mesh.

    Elements are ordered hex by hex (x fastest, then y, then z), six per hex, so that
    face neighbours are close in memory.
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    h = 1.0 / n
    g = np.arange(n + 1)
    # vertex id = i + (n+1) * (j + (n+1) * k)
    kk, jj, ii = np.meshgrid(g, g, g, indexing="ij")
    VX = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1).astype(np.float64) * h - 0.5

    def vid(i, j, k):
        return i + (n + 1) * (j + (n + 1) * k)

    # The six monotone lattice paths 000 -> 111 (one per permutation of the axes).
    paths = []
    for perm in itertools.permutations(range(3)):
        corner = [0, 0, 0]
        path = [tuple(corner)]
        for ax in perm:
            corner[ax] += 1
            path.append(tuple(corner))
        paths.append(path)

    tets = []
    for k in range(n):
        for j in range(n):
            for i in range(n):
                for path in paths:
                    tets.append([vid(i + a, j + b, k + c) for (a, b, c) in path])
    EToV = np.asarray(tets, dtype=np.int64)

    # positive orientation: swap two vertices where the signed volume is negative
    v = VX[EToV]
    d = np.einsum("ki,ki->k", np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]), v[:, 3] - v[:, 0])
    neg = d < 0
    EToV[neg, 2], EToV[neg, 3] = EToV[neg, 3].copy(), EToV[neg, 2].copy()

    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        interior = np.all(np.abs(VX) < 0.5 - 1e-12, axis=1)
        off = rng.uniform(-jitter * h, jitter * h, size=VX.shape)
        VX = VX + off * interior[:, None]
    return VX, EToV.astype(np.int32)


def element_centroids(VX, EToV):
    return VX[EToV].mean(axis=1)


def uniform_wavespeed(K: int, lo: float = 1.0, hi: float = 3.0, seed: int = SEED_WAVESPEED):
    """Per-element wavespeed c ~ U[lo, hi] (seeded)."""
    return np.random.default_rng(seed).uniform(lo, hi, size=K)


def layered_wavespeed(VX, EToV, bands=((-1.0 / 6.0, 2.5), (1.0 / 6.0, 1.5)), top=1.0):
    """Wavespeed by element-centroid z bands: z < -1/6 -> 2.5, -1/6 <= z < 1/6 -> 1.5,
    z >= 1/6 -> 1.0."""
    z = element_centroids(VX, EToV)[:, 2]
    c = np.full(z.shape, top)
    for zmax, val in reversed(bands):
        c[z < zmax] = val
    return c


def materials_from_wavespeed(c):
    """rho = 1 and kappa = c^2 per element."""
    c = np.asarray(c, dtype=np.float64)
    return np.ones_like(c), c * c


def random_points(count: int, lo, hi, seed: int = SEED_SOURCES):
    lo = np.broadcast_to(np.asarray(lo, dtype=np.float64), (3,))
    hi = np.broadcast_to(np.asarray(hi, dtype=np.float64), (3,))
    return np.random.default_rng(seed).uniform(lo, hi, size=(count, 3))


def receiver_plane(h: float, count_per_side: int = 16, extent: float = 0.45):
    """A count x count grid over x, y in [-extent, extent] on the plane z = 1/2 - h."""
    s = np.linspace(-extent, extent, count_per_side)
    X, Y = np.meshgrid(s, s, indexing="ij")
    Z = np.full_like(X, 0.5 - h)
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def num_nodes(N: int) -> int:
    """N_p = (N+1)(N+2)(N+3)/6, the dimension of P^N on a tetrahedron."""
    return (N + 1) * (N + 2) * (N + 3) // 6


def random_state(K: int, N: int, S: int = 1, seed: int = SEED_STATE, dtype=np.float64):
    """Seeded standard-normal coefficients, field-major [S][K][4][N_p] (the CPU oracle's
    layout; abi_layout() gives the library's)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((S, K, 4, num_nodes(N))).astype(dtype)


def abi_layout(q):
    """[..., 4, N_p] (field-major) -> [..., N_p, 4]: the library's state layout, in which the
    four fields of a coefficient are adjacent."""
    return np.ascontiguousarray(np.swapaxes(np.asarray(q), -1, -2))


def oracle_layout(q):
    """[..., N_p, 4] (library) -> [..., 4, N_p] (field-major)."""
    return np.ascontiguousarray(np.swapaxes(np.asarray(q), -1, -2))
