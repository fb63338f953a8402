"""Mesh connectivity, trace matching and affine geometry for the oracle.

TEST INFRASTRUCTURE ONLY (part of the CPU oracle; see ``oracle/__init__``).

Section 3: each element D^k is an affine image of the reference tetrahedron; the
geometric factors G^k = d(r,s,t)/d(x,y,z), the volume Jacobian J^k and the face Jacobians
J^f are constant per element / face.  Neighbouring traces are matched through the
equispaced-lattice correspondence of the Bernstein coefficients (Section 3.1): a face node
of element k and a face node of its neighbour are the same node when their barycentric
multi-indices agree on the three shared (global) vertices.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import operators as ops


@dataclass
class Mesh:
    VX: np.ndarray          # [Nv, 3]
    EToV: np.ndarray        # [K, 4]
    J: np.ndarray           # [K]      J^k = vol / (4/3)
    G: np.ndarray           # [K, 3, 3] G[k, i, a] = d(r,s,t)_a / dx_i (rows x,y,z; Section 3)
    normal: np.ndarray      # [K, 4, 3] outward unit normal of face m
    Jf: np.ndarray          # [K, 4]   J^f = area / 2
    nbr: np.ndarray         # [K, 4]   neighbour element, -1 on the boundary
    nbr_face: np.ndarray    # [K, 4]   neighbour's local face, -1 on the boundary
    vol_centroid: np.ndarray  # [K, 3]


def build_mesh(VX, EToV) -> Mesh:
    VX = np.asarray(VX, dtype=np.float64)
    EToV = np.asarray(EToV, dtype=np.int64)
    K = EToV.shape[0]
    v = VX[EToV]                                            # [K, 4, 3]
    # x = sum_i lambda_i v_i  =>  dx/dr = (v1-v0)/2, dx/ds = (v2-v0)/2, dx/dt = (v3-v0)/2
    Jm = np.stack([(v[:, 1] - v[:, 0]) / 2, (v[:, 2] - v[:, 0]) / 2, (v[:, 3] - v[:, 0]) / 2], axis=2)
    J = np.linalg.det(Jm)
    if np.any(J <= 0):
        raise ValueError("element with non-positive Jacobian")
    G = np.transpose(np.linalg.inv(Jm), (0, 2, 1))          # G[k, i, a] = (Jm^{-1})[a, i]

    normal = np.zeros((K, 4, 3))
    Jf = np.zeros((K, 4))
    for m in range(4):
        a, b, c = ops.face_vertices(m)
        cr = np.cross(v[:, b] - v[:, a], v[:, c] - v[:, a])
        area = np.linalg.norm(cr, axis=1) / 2
        n = cr / (2 * area[:, None])
        # outward: pointing away from the opposite vertex m
        flip = np.einsum("ki,ki->k", n, v[:, m] - v[:, a]) > 0
        n[flip] *= -1
        normal[:, m] = n
        Jf[:, m] = area / 2

    # face matching by sorted global vertex triples
    nbr = -np.ones((K, 4), dtype=np.int64)
    nbr_face = -np.ones((K, 4), dtype=np.int64)
    table = {}
    for k in range(K):
        for m in range(4):
            key = tuple(sorted(int(EToV[k, c]) for c in ops.face_vertices(m)))
            table.setdefault(key, []).append((k, m))
    for key, lst in table.items():
        if len(lst) == 2:
            (k1, m1), (k2, m2) = lst
            nbr[k1, m1], nbr_face[k1, m1] = k2, m2
            nbr[k2, m2], nbr_face[k2, m2] = k1, m1
        elif len(lst) > 2:
            raise ValueError("non-manifold face")
    return Mesh(VX=VX, EToV=EToV, J=J, G=G, normal=normal, Jf=Jf, nbr=nbr, nbr_face=nbr_face,
                vol_centroid=v.mean(axis=1))


def neighbour_node_map(mesh: Mesh, N: int) -> np.ndarray:
    """[K, 4, N^f_p] volume index, in the neighbour element, of each face node of (k, m)
    (-1 on boundary faces).  Node alpha of face m of k (alpha_m = 0) matches node beta of
    face m' of k' when beta gives each shared global vertex the exponent alpha gives it."""
    K = mesh.EToV.shape[0]
    Nfp = ops.num_face_nodes(N)
    pos = ops.tet_position(N)
    out = -np.ones((K, 4, Nfp), dtype=np.int64)
    cache = {}
    for m in range(4):
        fv = ops.face_vertices(m)
        ks = np.nonzero(mesh.nbr[:, m] >= 0)[0]
        if ks.size == 0:
            continue
        k2 = mesh.nbr[ks, m]
        # local index, in k2, of each of our face vertices
        d = np.empty((ks.size, 3), dtype=np.int64)
        for r, c in enumerate(fv):
            g = mesh.EToV[ks, c]
            d[:, r] = np.argmax(mesh.EToV[k2] == g[:, None], axis=1)
        keys = d[:, 0] * 16 + d[:, 1] * 4 + d[:, 2]
        for key in np.unique(keys):
            sel = keys == key
            dd = (key // 16, (key // 4) % 4, key % 4)
            if (m, dd) not in cache:
                idx = []
                for g in ops.tri_multi_indices(N):
                    b = [0, 0, 0, 0]
                    for r in range(3):
                        b[dd[r]] = g[r]
                    idx.append(pos[tuple(b)])
                cache[(m, dd)] = np.asarray(idx)
            out[ks[sel], m, :] = cache[(m, dd)]
    return out


def barycentric_of_points(mesh: Mesh, pts: np.ndarray, k: np.ndarray) -> np.ndarray:
    """Barycentric coordinates (lambda0..3) of points pts[i] in element k[i]."""
    v = mesh.VX[mesh.EToV[k]]                                # [n, 4, 3]
    A = np.stack([v[:, 1] - v[:, 0], v[:, 2] - v[:, 0], v[:, 3] - v[:, 0]], axis=2)
    lam123 = np.linalg.solve(A, (pts - v[:, 0])[..., None])[..., 0]
    return np.concatenate([1 - lam123.sum(axis=1, keepdims=True), lam123], axis=1)


def locate_points(mesh: Mesh, pts: np.ndarray, tol: float = 1e-12) -> np.ndarray:
    """Lowest-index element containing each point (all lambda >= -tol)."""
    pts = np.atleast_2d(np.asarray(pts, dtype=np.float64))
    K = mesh.EToV.shape[0]
    out = np.empty(len(pts), dtype=np.int64)
    for i, x in enumerate(pts):
        lam = barycentric_of_points(mesh, np.repeat(x[None], K, axis=0), np.arange(K))
        hit = np.nonzero(np.all(lam >= -tol, axis=1))[0]
        if hit.size == 0:
            raise ValueError("point outside the mesh")
        out[i] = hit[0]
    return out
