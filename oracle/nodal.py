"""Warp & Blend nodes and the nodal (Lagrange) DG operators, for the dense nodal path.

TEST INFRASTRUCTURE ONLY (part of the CPU oracle; see ``oracle/__init__``).

Section 3.1: the nodal basis is the Lagrange basis on the Warp & Blend nodes of
[warburton2006explicit].  The construction, restated here from that paper:
  * start from the equispaced barycentric lattice lambda = alpha / N on a regular
    (equilateral) tetrahedron with vertices V_0..V_3;
  * 1D warp: g(r) = sum_i (x^LGL_i - x^eq_i) l^eq_i(r) / (1 - r^2), the interpolant
    through the equispaced points of the displacement that moves them onto the
    Legendre-Gauss-Lobatto points, divided by (1 - r^2);
  * a face with barycentrics (l_a, l_b, l_c) is warped by
        w_f = sum over its edges (a -> b) of 4 l_a l_b (1 + (alpha l_c)^2) g(l_b - l_a) e_ab,
    e_ab the unit vector from V_a to V_b;
  * the volume shift is sum_f beta_f w_f with the blend
        beta_f = (1 + (alpha l_f)^2) l_a l_b l_c / ((l_a + l_f/2)(l_b + l_f/2)(l_c + l_f/2)),
    l_f the barycentric coordinate opposite face f; on an edge of the tetrahedron the
    shift is the edge warp itself;
  * alpha is the optimised blend parameter of [warburton2006explicit] for the
    tetrahedron (its table for N = 1..15).

Nodal operators follow from the BB ones by the change of basis V_B[i, alpha] =
B_alpha(x_i) (both bases span P^N, Section 4.1): D^r_nodal = V_B D^r_BB V_B^{-1} and
L^f_nodal = V_B L^f_BB V_f^{-1}, V_f the restriction of V_B to the face nodes.

PARITY UNPINNED (loosely pinned): the node coordinates are pinned only through the
condition numbers and min/max entries that the paper prints for the nodal operators
(three to six digits; tests/golden/paper_nodal_values.txt).
"""
from __future__ import annotations

from functools import lru_cache

import numpy as np
from numpy.polynomial import legendre

from . import operators as ops

# Optimised blend parameter alpha for the tetrahedron, N = 1..15 ([warburton2006explicit]).
ALPHA_OPT = (0.0, 0.0, 0.0, 0.1002, 1.1332, 1.5608, 1.3413, 1.2577, 1.1603, 1.10153,
             0.6080, 0.4523, 0.8856, 0.8717, 0.9655)

_TOL = 1e-10


def lgl_points(N: int) -> np.ndarray:
    """Legendre-Gauss-Lobatto points on [-1, 1] (ascending): +-1 and the roots of P_N'."""
    if N == 1:
        return np.array([-1.0, 1.0])
    inner = np.sort(legendre.Legendre.basis(N).deriv().roots().real)
    return np.concatenate([[-1.0], inner, [1.0]])


def warp_factor(N: int, r: np.ndarray) -> np.ndarray:
    """g(r): LGL displacement interpolated through equispaced points, / (1 - r^2);
    zero at r = +-1."""
    xe = np.linspace(-1.0, 1.0, N + 1)
    d = lgl_points(N) - xe
    w = np.zeros_like(r)
    for i in range(N + 1):
        li = np.ones_like(r)
        for j in range(N + 1):
            if j != i:
                li *= (r - xe[j]) / (xe[i] - xe[j])
        w += d[i] * li
    inside = np.abs(r) < 1.0 - _TOL
    out = np.zeros_like(r)
    out[inside] = w[inside] / (1.0 - r[inside] ** 2)
    return out


def _regular_tet():
    V = np.array([[-1.0, -1 / np.sqrt(3), -1 / np.sqrt(6)],
                  [1.0, -1 / np.sqrt(3), -1 / np.sqrt(6)],
                  [0.0, 2 / np.sqrt(3), -1 / np.sqrt(6)],
                  [0.0, 0.0, 3 / np.sqrt(6)]])
    return V


def _face_warp(N, alpha, lam, face_verts, V):
    """w_f for the face with vertices face_verts (three vertex ids)."""
    a, b, c = face_verts
    out = np.zeros((lam.shape[0], 3))
    for (x, y, z) in ((a, b, c), (b, c, a), (c, a, b)):
        e = V[y] - V[x]
        e /= np.linalg.norm(e)
        amp = 4 * lam[:, x] * lam[:, y] * (1 + (alpha * lam[:, z]) ** 2) * warp_factor(N, lam[:, y] - lam[:, x])
        out += amp[:, None] * e[None, :]
    return out


@lru_cache(maxsize=None)
def warp_blend_barycentric(N: int) -> np.ndarray:
    """Barycentric coordinates [N_p, 4] of the Warp & Blend nodes, in BB node order
    (node alpha is the warped lattice point alpha / N)."""
    alpha = ALPHA_OPT[N - 1] if N <= 15 else 1.0
    lam = np.asarray(ops.tet_multi_indices(N), dtype=np.float64) / N
    V = _regular_tet()
    X = lam @ V
    shift = np.zeros_like(X)
    on_edge = (lam > _TOL).sum(axis=1) <= 2
    for f in range(4):
        fv = ops.face_vertices(f)
        w = _face_warp(N, alpha, lam, fv, V)
        la, lb, lc = lam[:, fv[0]], lam[:, fv[1]], lam[:, fv[2]]
        lf = lam[:, f]
        den = (la + lf / 2) * (lb + lf / 2) * (lc + lf / 2)
        blend = np.where(den > _TOL, (1 + (alpha * lf) ** 2) * la * lb * lc / np.where(den > _TOL, den, 1.0), 0.0)
        shift += blend[:, None] * w
        # edges of this face: the shift is the (unblended) edge warp
        fix = on_edge & (lf < _TOL)
        shift[fix] = w[fix]
    X = X + shift
    # back to barycentric coordinates of the regular tetrahedron
    A = np.stack([V[1] - V[0], V[2] - V[0], V[3] - V[0]], axis=1)
    l123 = np.linalg.solve(A, (X - V[0]).T).T
    return np.concatenate([1 - l123.sum(axis=1, keepdims=True), l123], axis=1)


@lru_cache(maxsize=None)
def bb_vandermonde(N: int) -> np.ndarray:
    """V_B[i, alpha] = B_alpha at Warp & Blend node i."""
    return ops.bernstein_eval(N, warp_blend_barycentric(N))


@lru_cache(maxsize=None)
def nodal_derivatives(N: int):
    """Dense nodal D^r, D^s, D^t = V_B D_BB V_B^{-1}."""
    V = bb_vandermonde(N)
    return tuple(np.linalg.solve(V.T, (V @ D).T).T for D in ops.reference_derivatives(N))


@lru_cache(maxsize=None)
def nodal_lift(N: int) -> np.ndarray:
    """[4, N_p, N^f_p] nodal face lifts L^f_nodal = V_B L^f_BB V_f^{-1}."""
    V = bb_vandermonde(N)
    L = ops.lift_faces(N)
    out = []
    for m in range(4):
        fn = ops.face_nodes(N, m)
        Vf = V[np.ix_(fn, fn)]
        out.append(np.linalg.solve(Vf.T, (V @ L[m]).T).T)
    return np.stack(out)


def to_nodal(N: int, q: np.ndarray) -> np.ndarray:
    """Nodal values (at the Warp & Blend nodes) of BB coefficients q[..., N_p]."""
    return q @ bb_vandermonde(N).T


def from_nodal(N: int, u: np.ndarray) -> np.ndarray:
    return np.linalg.solve(bb_vandermonde(N), u.reshape(-1, u.shape[-1]).T).T.reshape(u.shape)
