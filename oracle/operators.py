"""Exact reference-element operators of the Bernstein-Bezier (BB) basis.

TEST INFRASTRUCTURE ONLY (part of the CPU oracle; see ``oracle/__init__``).

Everything here is built in exact rational arithmetic (``fractions.Fraction`` / Python
integers) and rounded to float64 once, at the end.

Conventions (Section 3 and 3.1 of the paper):
  * reference tetrahedron with vertices v0=(-1,-1,-1), v1=(1,-1,-1), v2=(-1,1,-1),
    v3=(-1,-1,1); barycentric coordinates
        lambda0 = -(1+r+s+t)/2, lambda1 = (1+r)/2, lambda2 = (1+s)/2, lambda3 = (1+t)/2
    (Section 3.1).  The paper prints the domain as "r+s+t <= 1"; lambda0 >= 0 needs
    r+s+t <= -1, which is the reading used here.
  * multi-index alpha = (a0, a1, a2, a3), |alpha| = N; node order
        for a0 in 0..N: for a1 in 0..N-a0: for a2 in 0..N-a0-a1: a3 = N-a0-a1-a2
  * face m is {lambda_m = 0}, the face opposite vertex m.  Its nodes are the alpha with
    alpha_m = 0, ordered by the remaining three indices (in increasing vertex order) with
    the same lexicographic rule in 2D: for a in 0..n: for b in 0..n-a: c = n-a-b.
  * reference volume |T| = 4/3; every reference face is given area 2, so that
    J^k = vol(D^k) / (4/3) and J^f = area(f) / 2 (reading of Section 3: with this choice
    L^f = M^{-1} M^f is the same matrix for every face up to a row permutation, as
    Section 3 states).
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache
from math import comb, factorial

import numpy as np

TET_VOLUME = Fraction(4, 3)
FACE_AREA = Fraction(2)


# ----------------------------------------------------------------------------------------
# multi-indices
# ----------------------------------------------------------------------------------------
@lru_cache(maxsize=None)
def tet_multi_indices(N: int):
    """All alpha with |alpha| = N in node order (Section 3.1; the first N^f_p nodes are
    those of face 0, then the next layer parallel to it, ...)."""
    return tuple((a0, a1, a2, N - a0 - a1 - a2)
                 for a0 in range(N + 1)
                 for a1 in range(N + 1 - a0)
                 for a2 in range(N + 1 - a0 - a1))


@lru_cache(maxsize=None)
def tri_multi_indices(n: int):
    """All 2D multi-indices (a, b, c), a+b+c = n, in face-node order."""
    return tuple((a, b, n - a - b) for a in range(n + 1) for b in range(n + 1 - a))


@lru_cache(maxsize=None)
def tet_position(N: int):
    return {a: i for i, a in enumerate(tet_multi_indices(N))}


@lru_cache(maxsize=None)
def tri_position(n: int):
    return {a: i for i, a in enumerate(tri_multi_indices(n))}


def num_nodes(N: int) -> int:
    return (N + 1) * (N + 2) * (N + 3) // 6


def num_face_nodes(N: int) -> int:
    return (N + 1) * (N + 2) // 2


def face_vertices(m: int):
    """Local vertices of face m (opposite vertex m), in increasing order."""
    return tuple(c for c in range(4) if c != m)


@lru_cache(maxsize=None)
def face_nodes(N: int, m: int) -> np.ndarray:
    """Volume node index of each node of face m, in face-node order."""
    pos = tet_position(N)
    fv = face_vertices(m)
    out = []
    for g in tri_multi_indices(N):
        a = [0, 0, 0, 0]
        for c, v in zip(fv, g):
            a[c] = v
        out.append(pos[tuple(a)])
    return np.asarray(out, dtype=np.int64)


# ----------------------------------------------------------------------------------------
# basis evaluation (for sources, receivers and tests)
# ----------------------------------------------------------------------------------------
def rst_to_barycentric(r, s, t):
    """lambda0..lambda3 of reference coordinates (Section 3.1)."""
    r, s, t = (np.asarray(x, dtype=np.float64) for x in (r, s, t))
    return np.stack([-(1 + r + s + t) / 2, (1 + r) / 2, (1 + s) / 2, (1 + t) / 2], axis=-1)


def bernstein_eval(N: int, lam: np.ndarray) -> np.ndarray:
    """B^N_alpha(lambda) = N!/(a0! a1! a2! a3!) prod_i lambda_i^{a_i}, for points
    lam[..., 4]; returns [..., N_p] (Section 3.1)."""
    lam = np.asarray(lam, dtype=np.float64)
    out = []
    for a in tet_multi_indices(N):
        c = factorial(N) // (factorial(a[0]) * factorial(a[1]) * factorial(a[2]) * factorial(a[3]))
        out.append(c * lam[..., 0] ** a[0] * lam[..., 1] ** a[1] * lam[..., 2] ** a[2] * lam[..., 3] ** a[3])
    return np.stack(out, axis=-1)


# ----------------------------------------------------------------------------------------
# derivative operators (Lemma 1; row form of the appendix lemma)
# ----------------------------------------------------------------------------------------
@lru_cache(maxsize=None)
def barycentric_derivative(N: int, i: int) -> np.ndarray:
    """Integer matrix D^i (derivative with respect to lambda_i in the BB basis).

    Row alpha has the entries D^i[alpha, beta] = alpha_j at beta = alpha + e_i - e_j,
    j = 0..3 (appendix, derivative lemma, row form).  Terms with alpha_j = 0 vanish.
    """
    Np = num_nodes(N)
    pos = tet_position(N)
    D = np.zeros((Np, Np), dtype=np.int64)
    for row, a in enumerate(tet_multi_indices(N)):
        for j in range(4):
            if a[j] == 0:
                continue
            b = list(a)
            b[i] += 1
            b[j] -= 1
            D[row, pos[tuple(b)]] += a[j]
    return D


@lru_cache(maxsize=None)
def reference_derivatives(N: int):
    """D^r, D^s, D^t (float64) through the chain rule of Algorithm 2:
    d/dr = (D^1 - D^0)/2, d/ds = (D^2 - D^0)/2, d/dt = (D^3 - D^0)/2."""
    D0 = barycentric_derivative(N, 0)
    return tuple((barycentric_derivative(N, a) - D0).astype(np.float64) / 2.0 for a in (1, 2, 3))


# ----------------------------------------------------------------------------------------
# mass matrices
# ----------------------------------------------------------------------------------------
def _bernstein_product_integral(alpha, beta, n: int, dim: int, measure: Fraction) -> Fraction:
    """int_T B^n_alpha B^n_beta over a dim-simplex of measure |T|:
       |T| (n!)^2 dim! / (2n+dim)! * prod_i (alpha_i+beta_i)! / (alpha_i! beta_i!).
    (Product of two Bernstein polynomials is a scaled Bernstein polynomial of degree 2n,
    and int_T B^{2n}_gamma = |T| / C(2n+dim, dim).)"""
    num = 1
    for a, b in zip(alpha, beta):
        num *= comb(a + b, a)
    return measure * Fraction(factorial(n) ** 2 * factorial(dim), factorial(2 * n + dim)) * num


@lru_cache(maxsize=None)
def mass_tet_integer(N: int):
    """(scale, Mint) with M = scale * Mint, Mint integer (object array)."""
    mi = tet_multi_indices(N)
    Np = len(mi)
    Mint = np.empty((Np, Np), dtype=object)
    for r, a in enumerate(mi):
        for c, b in enumerate(mi):
            v = 1
            for x, y in zip(a, b):
                v *= comb(x + y, x)
            Mint[r, c] = v
    scale = TET_VOLUME * Fraction(factorial(N) ** 2 * factorial(3), factorial(2 * N + 3))
    return scale, Mint


@lru_cache(maxsize=None)
def mass_tri_integer(n: int):
    mi = tri_multi_indices(n)
    nf = len(mi)
    Mint = np.empty((nf, nf), dtype=object)
    for r, a in enumerate(mi):
        for c, b in enumerate(mi):
            v = 1
            for x, y in zip(a, b):
                v *= comb(x + y, x)
            Mint[r, c] = v
    scale = FACE_AREA * Fraction(factorial(n) ** 2 * factorial(2), factorial(2 * n + 2))
    return scale, Mint


def mass_tet(N: int) -> np.ndarray:
    """Reference BB mass matrix M_ij = int_T phi_j phi_i (Section 3), float64."""
    scale, Mint = mass_tet_integer(N)
    return np.asarray([[float(scale * int(v)) for v in row] for row in Mint])


def mass_tri(n: int) -> np.ndarray:
    """Reference BB face mass matrix on a triangle of area 2, float64."""
    scale, Mint = mass_tri_integer(n)
    return np.asarray([[float(scale * int(v)) for v in row] for row in Mint])


# ----------------------------------------------------------------------------------------
# degree elevation / reduction and the lift factors (Section 3.1.2, appendix A.3)
# ----------------------------------------------------------------------------------------
@lru_cache(maxsize=None)
def elevation_tri(n: int):
    """One-degree elevation E^n_{n-1} on a triangle as a Fraction matrix of shape
    (n+1)(n+2)/2 x n(n+1)/2, from B^{n-1}_g = sum_c (g_c+1)/n B^n_{g+e_c} (appendix A)."""
    rows = tri_position(n)
    cols = tri_multi_indices(n - 1)
    E = [[Fraction(0)] * len(cols) for _ in range(len(rows))]
    for ci, g in enumerate(cols):
        for c in range(3):
            b = list(g)
            b[c] += 1
            E[rows[tuple(b)]][ci] += Fraction(g[c] + 1, n)
    return E


def _transpose(A):
    return [list(col) for col in zip(*A)]


def _matmul(A, B):
    Bt = _transpose(B)
    return [[sum((x * y for x, y in zip(row, col) if x and y), Fraction(0)) for col in Bt] for row in A]


@lru_cache(maxsize=None)
def L0_exact(N: int):
    """L0 = (N+1)^2/2 (E^{N+1}_N)^T E^{N+1}_N (Section 3.1.2), Fraction N^f_p x N^f_p."""
    E = elevation_tri(N + 1)
    s = Fraction((N + 1) ** 2, 2)
    return [[s * v for v in row] for row in _matmul(_transpose(E), E)]


def ell(N: int, j: int) -> Fraction:
    """l_j = (-1)^j C(N, j) / (1 + j) (Section 3.1.2)."""
    return Fraction((-1) ** j * comb(N, j), 1 + j)


def reduce_once(v, n: int):
    """Apply the one-degree reduction (E^n_{n-1})^T to a degree-n face vector v (list in
    face-node order): out[g] = sum_c (g_c+1)/n v[g+e_c], |g| = n-1 (appendix A)."""
    pos = tri_position(n)
    out = []
    for g in tri_multi_indices(n - 1):
        acc = 0
        for c in range(3):
            b = list(g)
            b[c] += 1
            acc = acc + Fraction(g[c] + 1, n) * v[pos[tuple(b)]]
        out.append(acc)
    return out


@lru_cache(maxsize=None)
def lift_layers_exact(N: int):
    """[l_j (E^N_{N-j})^T L0 for j = 0..N] as Fraction matrices ((N-j)^f_p x N^f_p).
    (E^N_{N-j})^T is the product of one-degree reductions (Section 3.1.2), applied here
    column by column, one degree at a time (Algorithm 1)."""
    L0 = L0_exact(N)
    cols = _transpose(L0)
    layers = []
    cur = cols
    for j in range(N + 1):
        if j > 0:
            cur = [reduce_once(col, N - j + 1) for col in cur]
        layers.append([[ell(N, j) * v for v in row] for row in _transpose(cur)])
    return layers


@lru_cache(maxsize=None)
def lift_face_exact(N: int, m: int):
    """The face lift L^f = M^{-1} M^f of face m restricted to its face columns
    (N_p x N^f_p, Fraction), from the factorization L^f = E_L^f L0 (Section 3.1.2 and
    appendix A.3): the row of node alpha with alpha_m = j is row gamma of
    l_j (E^N_{N-j})^T L0, gamma = the other three indices of alpha.

    ``tests/test_oracle_operators.py`` proves that this is M^{-1} M^f for every N used by
    checking M (E_L^f L0) = M^f exactly in integer arithmetic (M is SPD, so the solution
    of M X = M^f is unique)."""
    layers = lift_layers_exact(N)
    fv = face_vertices(m)
    rows = []
    for a in tet_multi_indices(N):
        j = a[m]
        g = tuple(a[c] for c in fv)
        rows.append(layers[j][tri_position(N - j)[g]])
    return rows


@lru_cache(maxsize=None)
def EL_face_exact(N: int, m: int):
    """E_L^f of face m (N_p x N^f_p, Fraction), rows in volume node order:
    the row of node alpha with alpha_m = j is row gamma of l_j (E^N_{N-j})^T."""
    Nfp = num_face_nodes(N)
    ident = [[Fraction(int(r == c)) for c in range(Nfp)] for r in range(Nfp)]
    cur = ident
    layers = []
    for j in range(N + 1):
        if j > 0:
            cur = [reduce_once(col, N - j + 1) for col in cur]  # columns of (E^N_{N-j})^T
        layers.append([[ell(N, j) * v for v in row] for row in _transpose(cur)])
    fv = face_vertices(m)
    return [layers[a[m]][tri_position(N - a[m])[tuple(a[c] for c in fv)]] for a in tet_multi_indices(N)]


def to_float(A) -> np.ndarray:
    return np.asarray([[float(v) for v in row] for row in A], dtype=np.float64)


@lru_cache(maxsize=None)
def lift_faces(N: int) -> np.ndarray:
    """float64 [4, N_p, N^f_p]: L^f for the four faces (exact values rounded once)."""
    return np.stack([to_float(lift_face_exact(N, m)) for m in range(4)])


@lru_cache(maxsize=None)
def mass_inverse(N: int) -> np.ndarray:
    """M^{-1} (float64) from an exact rational Gauss-Jordan elimination on the integer
    matrix; used for point sources."""
    scale, Mint = mass_tet_integer(N)
    Np = Mint.shape[0]
    A = [[Fraction(int(Mint[r, c])) for c in range(Np)] + [Fraction(int(r == c)) for c in range(Np)]
         for r in range(Np)]
    for col in range(Np):
        piv = next(r for r in range(col, Np) if A[r][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        inv = 1 / A[col][col]
        A[col] = [v * inv for v in A[col]]
        for r in range(Np):
            if r != col and A[r][col] != 0:
                f = A[r][col]
                A[r] = [x - f * y for x, y in zip(A[r], A[col])]
    return np.asarray([[float(v / scale) for v in row[Np:]] for row in A])
