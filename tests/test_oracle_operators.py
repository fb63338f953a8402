"""Pins of the oracle's reference-element operators against what the paper and the
mathematics fix: printed values (tests/golden), exact identities, calculus and quadrature."""
from fractions import Fraction
from math import comb

import numpy as np
import pytest

from conftest import read_golden
from oracle import dg, nodal
from oracle import operators as ops


def cond(A):
    s = np.linalg.svd(A, compute_uv=False)
    s = s[s > s[0] * 1e-10]
    return s[0] / s[-1]


def close_printed(computed, printed):
    """Agreement to the digits the paper prints (about 6 significant, or 0.5e-5 abs)."""
    return abs(computed - printed) <= max(6e-6 * abs(printed), 5e-6)


GOLD = read_golden("paper_operator_values.txt")


@pytest.mark.parametrize("N", range(1, 10))
def test_printed_bernstein_values(N):
    """Fig. liftRoundoff and Fig. liftMinMax (Section 4.1)."""
    L = ops.lift_faces(N)[0]
    L0 = ops.to_float(ops.L0_exact(N))
    EL = ops.to_float(ops.EL_face_exact(N, 0))
    D0 = ops.barycentric_derivative(N, 0).astype(float)
    got = {
        "cond_L0": cond(L0), "cond_EL": cond(EL), "cond_bb_lift": cond(L), "cond_bb_D0": cond(D0),
        "min_bb_lift": L.min(), "max_bb_lift": L.max(), "min_EL": EL.min(), "max_EL": EL.max(),
        "min_L0": L0.min(), "max_L0": L0.max(),
    }
    for k, v in got.items():
        assert close_printed(v, GOLD[k][N - 1]), (k, N, v, GOLD[k][N - 1])


GOLD_NODAL = read_golden("paper_nodal_values.txt")


@pytest.mark.parametrize("N", range(1, 10))
def test_printed_nodal_values(N):
    """Warp & Blend nodal operators against the nodal series of Fig. liftRoundoff and
    Fig. liftMinMax (Section 4.1)."""
    Dr = nodal.nodal_derivatives(N)[0]
    L = nodal.nodal_lift(N)[0]
    got = {"cond_nodal_lift": cond(L), "cond_nodal_Dr": cond(Dr),
           "min_nodal_lift": L.min(), "max_nodal_lift": L.max()}
    for k, v in got.items():
        assert close_printed(v, GOLD_NODAL[k][N - 1]), (k, N, v, GOLD_NODAL[k][N - 1])


@pytest.mark.parametrize("N", range(1, 11))
def test_lift_is_inverse_mass_times_face_mass(N):
    """M (E_L^f L0) = M^f exactly (integer arithmetic), for every face: the factorized lift
    of Section 3.1.2 is M^{-1} M^f (M is SPD, so the solution is unique)."""
    sT, Mint = ops.mass_tet_integer(N)
    sF, M2int = ops.mass_tri_integer(N)
    for m in range(4):
        L = ops.lift_face_exact(N, m)
        den = 1
        for row in L:
            for v in row:
                den = den * v.denominator // np.gcd(den, v.denominator)
        Lint = np.array([[int(v * den) for v in row] for row in L], dtype=object)
        lhs = Mint.dot(Lint)                                   # (Np x Nfp) integers
        fn = ops.face_nodes(N, m)
        rhs = np.zeros_like(lhs)
        rhs[fn, :] = M2int * den                               # M^f restricted to the face columns
        # M = sT Mint, M^f = sF M2int:  sT Mint L = sF M2int  <=>  Mint Lint * sT = sF * den M2int
        r = sF / sT
        assert np.all(lhs * r.denominator == rhs * r.numerator)


@pytest.mark.parametrize("N", [1, 2, 3])
def test_lift_matches_exact_solve(N):
    """Small N: the factorized lift equals a direct exact rational solve of M X = M^f."""
    sT, Mint = ops.mass_tet_integer(N)
    sF, M2int = ops.mass_tri_integer(N)
    Np = Mint.shape[0]
    fn = list(ops.face_nodes(N, 2))
    A = [[Fraction(int(Mint[r, c])) * sT for c in range(Np)] for r in range(Np)]
    B = [[Fraction(0)] * len(fn) for _ in range(Np)]
    for i, r in enumerate(fn):
        for j in range(len(fn)):
            B[r][j] = Fraction(int(M2int[i, j])) * sF
    # Gauss-Jordan
    for col in range(Np):
        piv = next(r for r in range(col, Np) if A[r][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        B[col], B[piv] = B[piv], B[col]
        inv = 1 / A[col][col]
        A[col] = [v * inv for v in A[col]]
        B[col] = [v * inv for v in B[col]]
        for r in range(Np):
            if r != col and A[r][col] != 0:
                f = A[r][col]
                A[r] = [x - f * y for x, y in zip(A[r], A[col])]
                B[r] = [x - f * y for x, y in zip(B[r], B[col])]
    assert B == ops.lift_face_exact(N, 2)


@pytest.mark.parametrize("N", range(1, 11))
def test_L0_spectrum_and_sparsity(N):
    """eig(L0) = (N+i+3)(N+1-i)/2, i = 0..N, multiplicity i+1 (appendix A.3, d = 3 for the
    face operator); at most 7 nonzeros per row of L0 and N^f_p + 3 per row of E_L."""
    L0 = ops.to_float(ops.L0_exact(N))
    ev = np.sort(np.linalg.eigvalsh(L0))
    want = np.sort(np.concatenate([[(N + i + 3) * (N + 1 - i) / 2] * (i + 1) for i in range(N + 1)]))
    np.testing.assert_allclose(ev, want, rtol=1e-12)
    assert (np.count_nonzero(L0, axis=1) <= 7).all()
    EL = np.concatenate([ops.to_float(ops.EL_face_exact(N, m)) for m in range(4)], axis=1)
    assert np.count_nonzero(EL, axis=1).max() <= ops.num_face_nodes(N) + 3


@pytest.mark.parametrize("N", range(1, 8))
def test_derivative_row_and_column_forms(N):
    """Lemma 1: the column form D^i[alpha, beta] = alpha_j + 1 at alpha = beta - e_i + e_j
    builds the same matrix as the row form."""
    pos = ops.tet_position(N)
    for i in range(4):
        D = np.zeros((ops.num_nodes(N),) * 2, dtype=np.int64)
        for col, b in enumerate(ops.tet_multi_indices(N)):
            if b[i] == 0:
                continue
            for j in range(4):
                a = list(b)
                a[i] -= 1
                a[j] += 1
                D[pos[tuple(a)], col] += a[j] if j != i else b[i]
        np.testing.assert_array_equal(D, ops.barycentric_derivative(N, i))


@pytest.mark.parametrize("N", [1, 3, 6, 10])
def test_derivatives_match_calculus(N):
    """sum_alpha (D^r c)_alpha B_alpha = d/dr sum_alpha c_alpha B_alpha at random points,
    with the right side from the product rule on lambda^alpha (d lambda/dr = (-1/2, 1/2,
    0, 0), etc.)."""
    rng = np.random.default_rng(0)
    c = rng.standard_normal(ops.num_nodes(N))
    lam = rng.dirichlet(np.ones(4), size=40)
    B = ops.bernstein_eval(N, lam)
    dlam = {0: np.array([-0.5, 0.5, 0, 0]), 1: np.array([-0.5, 0, 0.5, 0]), 2: np.array([-0.5, 0, 0, 0.5])}
    from math import factorial
    for a_dir, Dm in zip(range(3), ops.reference_derivatives(N)):
        want = np.zeros(len(lam))
        for coef, a in zip(c, ops.tet_multi_indices(N)):
            C = factorial(N) // np.prod([factorial(x) for x in a])
            for i in range(4):
                if a[i] == 0 or dlam[a_dir][i] == 0:
                    continue
                term = dlam[a_dir][i] * a[i] * lam[:, i] ** (a[i] - 1)
                for j in range(4):
                    if j != i:
                        term = term * lam[:, j] ** a[j]
                want += coef * C * term
        np.testing.assert_allclose(B @ (Dm @ c), want, rtol=1e-11, atol=1e-11 * np.abs(want).max())


@pytest.mark.parametrize("N", [1, 2, 5])
def test_mass_matrices_match_quadrature(N):
    """The closed-form BB mass matrices equal numerical quadrature of B_alpha B_beta."""
    lam, w = dg.tet_quadrature(N + 2)
    B = ops.bernstein_eval(N, lam)
    M_quad = (4.0 / 3.0) * 6.0 * (B.T * w) @ B          # reference volume 4/3
    np.testing.assert_allclose(ops.mass_tet(N), M_quad, rtol=1e-12, atol=1e-15)
    # face: Gauss-Jacobi on the unit triangle, reference area 2
    from scipy.special import roots_jacobi
    tu, wu = roots_jacobi(N + 2, 1.0, 0.0)
    tv, wv = roots_jacobi(N + 2, 0.0, 0.0)
    U, V = np.meshgrid((1 + tu) / 2, (1 + tv) / 2, indexing="ij")
    W = np.outer(wu / 4, wv / 2)
    x, y = U.ravel(), ((1 - U) * V).ravel()
    l2 = np.stack([1 - x - y, x, y], axis=1)
    from math import factorial
    Bt = np.stack([factorial(N) // (factorial(a) * factorial(b) * factorial(c))
                   * l2[:, 0] ** a * l2[:, 1] ** b * l2[:, 2] ** c for (a, b, c) in ops.tri_multi_indices(N)], axis=1)
    M2_quad = 2.0 * 2.0 * (Bt.T * W.ravel()) @ Bt      # area 2, unit triangle area 1/2
    np.testing.assert_allclose(ops.mass_tri(N), M2_quad, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("N", [2, 5])
def test_face_lifts_are_row_permutations(N):
    """Section 3: the four face lifts are identical up to a row permutation."""
    L = ops.lift_faces(N)
    ref = sorted(map(tuple, L[0]))
    for m in range(1, 4):
        assert sorted(map(tuple, L[m])) == ref


def test_ell_closed_form():
    assert ops.ell(5, 0) == 1
    assert ops.ell(5, 2) == Fraction(comb(5, 2), 3)
    assert ops.ell(4, 3) == Fraction(-4, 4)
