"""Pins of the oracle's right-hand side, time integrator, sources and receivers against
invariants and closed forms (Sections 2, 3, 4.1, 4.2)."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import dg
from oracle import operators as ops
from paper_1512_06025_gb300 import inputs


def problem(n, N, jitter=0.1, hetero=True):
    VX, EToV = inputs.kuhn_cube_mesh(n, jitter=jitter)
    K = len(EToV)
    if hetero:
        c = inputs.uniform_wavespeed(K)
        rho = np.random.default_rng(11).uniform(0.5, 2.0, K)
        kappa = rho * c * c
    else:
        rho, kappa = np.ones(K), np.ones(K)
    return dg.make_problem(VX, EToV, N, rho, kappa)


@pytest.mark.parametrize("n,N", [(1, 1), (2, 2), (2, 3), (2, 5), (1, 8)])
def test_energy_identity_upwind(n, N):
    """q^T W A q equals the face-jump dissipation of the Section 2 energy statement, for a
    random q (interior cross terms cancel; mirror faces give -tau_p (p^-)^2)."""
    P = problem(n, N)
    q = inputs.random_state(P.K, N)[0]
    a, b = dg.energy_rate(P, q), dg.energy_dissipation(P, q)
    assert b < 0
    assert abs(a - b) <= 1e-12 * abs(b)


@pytest.mark.parametrize("n,N", [(1, 1), (2, 3), (2, 5)])
def test_energy_identity_absorbing_boundary(n, N):
    """Zero exterior state on the boundary: q^T W A q equals the interior jump terms plus
    -1/2 int (tau_p p^2 + tau_u u_n^2) per boundary face, exactly; and it differs from the
    mirror case (the pin sees the boundary condition)."""
    P = problem(n, N)
    q = inputs.random_state(P.K, N)[0]
    mirror = dg.energy_rate(P, q)
    P.bc = "absorbing"
    a, b = dg.energy_rate(P, q), dg.energy_dissipation(P, q)
    assert b < 0
    assert abs(a - b) <= 1e-12 * abs(b)
    assert abs(a - mirror) > 1e-3 * abs(b)
    # interior faces untouched: the right-hand side changes only on boundary elements
    bnd = (P.mesh.nbr < 0).any(axis=1)
    r_abs = dg.rhs(P, q)
    P.bc = "mirror"
    r_mir = dg.rhs(P, q)
    assert np.array_equal(r_abs[~bnd], r_mir[~bnd]) and not np.allclose(r_abs[bnd], r_mir[bnd])


@pytest.mark.parametrize("n,N", [(2, 2), (2, 4)])
def test_energy_conserved_central(n, N):
    """With central fluxes (tau = 0) the semi-discrete energy is conserved: q^T W A q = 0."""
    P = problem(n, N)
    q = inputs.random_state(P.K, N)[0]
    r = dg.energy_rate(P, q, central=True)
    scale = dg.energy(P, q) * np.abs(dg.rhs(P, q)).max()
    assert abs(r) <= 1e-13 * scale


@pytest.mark.parametrize("N", [1, 2, 4])
def test_divergence_of_global_polynomial(N):
    """p = 0 and u a global polynomial of degree <= N: all jumps vanish, so
    rhs_p = -kappa div u exactly and rhs_u = 0."""
    P = problem(2, N)
    rng = np.random.default_rng(3)
    cu = rng.standard_normal((3, 4))

    def poly(x, y, z, c):      # degree <= min(N, 2) polynomial with coefficients c
        base = [np.ones_like(x), x, y, z]
        if N >= 2:
            base = [np.ones_like(x), x * y, y * z + x, x * x - z]
        return sum(ci * b for ci, b in zip(c, base))

    def div(x, y, z):
        if N >= 2:
            # d/dx of u0 + d/dy of u1 + d/dz of u2 with base [1, xy, yz + x, x^2 - z]
            return (cu[0, 1] * y + cu[0, 2] + cu[0, 3] * 2 * x) + (cu[1, 1] * x + cu[1, 2] * z) \
                + (cu[2, 2] * y - cu[2, 3])
        return (cu[0, 1] + cu[1, 2] + cu[2, 3]) * np.ones_like(x)

    q = np.zeros((P.K, 4, P.Np))
    for i in range(3):
        q[:, 1 + i] = dg.interpolate(P, lambda x, y, z, i=i: poly(x, y, z, cu[i]))
    r = dg.rhs(P, q)
    want = -P.kappa[:, None] * dg.interpolate(P, div)
    np.testing.assert_allclose(r[:, 0], want, atol=1e-11 * np.abs(want).max())
    assert np.abs(r[:, 1:]).max() <= 1e-11 * np.abs(want).max()


def test_gradient_of_boundary_vanishing_polynomial():
    """u = 0 and p = (x^2-1/4)(y^2-1/4)(z^2-1/4) (degree 6, zero on the boundary so the
    mirror jump vanishes): rhs_u = -grad p / rho exactly and rhs_p = 0."""
    N = 6
    P = problem(1, N)
    f = lambda x, y, z: (x * x - 0.25) * (y * y - 0.25) * (z * z - 0.25)
    g = [lambda x, y, z: 2 * x * (y * y - 0.25) * (z * z - 0.25),
         lambda x, y, z: 2 * y * (x * x - 0.25) * (z * z - 0.25),
         lambda x, y, z: 2 * z * (x * x - 0.25) * (y * y - 0.25)]
    q = np.zeros((P.K, 4, P.Np))
    q[:, 0] = dg.interpolate(P, f)
    r = dg.rhs(P, q)
    for i in range(3):
        want = -dg.interpolate(P, g[i]) / P.rho[:, None]
        np.testing.assert_allclose(r[:, 1 + i], want, atol=1e-11)
    assert np.abs(r[:, 0]).max() <= 1e-11


def butcher_from_lserk():
    """Butcher tableau of the 2N-storage scheme res = a_s res + dt f_s; q += b_s res."""
    A, B = dg.LSERK_A, dg.LSERK_B
    s = 5
    # stage s sees q_s = q_0 + sum_{j<s} Acoef[s][j] dt f_j
    R = [[Fraction(0)] * s for _ in range(s)]   # res after stage i: R[i][j] coefficient of f_j
    Q = [[Fraction(0)] * s for _ in range(s + 1)]
    for i in range(s):
        prev = R[i - 1] if i > 0 else [Fraction(0)] * s
        R[i] = [A[i] * v for v in prev]
        R[i][i] += 1
        Q[i + 1] = [Q[i][j] + B[i] * R[i][j] for j in range(s)]
    return Q[:s], Q[s]


def test_lserk4_order_conditions():
    """Carpenter-Kennedy LSERK4 (Section 4.2): the equivalent Butcher tableau satisfies all
    eight order conditions of order 4, and c_s = sum_j a_sj."""
    Am, b = butcher_from_lserk()
    c = [sum(row) for row in Am]
    tol = 1e-14
    for cs, cd in zip(c, dg.LSERK_C):
        assert abs(float(cs - cd)) < tol
    Am = np.array([[float(v) for v in row] for row in Am])
    b = np.array([float(v) for v in b])
    c = Am.sum(axis=1)
    conds = [(b.sum(), 1), (b @ c, 1 / 2), (b @ c ** 2, 1 / 3), (b @ (Am @ c), 1 / 6),
             (b @ c ** 3, 1 / 4), (b @ (c * (Am @ c)), 1 / 8), (b @ (Am @ c ** 2), 1 / 12),
             (b @ (Am @ (Am @ c)), 1 / 24)]
    for got, want in conds:
        assert abs(got - want) < 1e-12
    # stability polynomial coefficient of z^5 (not fixed by the order conditions)
    assert abs(b @ (Am @ (Am @ (Am @ c))) - 1 / 200) < 1e-12


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_standing_mode_convergence(N):
    """Standing mode of Section 4.1: L2 error at T = 0.5 (past a quarter period of the mode,
    sqrt(3) pi T = 2.7) converges at about O(h^{N+1}) on h = 1/2, 1/4, 1/8 (measured rates
    between h = 1/4 and 1/8: 1.90, 3.08, 3.85, 4.96)."""
    T = 0.5
    errs = []
    for n in (2, 4, 8):
        P = problem(n, N, jitter=0.0, hetero=False)
        q0 = dg.interpolate_state(P, dg.standing_mode(0.0))
        h = 1.0 / n
        ns = int(np.ceil(T / (0.3 * h / (N + 1) ** 2)))
        q, _, _ = dg.run(P, q0, 0.0, T / ns, ns)
        errs.append(dg.l2_error(P, q, dg.standing_mode(T)))
    rate = np.log2(errs[-2] / errs[-1])
    assert rate > N + 1 - 0.35, (N, errs)


def test_fully_discrete_energy_decreases():
    """Upwind flux at a stable dt: the discrete energy does not grow over LSERK4 steps."""
    P = problem(2, 3)
    q = inputs.random_state(P.K, 3)[0]
    dt = 0.25 * 0.5 / 16 / np.sqrt(P.kappa.max() / P.rho.min())
    e = [dg.energy(P, q)]
    res = np.zeros_like(q)
    for _ in range(10):
        q, res = dg.lserk4_step(lambda x, t: dg.rhs(P, x), q, res, 0.0, dt)
        e.append(dg.energy(P, q))
    assert all(e[i + 1] <= e[i] * (1 + 1e-14) for i in range(len(e) - 1))


def test_point_source_weak_form():
    """The source vector v = M^{-1} b / J^e satisfies J^e phi^T M v = phi(x_s) for every
    polynomial phi in the element (the weak form of delta(x - x_s))."""
    P = problem(2, 3)
    xs = np.array([[0.1, -0.2, 0.05]])
    src = dg.make_sources(P, xs)
    e = src.elem[0]
    M = ops.mass_tet(3)
    rng = np.random.default_rng(2)
    phi = rng.standard_normal(P.Np)
    lam = dg.meshmod.barycentric_of_points(P.mesh, xs, src.elem)
    val = ops.bernstein_eval(3, lam)[0] @ phi
    assert abs(P.mesh.J[e] * phi @ M @ src.vec[0] - val) < 1e-12 * max(1, abs(val))
    assert np.all(lam >= -1e-12)


def test_receiver_sampling_reproduces_polynomial():
    P = problem(2, 2)
    f = lambda x, y, z: 1 + x - 2 * y * z + z * z
    q = np.zeros((P.K, 4, P.Np))
    q[:, 0] = dg.interpolate(P, f)
    pts = inputs.random_points(10, -0.45, 0.45)
    rec = dg.make_receivers(P, pts)
    np.testing.assert_allclose(dg.sample(rec, q), f(*pts.T), rtol=1e-12, atol=1e-12)


def test_ricker_peak():
    assert dg.ricker(0.05) == 1.0
    assert abs(dg.ricker(0.05 + 1 / (np.pi * 10 * np.sqrt(2)))) < 1e-15


def test_complex_step_gradient_matches_central_differences():
    """The oracle's complex-step dJ/dkappa agrees with central differences of its misfit."""
    from oracle import adjoint
    VX, EToV = inputs.kuhn_cube_mesh(2, jitter=0.1)
    K = len(EToV)
    rho, kap = inputs.materials_from_wavespeed(inputs.uniform_wavespeed(K))
    P = dg.make_problem(VX, EToV, 2, rho, kap)
    src = dg.make_sources(P, [[0.1, -0.1, 0.05]])
    rec = dg.make_receivers(P, inputs.receiver_plane(0.5, 3))
    dt, ns = 0.25 * 0.5 / 9 / 3, 5
    data = adjoint.traces(P, src, rec, dt, ns, kap * 1.05)
    g = adjoint.gradient_complex_step(P, src, rec, dt, ns, data, kap, elements=[3, 20])
    for k in (3, 20):
        e = 1e-3 * kap[k]          # central-difference truncation ~1e-7 relative here
        kp, km = kap.copy(), kap.copy()
        kp[k] += e
        km[k] -= e
        fd = (adjoint.misfit(P, src, rec, dt, ns, data, kp) - adjoint.misfit(P, src, rec, dt, ns, data, km)) / (2 * e)
        assert abs(g[k] - fd) <= 1e-5 * abs(fd)


def test_rhs_on_element_subset_equals_full_rows():
    """rhs(P, q, elements=ks) is the ks rows of the full right-hand side (the sampled-output
    oracle used by the full-size GPU parity tests), including boundary and interior faces."""
    VX, EToV = inputs.kuhn_cube_mesh(3, jitter=0.1)
    K = len(EToV)
    c = inputs.uniform_wavespeed(K)
    rho, kappa = inputs.materials_from_wavespeed(c)
    P = dg.make_problem(VX, EToV, 3, rho, kappa)
    q = inputs.random_state(K, 3)[0]
    full = dg.rhs(P, q)
    ks = np.random.default_rng(0).choice(K, size=17, replace=False)
    np.testing.assert_allclose(dg.rhs(P, q, elements=ks), full[ks], rtol=1e-13, atol=1e-13 * np.abs(full).max())
    np.testing.assert_allclose(dg.rhs(P, q, central=True, elements=ks[::-1]), dg.rhs(P, q, central=True)[ks[::-1]],
                               rtol=1e-13, atol=1e-13 * np.abs(full).max())
