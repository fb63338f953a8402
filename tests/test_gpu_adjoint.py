"""Discrete adjoint on the GPU: dot-product test of A^T against A, the transpose against
the oracle's assembled operator, the kappa-gradient against the oracle's complex-step
derivative of the same fully discrete scheme, and central finite differences."""
import numpy as np
import pytest

from oracle import adjoint as oadj
from oracle import dg
from paper_1512_06025_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bb():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1512_06025_gb300 import bbdg
    return bbdg


def hetero(n, jitter=0.1, seed=2):
    VX, EToV = inputs.kuhn_cube_mesh(n, jitter=jitter)
    K = len(EToV)
    c = inputs.uniform_wavespeed(K, seed=seed)
    rho = np.random.default_rng(seed + 10).uniform(0.5, 2.0, K)
    return VX, EToV, rho, rho * c * c


@pytest.mark.parametrize("N", [1, 2, 3, 5, 7, 10])
def test_dot_product(bb, N):
    """<A v, w> = <v, A^T w> for random v, w (jittered mesh, heterogeneous rho, kappa)."""
    VX, EToV, rho, kappa = hetero(3 if N <= 5 else 2, seed=N)
    K = len(EToV)
    s = bb.Solver(VX, EToV, rho, kappa, N)
    v = torch.tensor(inputs.abi_layout(inputs.random_state(K, N, seed=1)), device="cuda")
    w = torch.tensor(inputs.abi_layout(inputs.random_state(K, N, seed=2)), device="cuda")
    Av, ATw = torch.empty_like(v), torch.empty_like(w)
    bb.bbdg_rhs(s.ctx, v, Av)
    bb.bbdg_adjoint_rhs(s.ctx, w, ATw)
    lhs, rhs = float((Av * w).sum()), float((v * ATw).sum())
    scale = float(Av.norm() * w.norm())
    assert abs(lhs - rhs) <= 1e-13 * scale, (lhs, rhs)
    s.close()


def test_transpose_matches_assembled_oracle(bb):
    """A^T w equals the transpose of the oracle's operator assembled column by column."""
    N = 2
    VX, EToV, rho, kappa = hetero(1)
    K = len(EToV)
    P = dg.make_problem(VX, EToV, N, rho, kappa)
    n = K * 4 * P.Np
    A = np.empty((n, n))
    e = np.zeros(n)
    for j in range(n):
        e[j] = 1.0
        A[:, j] = dg.rhs(P, e.reshape(K, 4, P.Np)).ravel()
        e[j] = 0.0
    w = inputs.random_state(K, N, seed=3)
    want = (A.T @ w.ravel()).reshape(w.shape)
    s = bb.Solver(VX, EToV, rho, kappa, N)
    out = torch.empty((1, K, P.Np, 4), dtype=torch.float64, device="cuda")
    bb.bbdg_adjoint_rhs(s.ctx, torch.tensor(inputs.abi_layout(w), device="cuda"), out)
    got = inputs.oracle_layout(out.cpu().numpy())
    assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)
    s.close()


def small_inversion(bb, N=2, n=2, nsteps=6, C=4):
    from paper_1512_06025_gb300.gradient import MisfitGradient
    VX, EToV = inputs.kuhn_cube_mesh(n, jitter=0.1)
    K = len(EToV)
    c = inputs.uniform_wavespeed(K)
    rho, kappa = inputs.materials_from_wavespeed(c)
    xs = np.array([[0.1, -0.1, 0.05], [-0.2, 0.2, 0.1]])
    rec = inputs.receiver_plane(1.0 / n, 3)
    dt = 0.25 * (1.0 / n) / (N + 1) ** 2 / 3.0
    P = dg.make_problem(VX, EToV, N, rho, kappa)
    src = dg.make_sources(P, xs)
    recs = dg.make_receivers(P, rec)
    ctrue = c * (1 + 0.05 * np.random.default_rng(inputs.SEED_CTRUE).uniform(-1, 1, K))
    data = oadj.traces(P, src, recs, dt, nsteps, ctrue ** 2)
    P.set_materials(rho, kappa)
    s = bb.Solver(VX, EToV, rho, kappa, N)
    bb.bbdg_set_sources(s.ctx, xs, np.zeros(len(xs), dtype=np.int64), 10.0, 0.05)
    bb.bbdg_set_receivers(s.ctx, rec)
    drv = MisfitGradient(s, dt, nsteps, torch.tensor(data, device="cuda"), checkpoint_every=C)
    return P, src, recs, data, dt, rho, kappa, s, drv


def test_gradient_matches_complex_step(bb):
    """dJ/dkappa from the GPU adjoint (checkpoint segments of 4 steps, 6 steps) equals the
    oracle's complex-step derivative of the same discrete scheme for every element."""
    P, src, recs, data, dt, rho, kappa, s, drv = small_inversion(bb)
    J, _ = drv.forward()
    assert abs(J - oadj.misfit(P, src, recs, dt, drv.nsteps, data)) <= 1e-12 * abs(J)
    g = drv.backward().cpu().numpy()
    want = oadj.gradient_complex_step(P, src, recs, dt, drv.nsteps, data, kappa)
    want = np.array([want[k] for k in range(P.K)])
    assert np.abs(g - want).max() <= 1e-10 * np.abs(want).max(), np.abs(g - want).max() / np.abs(want).max()
    s.close()


def test_whole_trajectory_plan_matches_checkpoints(bb):
    """Keeping every stage (no recomputation) gives the checkpointed gradient bit for bit
    up to summation order, and the oracle's complex-step derivative."""
    P, src, recs, data, dt, rho, kappa, s, drv = small_inversion(bb)
    from paper_1512_06025_gb300.gradient import MisfitGradient
    assert not drv.keep_all
    J1, _ = drv.forward()
    g1 = drv.backward().cpu().numpy()
    drv2 = MisfitGradient(s, dt, drv.nsteps, drv.data, checkpoint_every=None)
    assert drv2.keep_all and drv2.stages.shape[0] == 5 * drv.nsteps + 1
    J2, _ = drv2.forward()
    g2 = drv2.backward().cpu().numpy()
    assert abs(J1 - J2) <= 1e-14 * abs(J1)
    assert np.abs(g1 - g2).max() <= 1e-13 * np.abs(g1).max()
    want = oadj.gradient_complex_step(P, src, recs, dt, drv.nsteps, data, kappa)
    want = np.array([want[k] for k in range(P.K)])
    assert np.abs(g2 - want).max() <= 1e-10 * np.abs(want).max()
    # a budget too small for the trajectory falls back to checkpoints
    drv3 = MisfitGradient(s, dt, drv.nsteps, drv.data, checkpoint_every=None, memory_budget=1)
    assert not drv3.keep_all and drv3.C == 20
    s.close()


def test_autograd_function(bb):
    from paper_1512_06025_gb300.gradient import kappa_misfit
    P, src, recs, data, dt, rho, kappa, s, drv = small_inversion(bb)
    kt = torch.tensor(kappa, dtype=torch.float64, device="cuda", requires_grad=True)
    J = kappa_misfit(kt, drv, rho)
    J.backward()
    drv2 = drv
    drv2.set_kappa(rho, kappa)
    drv2.forward()
    g = drv2.backward()
    assert torch.allclose(kt.grad, g, rtol=1e-13, atol=0)
    s.close()


def test_gradient_central_differences(bb):
    """16 seeded elements with |g_k| >= 1e-3 max|g|: central differences of J (GPU forward,
    relative step 1e-4 kappa_k) agree with the adjoint to 1e-6 relative."""
    P, src, recs, data, dt, rho, kappa, s, drv = small_inversion(bb, N=5, n=3, nsteps=40, C=20)
    drv.set_kappa(rho, kappa)
    drv.forward()
    g = drv.backward().cpu().numpy()
    big = np.nonzero(np.abs(g) >= 1e-3 * np.abs(g).max())[0]
    rng = np.random.default_rng(inputs.SEED_FD_ELEMENTS)
    pick = rng.choice(big, size=min(16, len(big)), replace=False)
    floor = 1e-3 * np.abs(g).max()
    for k in pick:
        eps = 1e-4 * kappa[k]
        kp, km = kappa.copy(), kappa.copy()
        kp[k] += eps
        km[k] -= eps
        drv.set_kappa(rho, kp)
        Jp, _ = drv.forward()
        drv.set_kappa(rho, km)
        Jm, _ = drv.forward()
        fd = (Jp - Jm) / (2 * eps)
        assert abs(g[k] - fd) <= 1e-6 * max(abs(fd), floor), (k, g[k], fd)
    s.close()


def test_gradient_taylor_remainder(bb):
    """Taylor test along a seeded random direction d (all elements): the remainder
    r(eps) = J(kappa + eps d) - J(kappa) - eps g.d falls as eps^2 (ratios r(eps)/r(eps/2)
    near 4 over eps = 1e-2 .. 1.25e-3 relative): g is the derivative of the same discrete
    misfit, so no first-order term is left."""
    P, src, recs, data, dt, rho, kappa, s, drv = small_inversion(bb, N=4, n=3, nsteps=30, C=10)
    drv.set_kappa(rho, kappa)
    J0, _ = drv.forward()
    g = drv.backward().cpu().numpy()
    d = np.random.default_rng(inputs.SEED_FD_ELEMENTS + 1).uniform(-1.0, 1.0, len(kappa)) * kappa
    gd = float(g @ d)
    rem = []
    for eps in (1e-2, 5e-3, 2.5e-3, 1.25e-3):
        drv.set_kappa(rho, kappa + eps * d)
        J, _ = drv.forward()
        rem.append(abs(J - J0 - eps * gd))
    s.close()
    assert rem[-1] > 1e-9 * abs(J0), rem          # above round-off, so the ratios mean something
    for a, b in zip(rem, rem[1:]):
        assert 3.5 < a / b < 4.5, rem


def test_misfit_kernel(bb):
    """bbdg_misfit: r = p - d exactly, J = 1/2 sum r^2 to the correctly rounded sum (math.fsum
    of the exact squares' halves, within a few ulps), the same bits on a second call."""
    import math
    VX, EToV = inputs.kuhn_cube_mesh(1)
    s = bb.Solver(VX, EToV, np.ones(len(EToV)), np.ones(len(EToV)), 2)
    rng = np.random.default_rng(31)
    tr = rng.standard_normal((400, 256)) * np.exp(rng.uniform(-20, 5, (400, 256)))
    d = tr + rng.standard_normal((400, 256)) * 1e-3
    tt, dd = torch.tensor(tr, device="cuda"), torch.tensor(d, device="cuda")
    r = torch.empty_like(tt)
    J = torch.zeros(1, dtype=torch.float64, device="cuda")
    bb.bbdg_misfit(s.ctx, tt, dd, r, J)
    J1 = float(J.item())
    bb.bbdg_misfit(s.ctx, tt, dd, r, J)
    s.close()
    rr = tr - d
    assert np.array_equal(r.cpu().numpy(), rr)
    want = math.fsum((0.5 * rr * rr).ravel())
    assert abs(J1 - want) <= 4e-16 * want, (J1, want)
    assert float(J.item()) == J1


def c5_inversion(bb, nsteps=400, C=20):
    """The adjoint workload: N = 5, 16^3 x 6 = 24 576 tets, c ~ U[1, 3], 8 Ricker sources in
    U([-0.4, 0.4]^2 x [0, 0.4]), 256 receivers on the plane z = 1/2 - h, FP64; data from the
    same solver with c_true = c (1 + 0.05 xi), xi ~ U[-1, 1]; checkpoints every C steps."""
    from paper_1512_06025_gb300.gradient import MisfitGradient
    N, n = 5, 16
    VX, EToV = inputs.kuhn_cube_mesh(n)
    K = len(EToV)
    c = inputs.uniform_wavespeed(K)
    rho, kappa = inputs.materials_from_wavespeed(c)
    dt = 0.25 * (1.0 / n) / (N + 1) ** 2 / c.max()
    s = bb.Solver(VX, EToV, rho, kappa, N, precision=bb.BBDG_F64)
    bb.bbdg_set_sources(s.ctx, inputs.random_points(8, (-0.4, -0.4, 0.0), (0.4, 0.4, 0.4)),
                        np.zeros(8, dtype=np.int64), 10.0, 0.05)
    bb.bbdg_set_receivers(s.ctx, inputs.receiver_plane(1.0 / n, 16))
    ctrue = c * (1 + 0.05 * np.random.default_rng(inputs.SEED_CTRUE).uniform(-1, 1, K))
    q = torch.zeros((1, K, s.Np, 4), dtype=torch.float64, device="cuda")
    traces = torch.zeros((nsteps, 1, 256), dtype=torch.float64, device="cuda")
    bb.bbdg_set_materials(s.ctx, ctrue ** 2, rho)
    bb.bbdg_step(s.ctx, q, torch.zeros_like(q), torch.empty_like(q), 0.0, dt, nsteps, traces=traces)
    data = traces[:, 0, :].clone()
    del q
    bb.bbdg_set_materials(s.ctx, kappa, rho)
    drv = MisfitGradient(s, dt, nsteps, data, checkpoint_every=C)
    return s, drv, rho, kappa


def test_c5_gradient_central_differences(bb):
    """The adjoint workload as configured (400 FP64 steps, checkpoints every 20): on 16
    seeded elements with |g_k| >= 1e-3 max|g|, central differences of J with relative step
    1e-4 kappa_k agree with the discrete-adjoint gradient to 1e-6 relative (error over
    max(|g_FD|, 1e-3 max|g|))."""
    s, drv, rho, kappa = c5_inversion(bb)
    J0, _ = drv.forward()
    g = drv.backward().cpu().numpy()
    assert np.isfinite(g).all() and J0 > 0
    big = np.nonzero(np.abs(g) >= 1e-3 * np.abs(g).max())[0]
    pick = np.random.default_rng(inputs.SEED_FD_ELEMENTS).choice(big, size=16, replace=False)
    floor = 1e-3 * np.abs(g).max()
    worst = 0.0
    for k in pick:
        eps = 1e-4 * kappa[k]
        kp, km = kappa.copy(), kappa.copy()
        kp[k] += eps
        km[k] -= eps
        drv.set_kappa(rho, kp)
        Jp, _ = drv.forward()
        drv.set_kappa(rho, km)
        Jm, _ = drv.forward()
        fd = (Jp - Jm) / (2 * eps)
        err = abs(g[k] - fd) / max(abs(fd), floor)
        worst = max(worst, err)
        assert err <= 1e-6, (k, g[k], fd, err)
    s.close()
