"""GPU parity of the Bernstein-Bezier path (through the C ABI) against the CPU oracle.

Tolerances: FP64 1e-12 relative in the 2-norm over all outputs (the stated FP64 bound);
FP32 right-hand side 1e-5 relative (single evaluation, FP32 arithmetic with about
cond(E_L) * 1e-7 growth at high N)."""
import numpy as np
import pytest

from oracle import dg
from paper_1512_06025_gb300 import inputs
from conftest import elem_rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bb():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1512_06025_gb300 import bbdg
    return bbdg


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def make(n, N, jitter=0.1, seed=2):
    VX, EToV = inputs.kuhn_cube_mesh(n, jitter=jitter)
    K = len(EToV)
    c = inputs.uniform_wavespeed(K, seed=seed)
    rho = np.random.default_rng(seed + 10).uniform(0.5, 2.0, K)
    return VX, EToV, rho, rho * c * c


@pytest.mark.parametrize("N", range(1, 11))
def test_rhs_f64_matches_oracle(bb, N):
    n = 3 if N <= 6 else 2          # K = 162 / 48: several blocks and a ragged tail
    VX, EToV, rho, kappa = make(n, N)
    K = len(EToV)
    P = dg.make_problem(VX, EToV, N, rho, kappa)
    q0 = inputs.random_state(K, N, S=2)
    want = np.stack([dg.rhs(P, q0[s]) for s in range(2)])
    s = bb.Solver(VX, EToV, rho, kappa, N, precision=bb.BBDG_F64)
    q = torch.tensor(inputs.abi_layout(q0), device="cuda")
    r = torch.empty_like(q)
    bb.bbdg_rhs(s.ctx, q, r)
    got = inputs.oracle_layout(r.cpu().numpy())
    s.close()
    assert rel(got, want) < 1e-12, rel(got, want)
    # element by element: every entry to 1e-12 of the output's scale
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("N", range(1, 11))
def test_rhs_f32_matches_oracle(bb, N):
    VX, EToV, rho, kappa = make(2, N)
    K = len(EToV)
    P = dg.make_problem(VX, EToV, N, rho, kappa)
    q0 = inputs.random_state(K, N, S=1)
    want = dg.rhs(P, q0[0].astype(np.float32).astype(np.float64))
    s = bb.Solver(VX, EToV, rho, kappa, N, precision=bb.BBDG_F32)
    q = torch.tensor(inputs.abi_layout(q0), device="cuda", dtype=torch.float32)
    r = torch.empty_like(q)
    bb.bbdg_rhs(s.ctx, q, r)
    got = inputs.oracle_layout(r.cpu().numpy())[0].astype(np.float64)
    s.close()
    assert rel(got, want) < 1e-5, rel(got, want)
    assert elem_rel(got, want) < 1e-5, elem_rel(got, want)


def test_single_element_all_boundary(bb):
    """K = 1: every face is a mirror boundary face."""
    VX = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.float64)
    EToV = np.array([[0, 1, 2, 3]], dtype=np.int32)
    rho, kappa = np.array([1.3]), np.array([2.1])
    for N in (1, 4, 10):
        P = dg.make_problem(VX, EToV, N, rho, kappa)
        q0 = inputs.random_state(1, N)
        want = dg.rhs(P, q0[0])
        s = bb.Solver(VX, EToV, rho, kappa, N)
        q = torch.tensor(inputs.abi_layout(q0), device="cuda")
        r = torch.empty_like(q)
        bb.bbdg_rhs(s.ctx, q, r)
        assert rel(inputs.oracle_layout(r.cpu().numpy())[0], want) < 1e-12
        s.close()


def test_central_flux_matches_oracle(bb):
    N = 4
    VX, EToV, rho, kappa = make(2, N)
    P = dg.make_problem(VX, EToV, N, rho, kappa)
    q0 = inputs.random_state(len(EToV), N)
    want = dg.rhs(P, q0[0], central=True)
    s = bb.Solver(VX, EToV, rho, kappa, N)
    bb.bbdg_set_flux(s.ctx, bb.BBDG_FLUX_CENTRAL)
    q = torch.tensor(inputs.abi_layout(q0), device="cuda")
    r = torch.empty_like(q)
    bb.bbdg_rhs(s.ctx, q, r)
    assert rel(inputs.oracle_layout(r.cpu().numpy())[0], want) < 1e-12
    s.close()


def test_step_f64_config_c1(bb):
    """N = 3, 4^3 x 6 = 384 tets, standing-mode initial state, dt = 0.25 h/(N+1)^2, 50
    LSERK4 steps: the GPU state matches the oracle's to 1e-12 after every 10 steps."""
    N, n = 3, 4
    VX, EToV = inputs.kuhn_cube_mesh(n)
    K = len(EToV)
    P = dg.make_problem(VX, EToV, N, np.ones(K), np.ones(K))
    q0 = np.ascontiguousarray(dg.interpolate_state(P, dg.standing_mode(0.0)))
    dt = 0.25 * (1.0 / n) / (N + 1) ** 2
    s = bb.Solver(VX, EToV, np.ones(K), np.ones(K), N)
    q = torch.tensor(inputs.abi_layout(q0[None]), device="cuda")
    res = torch.zeros_like(q)
    scratch = torch.empty_like(q)
    qo, reso = q0.copy(), np.zeros_like(q0)
    for chunk in range(5):
        bb.bbdg_step(s.ctx, q, res, scratch, chunk * 10 * dt, dt, 10)
        qo, reso = _advance(P, qo, reso, chunk * 10 * dt, dt, 10)
        assert rel(inputs.oracle_layout(q.cpu().numpy())[0], qo) < 1e-12
        assert rel(inputs.oracle_layout(res.cpu().numpy())[0], reso) < 1e-12
    # and the solution is the standing mode to discretisation accuracy
    err = dg.l2_error(P, inputs.oracle_layout(q.cpu().numpy())[0], dg.standing_mode(50 * dt))
    assert err < 2e-3
    s.close()


def _advance(P, q, res, t, dt, n):
    for i in range(n):
        q, res = dg.lserk4_step(lambda x, tt: dg.rhs(P, x), q, res, t + i * dt, dt)
    return q, res


def test_step_odd_steps_and_shots(bb):
    """S = 3 shots, 3 steps (odd: the result comes back through the ping-pong copy)."""
    N = 2
    VX, EToV, rho, kappa = make(2, N)
    K = len(EToV)
    P = dg.make_problem(VX, EToV, N, rho, kappa)
    q0 = inputs.random_state(K, N, S=3)
    dt = 0.25 * 0.5 / 9 / np.sqrt(kappa.max())
    s = bb.Solver(VX, EToV, rho, kappa, N)
    q = torch.tensor(inputs.abi_layout(q0), device="cuda")
    res = torch.zeros_like(q)
    bb.bbdg_step(s.ctx, q, res, torch.empty_like(q), 0.0, dt, 3)
    got = inputs.oracle_layout(q.cpu().numpy())
    for sh in range(3):
        want, _ = _advance(P, q0[sh], np.zeros_like(q0[sh]), 0.0, dt, 3)
        assert rel(got[sh], want) < 1e-12
    s.close()


def test_sources_and_receivers(bb):
    """Two shots, Ricker point sources (two in shot 0, one in shot 1), 16 receivers,
    20 steps from rest."""
    N = 3
    VX, EToV, rho, kappa = make(3, N)
    K = len(EToV)
    P = dg.make_problem(VX, EToV, N, rho, kappa)
    xs = np.array([[0.1, -0.2, 0.05], [-0.3, 0.25, -0.1], [0.2, 0.2, 0.2]])
    shots = np.array([0, 0, 1])
    rec_xyz = inputs.receiver_plane(1 / 3, count_per_side=4)
    src = dg.make_sources(P, xs, shot=shots, f0=10.0, t0=0.05)
    rec = dg.make_receivers(P, rec_xyz)
    dt = 0.25 * (1 / 3) / 16 / np.sqrt(kappa.max())
    nsteps = 20
    s = bb.Solver(VX, EToV, rho, kappa, N)
    bb.bbdg_set_sources(s.ctx, xs, shots, 10.0, 0.05)
    bb.bbdg_set_receivers(s.ctx, rec_xyz)
    q = torch.zeros((2, K, P.Np, 4), device="cuda", dtype=torch.float64)
    res = torch.zeros_like(q)
    traces = torch.zeros((nsteps, 2, len(rec_xyz)), device="cuda", dtype=torch.float64)
    bb.bbdg_step(s.ctx, q, res, torch.empty_like(q), 0.0, dt, nsteps, traces=traces)
    got_q = inputs.oracle_layout(q.cpu().numpy())
    got_tr = traces.cpu().numpy()
    for sh in range(2):
        want_q, _, want_tr = dg.run(P, np.zeros((K, 4, P.Np)), 0.0, dt, nsteps, src=src, rec=rec, shot=sh)
        assert rel(got_q[sh], want_q) < 1e-12
        assert rel(got_tr[:, sh], want_tr) < 1e-12
    s.close()


def test_rhs_rejects_bad_arguments(bb):
    N = 2
    VX, EToV, rho, kappa = make(1, N)
    s = bb.Solver(VX, EToV, rho, kappa, N)
    q = torch.zeros((1, len(EToV), 10, 4), device="cuda", dtype=torch.float64)
    with pytest.raises(bb.BBDGError):
        bb.bbdg_rhs(s.ctx, q, q)
    with pytest.raises(bb.BBDGError) as ei:
        bb.bbdg_setup_operators(s.ctx, 11)
    assert ei.value.code == -2
    s.close()
