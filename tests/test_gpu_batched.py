"""Batched shots (many independent sources sharing one mesh), shot tiling, and the CUDA
graph replay of bbdg_step_graph, against the oracle run shot by shot."""
import numpy as np
import pytest

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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def layered_problem(n, N):
    VX, EToV = inputs.kuhn_cube_mesh(n)
    c = inputs.layered_wavespeed(VX, EToV)
    rho, kappa = inputs.materials_from_wavespeed(c)
    return VX, EToV, rho, kappa


@pytest.mark.parametrize("ST", [1, 2, 4])
def test_shots_with_sources_match_oracle(bb, ST):
    """S = 4 shots, one Ricker source each (plus a second source in shot 2), layered
    wavespeed, 12 steps from rest, shot tile ST."""
    N, n, S = 3, 3, 4
    VX, EToV, rho, kappa = layered_problem(n, N)
    K = len(EToV)
    P = dg.make_problem(VX, EToV, N, rho, kappa)
    xs = inputs.random_points(S, -0.4, 0.4, seed=3)
    xs = np.concatenate([xs, [[0.05, 0.1, -0.2]]])
    shots = np.array([0, 1, 2, 3, 2])
    src = dg.make_sources(P, xs, shot=shots)
    dt = 0.25 * (1 / n) / (N + 1) ** 2 / 2.5
    nsteps = 12
    s = bb.Solver(VX, EToV, rho, kappa, N)
    bb.bbdg_set_sources(s.ctx, xs, shots, 10.0, 0.05)
    bb.bbdg_set_launch_shape(s.ctx, 4, ST)
    q = torch.zeros((S, K, P.Np, 4), device="cuda", dtype=torch.float64)
    res = torch.zeros_like(q)
    bb.bbdg_step(s.ctx, q, res, torch.empty_like(q), 0.0, dt, nsteps)
    got = inputs.oracle_layout(q.cpu().numpy())
    s.close()
    for sh in range(S):
        want, _, _ = dg.run(P, np.zeros((K, 4, P.Np)), 0.0, dt, nsteps, src=src, shot=sh)
        assert rel(got[sh], want) < 1e-12, (sh, rel(got[sh], want))


def test_graph_replay_equals_step(bb):
    """bbdg_step_graph: first call captures, second call replays; both equal bbdg_step
    exactly (same kernels, same arguments)."""
    N, n, S = 5, 2, 3
    VX, EToV, rho, kappa = layered_problem(n, N)
    K = len(EToV)
    xs = inputs.random_points(S, -0.4, 0.4, seed=3)
    s = bb.Solver(VX, EToV, rho, kappa, N, precision=bb.BBDG_F32)
    bb.bbdg_set_sources(s.ctx, xs, np.arange(S), 10.0, 0.05)
    bb.bbdg_set_receivers(s.ctx, inputs.receiver_plane(1 / n, 4))
    q0 = torch.tensor(inputs.abi_layout(inputs.random_state(K, N, S=S)), dtype=torch.float32, device="cuda")
    dt = 1e-3
    outs = []
    for mode in ("step", "graph"):
        q, res = q0.clone(), torch.zeros_like(q0)
        scratch = torch.empty_like(q0)
        tr = torch.zeros((7, S, 16), device="cuda", dtype=torch.float32)
        f = bb.bbdg_step if mode == "step" else bb.bbdg_step_graph
        f(s.ctx, q, res, scratch, 0.0, dt, 7, traces=tr)
        torch.cuda.synchronize()
        outs.append((q.clone(), res.clone(), tr.clone()))
        if mode == "graph":
            # replay from the same starting state: identical result
            q.copy_(q0)
            res.zero_()
            f(s.ctx, q, res, scratch, 0.0, dt, 7, traces=tr)
            torch.cuda.synchronize()
            outs.append((q.clone(), res.clone(), tr.clone()))
    s.close()
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert torch.equal(a, b)


def test_f32_batched_error_bound(bb):
    """FP32 one-step error from the rounded FP64 state: <= 1e-5 relative L2 per step."""
    N, n, S = 5, 3, 2
    VX, EToV, rho, kappa = layered_problem(n, N)
    K = len(EToV)
    P = dg.make_problem(VX, EToV, N, rho, kappa)
    q64 = inputs.random_state(K, N, S=S)
    q32 = q64.astype(np.float32)
    dt = 0.25 * (1 / n) / (N + 1) ** 2 / 2.5
    s = bb.Solver(VX, EToV, rho, kappa, N, precision=bb.BBDG_F32)
    q = torch.tensor(inputs.abi_layout(q32), device="cuda")
    bb.bbdg_step(s.ctx, q, torch.zeros_like(q), torch.empty_like(q), 0.0, dt, 1)
    got = inputs.oracle_layout(q.cpu().numpy()).astype(np.float64)
    s.close()
    for sh in range(S):
        want, _ = dg.lserk4_step(lambda x, t: dg.rhs(P, x), q32[sh].astype(np.float64), np.zeros_like(q64[sh]), 0.0, dt)
        assert rel(got[sh], want) < 1e-5


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_sources_through_the_ricker_peak(bb, prec):
    """The C4 set-up (N = 5, layered wavespeed, one Ricker source per shot, dt =
    0.25 h / (N + 1)^2 / c_max) on a 4^3 x 6 mesh, 2 shots, 150 steps captured in one graph:
    the run ends at t = 0.104, past the wavelet's peak at t0 = 0.05 (the 500 steps of the
    full-size C4 mesh end at t = 0.043, before it).  The state stays finite and matches the
    oracle shot by shot (FP64 1e-12, FP32 1e-5 relative)."""
    N, n, S = 5, 4, 2
    VX, EToV, rho, kappa = layered_problem(n, N)
    K = len(EToV)
    P = dg.make_problem(VX, EToV, N, rho, kappa)
    xs = inputs.random_points(S, -0.4, 0.4, seed=5)
    shots = np.arange(S)
    src = dg.make_sources(P, xs, shot=shots)
    dt = 0.25 * (1 / n) / (N + 1) ** 2 / 2.5
    nsteps = 150
    assert nsteps * dt > 2 * 0.05
    s = bb.Solver(VX, EToV, rho, kappa, N, precision=bb.BBDG_F64 if prec == "f64" else bb.BBDG_F32)
    bb.bbdg_set_sources(s.ctx, xs, shots, 10.0, 0.05)
    q = torch.zeros((S, K, P.Np, 4), device="cuda", dtype=s.torch_dtype)
    res = torch.zeros_like(q)
    bb.bbdg_step_graph(s.ctx, q, res, torch.empty_like(q), 0.0, dt, nsteps)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(q).all())
    got = inputs.oracle_layout(q.double().cpu().numpy())
    s.close()
    for sh in range(S):
        want, _, _ = dg.run(P, np.zeros((K, 4, P.Np)), 0.0, dt, nsteps, src=src, shot=sh)
        assert np.abs(want[:, 0]).max() > 0
        tol = 1e-12 if prec == "f64" else 1e-5
        assert rel(got[sh], want) < tol, (sh, rel(got[sh], want))
