"""GPU parity of the element-per-warp stage kernel (bbdg_set_stage_form(BBDG_FORM_WARP))
against the oracle: right-hand side for N = 1..10 in FP64 and FP32, both boundary
options, several warps per CTA, shots with point sources over LSERK4 steps, graph replay;
and its agreement with the group kernel."""
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


def make(n, seed=2):
    VX, EToV = inputs.kuhn_cube_mesh(n, jitter=0.1)
    K = len(EToV)
    c = inputs.uniform_wavespeed(K, seed=seed)
    rho = np.random.default_rng(seed + 10).uniform(0.5, 2.0, K)
    return VX, EToV, rho, rho * c * c


@pytest.mark.parametrize("N", range(1, 11))
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_warp_rhs(bb, N, prec):
    """Mirror boundary; K = 162 or 48 jittered tets (a ragged last CTA for every W)."""
    VX, EToV, rho, kappa = make(3 if N <= 6 else 2)
    K = len(EToV)
    P = dg.make_problem(VX, EToV, N, rho, kappa)
    q0 = inputs.random_state(K, N)[0]
    if prec == "f32":
        q0 = q0.astype(np.float32).astype(np.float64)
    want = dg.rhs(P, q0)
    s = bb.Solver(VX, EToV, rho, kappa, N, precision=bb.BBDG_F64 if prec == "f64" else bb.BBDG_F32)
    W = 1 + N % 8 if prec == "f64" else 8
    bb.bbdg_set_stage_form(s.ctx, bb.BBDG_FORM_WARP, W)
    q = torch.tensor(inputs.abi_layout(q0[None]), device="cuda", dtype=s.torch_dtype)
    r = torch.empty_like(q)
    bb.bbdg_rhs(s.ctx, q, r)
    got = inputs.oracle_layout(r.cpu().numpy())[0].astype(np.float64)
    s.close()
    tol = 1e-12 if prec == "f64" else 1e-5
    assert rel(got, want) < tol, rel(got, want)


@pytest.mark.parametrize("N", [2, 7])
def test_warp_absorbing(bb, N):
    VX, EToV, rho, kappa = make(3)
    K = len(EToV)
    P = dg.make_problem(VX, EToV, N, rho, kappa, bc="absorbing")
    q0 = inputs.random_state(K, N)[0]
    want = dg.rhs(P, q0)
    s = bb.Solver(VX, EToV, rho, kappa, N)
    bb.bbdg_set_boundary(s.ctx, bb.BBDG_BC_ABSORBING)
    bb.bbdg_set_stage_form(s.ctx, bb.BBDG_FORM_WARP, 4)
    q = torch.tensor(inputs.abi_layout(q0[None]), device="cuda")
    r = torch.empty_like(q)
    bb.bbdg_rhs(s.ctx, q, r)
    got = inputs.oracle_layout(r.cpu().numpy())[0]
    s.close()
    assert rel(got, want) < 1e-12, rel(got, want)


def test_warp_shots_sources_steps(bb):
    """S = 3 shots, one Ricker source each, 10 LSERK4 steps from rest, FP64."""
    N, n, S = 4, 3, 3
    VX, EToV, rho, kappa = make(n)
    K = len(EToV)
    P = dg.make_problem(VX, EToV, N, rho, kappa)
    xs = inputs.random_points(S, -0.4, 0.4, seed=3)
    shots = np.arange(S)
    src = dg.make_sources(P, xs, shot=shots)
    dt = 0.25 * (1 / n) / (N + 1) ** 2 / 3.0
    nsteps = 10
    s = bb.Solver(VX, EToV, rho, kappa, N)
    bb.bbdg_set_sources(s.ctx, xs, shots, 10.0, 0.05)
    bb.bbdg_set_stage_form(s.ctx, bb.BBDG_FORM_WARP, 16)
    q = torch.zeros((S, K, P.Np, 4), device="cuda", dtype=torch.float64)
    res = torch.zeros_like(q)
    bb.bbdg_step(s.ctx, q, res, torch.empty_like(q), 0.0, dt, nsteps)
    got = inputs.oracle_layout(q.cpu().numpy())
    s.close()
    for sh in range(S):
        want, _, _ = dg.run(P, np.zeros((K, 4, P.Np)), 0.0, dt, nsteps, src=src, shot=sh)
        assert rel(got[sh], want) < 1e-12, (sh, rel(got[sh], want))


def test_warp_equals_group_and_graph(bb):
    """FP32, N = 6, 2 shots: the warp form agrees with the group kernel to rounding over 5
    steps, its graph replay equals its stream-ordered steps bit for bit, and switching the
    form back gives the group kernel's result again (the captured graph is rebuilt)."""
    N, S = 6, 2
    VX, EToV, rho, kappa = make(3)
    K = len(EToV)
    q0 = torch.tensor(inputs.abi_layout(inputs.random_state(K, N, S=S)), dtype=torch.float32, device="cuda")
    s = bb.Solver(VX, EToV, rho, kappa, N, precision=bb.BBDG_F32)
    dt = 1e-3

    def run(f):
        q, res = q0.clone(), torch.zeros_like(q0)
        f(s.ctx, q, res, torch.empty_like(q0), 0.0, dt, 5)
        torch.cuda.synchronize()
        return q.cpu().numpy().astype(np.float64)

    group = run(bb.bbdg_step_graph)
    bb.bbdg_set_stage_form(s.ctx, bb.BBDG_FORM_WARP, 8)
    warp_step, warp_graph = run(bb.bbdg_step), run(bb.bbdg_step_graph)
    bb.bbdg_set_stage_form(s.ctx, bb.BBDG_FORM_GROUP, 0)
    group_again = run(bb.bbdg_step_graph)
    s.close()
    assert np.array_equal(warp_step, warp_graph)
    assert np.array_equal(group, group_again)
    assert rel(warp_step, group) < 1e-6, rel(warp_step, group)


def test_warp_form_limits(bb):
    VX, EToV, rho, kappa = make(1)
    s = bb.Solver(VX, EToV, rho, kappa, 3, precision=bb.BBDG_F32_LIFT64)
    with pytest.raises(bb.BBDGError):
        bb.bbdg_set_stage_form(s.ctx, bb.BBDG_FORM_WARP, 8)
    s.close()
    s = bb.Solver(VX, EToV, rho, kappa, 3)
    for W in (0, 17):
        with pytest.raises(bb.BBDGError):
            bb.bbdg_set_stage_form(s.ctx, bb.BBDG_FORM_WARP, W)
    with pytest.raises(bb.BBDGError):
        bb.bbdg_set_stage_form(s.ctx, 7, 8)
    s.close()
    s = bb.Solver(VX, EToV, rho, kappa, 3, basis=bb.BBDG_NODAL)
    with pytest.raises(bb.BBDGError):
        bb.bbdg_set_stage_form(s.ctx, bb.BBDG_FORM_WARP, 8)
    s.close()


@pytest.mark.parametrize("N", [9, 10])
def test_group_form_fp64_high_order(bb, N):
    """FP64 at N >= 9 defaults to the element-per-warp form; with the group kernel selected
    explicitly, both agree with the oracle."""
    VX, EToV, rho, kappa = make(2)
    K = len(EToV)
    P = dg.make_problem(VX, EToV, N, rho, kappa)
    q0 = inputs.random_state(K, N)[0]
    want = dg.rhs(P, q0)
    s = bb.Solver(VX, EToV, rho, kappa, N)
    q = torch.tensor(inputs.abi_layout(q0[None]), device="cuda")
    outs = []
    for form in (None, bb.BBDG_FORM_GROUP):
        if form is not None:
            bb.bbdg_set_stage_form(s.ctx, form, 0)
        r = torch.empty_like(q)
        bb.bbdg_rhs(s.ctx, q, r)
        outs.append(inputs.oracle_layout(r.cpu().numpy())[0])
    s.close()
    for got in outs:
        assert rel(got, want) < 1e-12, rel(got, want)
