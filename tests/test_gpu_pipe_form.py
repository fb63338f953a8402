"""GPU parity of the warp-specialised pipelined stage kernel
(bbdg_set_stage_form(BBDG_FORM_PIPE)) against the oracle: right-hand side for N = 1..8 in
FP64 and FP32 (FP32 also element by element), the absorbing boundary, shots with point
sources over LSERK4 steps (including a group holding more sources than its per-group list),
shot tiles, graph replay, and agreement with the group kernel."""
import numpy as np
import pytest

from oracle import dg
from paper_1512_06025_gb300 import inputs
from conftest import elem_rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PIPE_N = range(1, 9)


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


@pytest.mark.parametrize("N", PIPE_N)
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_pipe_rhs(bb, N, prec):
    """Mirror boundary, heterogeneous media; 162 jittered tets (n = 3): many element groups
    per CTA and a ragged last group at every N."""
    VX, EToV, rho, kappa = make(3)
    K = len(EToV)
    P = dg.make_problem(VX, EToV, N, rho, kappa)
    q0 = inputs.random_state(K, N)[0]
    if prec == "f32":
        q0 = q0.astype(np.float32).astype(np.float64)
    want = dg.rhs(P, q0)
    s = bb.Solver(VX, EToV, rho, kappa, N, precision=bb.BBDG_F64 if prec == "f64" else bb.BBDG_F32)
    bb.bbdg_set_stage_form(s.ctx, bb.BBDG_FORM_PIPE, 0)
    q = torch.tensor(inputs.abi_layout(q0[None]), device="cuda", dtype=s.torch_dtype)
    r = torch.empty_like(q)
    bb.bbdg_rhs(s.ctx, q, r)
    got = inputs.oracle_layout(r.cpu().numpy())[0].astype(np.float64)
    bb.bbdg_device_status(s.ctx)
    s.close()
    if prec == "f64":
        assert rel(got, want) < 1e-12, rel(got, want)
        assert elem_rel(got, want) < 1e-11, elem_rel(got, want)
    else:
        assert rel(got, want) < 1e-5, rel(got, want)
        assert elem_rel(got, want) < 1e-5, elem_rel(got, want)


@pytest.mark.parametrize("N", [4, 7])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_pipe_many_groups_per_cta(bb, N, prec):
    """12^3 x 6 = 10368 jittered tets: more element groups than resident CTAs, so every CTA
    runs several pipelined iterations (the loads of one group overlap the work of the two
    before it) and the last group of the mesh is ragged at N = 4; right-hand side against
    the oracle, element by element."""
    VX, EToV, rho, kappa = make(12)
    K = len(EToV)
    P = dg.make_problem(VX, EToV, N, rho, kappa)
    q0 = inputs.random_state(K, N)[0]
    if prec == "f32":
        q0 = q0.astype(np.float32).astype(np.float64)
    want = dg.rhs(P, q0)
    s = bb.Solver(VX, EToV, rho, kappa, N, precision=bb.BBDG_F64 if prec == "f64" else bb.BBDG_F32)
    bb.bbdg_set_stage_form(s.ctx, bb.BBDG_FORM_PIPE, 0)
    q = torch.tensor(inputs.abi_layout(q0[None]), device="cuda", dtype=s.torch_dtype)
    r = torch.empty_like(q)
    first = None
    for _ in range(3):                      # repeated launches give the same bits
        bb.bbdg_rhs(s.ctx, q, r)
        out = r.cpu().numpy()
        if first is None:
            first = out
        assert np.array_equal(out, first)
    got = inputs.oracle_layout(first)[0].astype(np.float64)
    tol = 1e-12 if prec == "f64" else 1e-5
    assert rel(got, want) < tol, rel(got, want)
    assert elem_rel(got, want) < 10 * tol, elem_rel(got, want)
    bb.bbdg_device_status(s.ctx)
    s.close()


@pytest.mark.parametrize("N", [2, 7])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_pipe_absorbing(bb, N, prec):
    VX, EToV, rho, kappa = make(3)
    K = len(EToV)
    P = dg.make_problem(VX, EToV, N, rho, kappa, bc="absorbing")
    q0 = inputs.random_state(K, N)[0]
    if prec == "f32":
        q0 = q0.astype(np.float32).astype(np.float64)
    want = dg.rhs(P, q0)
    s = bb.Solver(VX, EToV, rho, kappa, N, precision=bb.BBDG_F64 if prec == "f64" else bb.BBDG_F32)
    bb.bbdg_set_boundary(s.ctx, bb.BBDG_BC_ABSORBING)
    bb.bbdg_set_stage_form(s.ctx, bb.BBDG_FORM_PIPE, 0)
    q = torch.tensor(inputs.abi_layout(q0[None]), device="cuda", dtype=s.torch_dtype)
    r = torch.empty_like(q)
    bb.bbdg_rhs(s.ctx, q, r)
    got = inputs.oracle_layout(r.cpu().numpy())[0].astype(np.float64)
    s.close()
    tol = 1e-12 if prec == "f64" else 1e-5
    assert rel(got, want) < tol, rel(got, want)
    assert elem_rel(got, want) < 10 * tol, elem_rel(got, want)


@pytest.mark.parametrize("N", [3, 6])
@pytest.mark.parametrize("tile", [1, 2])
def test_pipe_shots_sources_steps(bb, N, tile):
    """S = 4 shots from rest, FP64, 10 LSERK4 steps: shots 0-2 have one Ricker source each;
    shot 3 has twelve sources inside one element (more than a group's list holds, so that
    group scans the shot's whole list)."""
    n, S = 3, 4
    VX, EToV, rho, kappa = make(n)
    K = len(EToV)
    P = dg.make_problem(VX, EToV, N, rho, kappa)
    xs = inputs.random_points(3, -0.4, 0.4, seed=3)
    # twelve points inside the element that holds the first random point of shot 3
    rng = np.random.default_rng(7)
    centre = VX[EToV[40]].mean(axis=0)
    cluster = centre + 0.02 * (rng.random((12, 3)) - 0.5) / n
    xs = np.vstack([xs, cluster])
    shots = np.array([0, 1, 2] + [3] * 12)
    src = dg.make_sources(P, xs, shot=shots)
    dt = 0.25 * (1 / n) / (N + 1) ** 2 / 3.0
    nsteps = 10
    s = bb.Solver(VX, EToV, rho, kappa, N)
    bb.bbdg_set_sources(s.ctx, xs, shots, 10.0, 0.05)
    bb.bbdg_set_stage_form(s.ctx, bb.BBDG_FORM_PIPE, 0)
    bb.bbdg_set_launch_shape(s.ctx, 0, tile)
    q = torch.zeros((S, K, P.Np, 4), device="cuda", dtype=torch.float64)
    res = torch.zeros_like(q)
    bb.bbdg_step(s.ctx, q, res, torch.empty_like(q), 0.0, dt, nsteps)
    got = inputs.oracle_layout(q.cpu().numpy())
    s.close()
    for sh in range(S):
        want, _, _ = dg.run(P, np.zeros((K, 4, P.Np)), 0.0, dt, nsteps, src=src, shot=sh)
        assert rel(got[sh], want) < 1e-12, (sh, rel(got[sh], want))


@pytest.mark.parametrize("N", [5, 7])
def test_pipe_steps_f32(bb, N):
    """FP32 LSERK4: 3 steps from an FP64 state rounded to FP32 against the oracle (the first
    stage of each step skips the residual read, a_1 = 0), element by element."""
    n = 3
    VX, EToV, rho, kappa = make(n)
    K = len(EToV)
    P = dg.make_problem(VX, EToV, N, rho, kappa)
    q0 = inputs.random_state(K, N)[0].astype(np.float32).astype(np.float64)
    dt = 0.25 * (1 / n) / (N + 1) ** 2 / 3.0
    want, _, _ = dg.run(P, q0, 0.0, dt, 3)
    s = bb.Solver(VX, EToV, rho, kappa, N, precision=bb.BBDG_F32)
    bb.bbdg_set_stage_form(s.ctx, bb.BBDG_FORM_PIPE, 0)
    q = torch.tensor(inputs.abi_layout(q0[None]), device="cuda", dtype=torch.float32)
    res = torch.full_like(q, float("nan"))       # never read: stage 1 has a_1 = 0
    bb.bbdg_step(s.ctx, q, res, torch.empty_like(q), 0.0, dt, 3)
    got = inputs.oracle_layout(q.cpu().numpy())[0].astype(np.float64)
    s.close()
    assert rel(got, want) < 1e-5, rel(got, want)
    assert elem_rel(got, want) < 1e-5, elem_rel(got, want)


def test_pipe_equals_group_and_graph(bb):
    """FP32, N = 7, 2 shots: the pipelined form agrees with the group kernel to rounding over
    5 steps, its graph replay equals its stream-ordered steps bit for bit, and switching the
    form back gives the group kernel's result again (the captured graph is rebuilt)."""
    N, S = 7, 2
    VX, EToV, rho, kappa = make(3)
    K = len(EToV)
    q0 = torch.tensor(inputs.abi_layout(inputs.random_state(K, N, S=S)), dtype=torch.float32, device="cuda")
    s = bb.Solver(VX, EToV, rho, kappa, N, precision=bb.BBDG_F32)
    bb.bbdg_set_stage_form(s.ctx, bb.BBDG_FORM_GROUP, 0)
    dt = 1e-3

    def run(f):
        q, res = q0.clone(), torch.zeros_like(q0)
        f(s.ctx, q, res, torch.empty_like(q0), 0.0, dt, 5)
        torch.cuda.synchronize()
        return q.cpu().numpy().astype(np.float64)

    group = run(bb.bbdg_step_graph)
    bb.bbdg_set_stage_form(s.ctx, bb.BBDG_FORM_PIPE, 0)
    pipe_step, pipe_graph = run(bb.bbdg_step), run(bb.bbdg_step_graph)
    bb.bbdg_set_stage_form(s.ctx, bb.BBDG_FORM_GROUP, 0)
    group2 = run(bb.bbdg_step_graph)
    s.close()
    assert np.array_equal(pipe_step, pipe_graph)
    assert np.array_equal(group, group2)
    assert rel(pipe_step, group) < 1e-5, rel(pipe_step, group)


def test_pipe_form_checks(bb):
    """The form is refused where it is not built (N = 9, 10; the FP64 lift; the sparse E_L
    lift; the nodal basis)."""
    VX, EToV, rho, kappa = make(1)
    for N, kw in [(9, {}), (10, {}), (4, {"precision": bb.BBDG_F32_LIFT64}),
                  (4, {"lift_variant": bb.BBDG_LIFT_SPARSE_EL}), (4, {"basis": bb.BBDG_NODAL})]:
        s = bb.Solver(VX, EToV, rho, kappa, N, **kw)
        with pytest.raises(bb.BBDGError):
            bb.bbdg_set_stage_form(s.ctx, bb.BBDG_FORM_PIPE, 0)
        s.close()
