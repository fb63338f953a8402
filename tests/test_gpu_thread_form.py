"""GPU parity of the element-per-thread stage kernel (bbdg_set_stage_form(BBDG_FORM_THREAD),
N <= 2) against the oracle: right-hand side in FP64 (1e-12) and FP32 (1e-5, also element by
element), mirror and absorbing boundary, shots with point sources over LSERK4 steps,
per-shot media, graph replay, agreement with the group kernel, and the form's refusals."""
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


def make(n, seed=2):
    VX, EToV = inputs.kuhn_cube_mesh(n, jitter=0.1)
    K = len(EToV)
    c = inputs.uniform_wavespeed(K, seed=seed)
    rho = np.random.default_rng(seed + 10).uniform(0.5, 2.0, K)
    return VX, EToV, rho, rho * c * c


@pytest.mark.parametrize("N", [1, 2])
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("bc", ["mirror", "absorbing"])
def test_thread_rhs(bb, N, prec, bc):
    """162 jittered tets (two 128-thread blocks, the second ragged), heterogeneous media."""
    VX, EToV, rho, kappa = make(3)
    K = len(EToV)
    P = dg.make_problem(VX, EToV, N, rho, kappa, bc=bc)
    q0 = inputs.random_state(K, N)[0]
    if prec == "f32":
        q0 = q0.astype(np.float32).astype(np.float64)
    want = dg.rhs(P, q0)
    s = bb.Solver(VX, EToV, rho, kappa, N, precision=bb.BBDG_F64 if prec == "f64" else bb.BBDG_F32)
    if bc == "absorbing":
        bb.bbdg_set_boundary(s.ctx, bb.BBDG_BC_ABSORBING)
    bb.bbdg_set_stage_form(s.ctx, bb.BBDG_FORM_THREAD, 0)
    q = torch.tensor(inputs.abi_layout(q0[None]), device="cuda", dtype=s.torch_dtype)
    r = torch.full_like(q, float("nan"))
    bb.bbdg_rhs(s.ctx, q, r)
    got = inputs.oracle_layout(r.cpu().numpy())[0].astype(np.float64)
    s.close()
    tol = 1e-12 if prec == "f64" else 1e-5
    assert np.isfinite(got).all()
    assert rel(got, want) < tol, rel(got, want)
    assert elem_rel(got, want) < 10 * tol, elem_rel(got, want)


@pytest.mark.parametrize("N", [1, 2])
def test_thread_shots_sources_steps(bb, N):
    """S = 3 shots from rest, FP64, 10 LSERK4 steps, one Ricker source per shot (two in
    shot 1), against the oracle shot by shot."""
    n, S = 3, 3
    VX, EToV, rho, kappa = make(n)
    K = len(EToV)
    P = dg.make_problem(VX, EToV, N, rho, kappa)
    xs = np.vstack([inputs.random_points(3, -0.4, 0.4, seed=3), [[0.1, -0.05, 0.2]]])
    shots = np.array([0, 1, 2, 1])
    src = dg.make_sources(P, xs, shot=shots)
    dt = 0.25 * (1 / n) / (N + 1) ** 2 / 3.0
    s = bb.Solver(VX, EToV, rho, kappa, N)
    bb.bbdg_set_sources(s.ctx, xs, shots, 10.0, 0.05)
    bb.bbdg_set_stage_form(s.ctx, bb.BBDG_FORM_THREAD, 0)
    q = torch.zeros((S, K, P.Np, 4), device="cuda", dtype=torch.float64)
    bb.bbdg_step(s.ctx, q, torch.zeros_like(q), torch.empty_like(q), 0.0, dt, 10)
    got = inputs.oracle_layout(q.cpu().numpy())
    s.close()
    for sh in range(S):
        want, _, _ = dg.run(P, np.zeros((K, 4, P.Np)), 0.0, dt, 10, src=src, shot=sh)
        assert rel(got[sh], want) < 1e-12, (sh, rel(got[sh], want))


def test_thread_per_shot_media_graph_and_group_agreement(bb):
    """FP32, N = 2, 2 shots with their own media: graph replay equals stream-ordered steps
    bit for bit, and the thread form agrees with the group kernel to FP32 rounding."""
    N = 2
    VX, EToV, rho, kappa = make(4)
    K = len(EToV)
    rng = np.random.default_rng(31)
    rho2 = rng.uniform(0.5, 2.0, (2, K))
    kap2 = rho2 * rng.uniform(1.0, 3.0, (2, K)) ** 2
    q0 = torch.tensor(inputs.abi_layout(inputs.random_state(K, N, S=2, seed=13)), device="cuda", dtype=torch.float32)
    outs = []
    for form in (bb.BBDG_FORM_GROUP, bb.BBDG_FORM_THREAD):
        s = bb.Solver(VX, EToV, rho, kappa, N, precision=bb.BBDG_F32)
        s.set_materials(kap2, rho2)
        bb.bbdg_set_stage_form(s.ctx, form, 0)
        q, res = q0.clone(), torch.zeros_like(q0)
        bb.bbdg_step(s.ctx, q, res, torch.empty_like(q0), 0.0, 1e-3, 3)
        if form == bb.BBDG_FORM_THREAD:
            qg, rg = q0.clone(), torch.zeros_like(q0)
            bb.bbdg_step_graph(s.ctx, qg, rg, torch.empty_like(q0), 0.0, 1e-3, 3)
            torch.cuda.synchronize()
            assert torch.equal(qg, q) and torch.equal(rg, res)
        outs.append(q.cpu().numpy().astype(np.float64))
        s.close()
    assert rel(outs[1], outs[0]) < 1e-5


def test_thread_form_refusals(bb):
    VX, EToV, rho, kappa = make(2)
    for kwargs in ({"N": 3}, {"N": 2, "basis": bb.BBDG_NODAL}, {"N": 2, "precision": bb.BBDG_F32_LIFT64}):
        N = kwargs.pop("N")
        s = bb.Solver(VX, EToV, rho, kappa, N, **kwargs)
        with pytest.raises(bb.BBDGError) as e:
            bb.bbdg_set_stage_form(s.ctx, bb.BBDG_FORM_THREAD, 0)
        assert e.value.code == -2
        s.close()


@pytest.mark.parametrize("N", [1, 2])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_group_kernel_low_orders(bb, N, prec):
    """The group kernel (no longer the default at N <= 2) against the oracle at N = 1, 2."""
    VX, EToV, rho, kappa = make(3)
    K = len(EToV)
    P = dg.make_problem(VX, EToV, N, rho, kappa)
    q0 = inputs.random_state(K, N)[0]
    if prec == "f32":
        q0 = q0.astype(np.float32).astype(np.float64)
    want = dg.rhs(P, q0)
    s = bb.Solver(VX, EToV, rho, kappa, N, precision=bb.BBDG_F64 if prec == "f64" else bb.BBDG_F32)
    bb.bbdg_set_stage_form(s.ctx, bb.BBDG_FORM_GROUP, 0)
    q = torch.tensor(inputs.abi_layout(q0[None]), device="cuda", dtype=s.torch_dtype)
    r = torch.empty_like(q)
    bb.bbdg_rhs(s.ctx, q, r)
    got = inputs.oracle_layout(r.cpu().numpy())[0].astype(np.float64)
    s.close()
    tol = 1e-12 if prec == "f64" else 1e-5
    assert rel(got, want) < tol, rel(got, want)
    assert elem_rel(got, want) < 10 * tol, elem_rel(got, want)
