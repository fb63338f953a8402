"""GPU parity of the tensor-core nodal path (basis BBDG_NODAL_TC: one product
[D^r D^s D^t L^1..L^4] x per-element columns, TF32 with a high/low split) against the
oracle: the nodal right-hand side is V_B A_BB V_B^{-1} applied to nodal values (both bases
span P^N, Section 4.1), so the oracle's BB right-hand side mapped to nodal values is the
expected result.  FP32 tolerance: 2e-5 in the relative 2-norm (the split products carry
FP32 accuracy; the FP32 SIMT nodal kernel meets the same bound)."""
import numpy as np
import pytest

from oracle import dg, nodal
from paper_1512_06025_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 2e-5


@pytest.fixture(scope="module")
def bb():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1512_06025_gb300 import bbdg
    return bbdg


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def problem(n, jitter=0.1):
    VX, EToV = inputs.kuhn_cube_mesh(n, jitter=jitter)
    K = len(EToV)
    c = inputs.uniform_wavespeed(K)
    rho = np.random.default_rng(5).uniform(0.5, 2.0, K)
    return VX, EToV, rho, rho * c * c


@pytest.mark.parametrize("N", range(1, 11))
def test_tc_rhs_matches_oracle(bb, N):
    """Node-row kernel: K = 162 (3^3 x 6): 10.1 element tiles of 16 (N <= 7) or 20.25 of 8, a
    ragged tail."""
    VX, EToV, rho, kappa = problem(3)
    K = len(EToV)
    P = dg.make_problem(VX, EToV, N, rho, kappa)
    cbb = inputs.random_state(K, N)[0]
    want = nodal.to_nodal(N, dg.rhs(P, cbb))
    s = bb.Solver(VX, EToV, rho, kappa, N, basis=bb.BBDG_NODAL_TC, precision=bb.BBDG_F32)
    bb.bbdg_set_stage_form(s.ctx, bb.BBDG_FORM_GROUP, 0)        # the node-row kernel at every N
    q = torch.tensor(inputs.abi_layout(nodal.to_nodal(N, cbb)[None]), device="cuda", dtype=torch.float32)
    r = torch.full_like(q, float("nan"))
    bb.bbdg_rhs(s.ctx, q, r)
    bb.bbdg_device_status(s.ctx)
    got = inputs.oracle_layout(r.cpu().numpy())[0].astype(np.float64)
    s.close()
    assert np.isfinite(got).all()
    assert rel(got, want) < TOL, rel(got, want)
    # every element and field, not only the norm: the worst element's error stays at the
    # FP32 level of that element's own scale
    err = np.linalg.norm(got - want, axis=2) / np.linalg.norm(want, axis=(1, 2))[:, None]
    assert err.max() < 20 * TOL, err.max()


def test_tc_equals_simt_nodal(bb):
    """The tensor-core and SIMT FP32 nodal kernels agree to FP32 rounding (N = 5, S = 2)."""
    N, S = 5, 2
    VX, EToV, rho, kappa = problem(3)
    K = len(EToV)
    q0 = inputs.random_state(K, N, S=S)
    q = torch.tensor(inputs.abi_layout(q0), device="cuda", dtype=torch.float32)
    outs = []
    for basis in (bb.BBDG_NODAL, bb.BBDG_NODAL_TC):
        s = bb.Solver(VX, EToV, rho, kappa, N, basis=basis, precision=bb.BBDG_F32)
        r = torch.empty_like(q)
        bb.bbdg_rhs(s.ctx, q, r)
        outs.append(r.cpu().numpy().astype(np.float64))
        s.close()
    assert rel(outs[1], outs[0]) < 1e-5


def test_tc_steps_with_shots_match_oracle(bb):
    """S = 3 shots, 3 LSERK4 steps (odd: the result returns through the ping-pong copy),
    against the oracle's BB steps mapped to nodal values."""
    N, S, n = 4, 3, 3
    VX, EToV, rho, kappa = problem(n)
    K = len(EToV)
    P = dg.make_problem(VX, EToV, N, rho, kappa)
    cbb = inputs.random_state(K, N, S=S)
    dt = 0.25 * (1.0 / n) / (N + 1) ** 2 / np.sqrt(kappa / rho).max()
    want = []
    for sh in range(S):
        qo, ro = cbb[sh], np.zeros_like(cbb[sh])
        for i in range(3):
            qo, ro = dg.lserk4_step(lambda x, tt: dg.rhs(P, x), qo, ro, i * dt, dt)
        want.append(nodal.to_nodal(N, qo))
    want = np.stack(want)
    s = bb.Solver(VX, EToV, rho, kappa, N, basis=bb.BBDG_NODAL_TC, precision=bb.BBDG_F32)
    q = torch.tensor(inputs.abi_layout(np.stack([nodal.to_nodal(N, c) for c in cbb])), device="cuda",
                     dtype=torch.float32)
    bb.bbdg_step(s.ctx, q, torch.zeros_like(q), torch.empty_like(q), 0.0, dt, 3)
    bb.bbdg_device_status(s.ctx)
    got = inputs.oracle_layout(q.cpu().numpy()).astype(np.float64)
    s.close()
    assert rel(got, want) < TOL, rel(got, want)


def test_tc_full_size_workload(bb):
    """The benchmark's workload in its launch configuration: N = 7, 16^3 x 6 = 24576
    elements, uniform-random wavespeed; the whole right-hand side against the oracle."""
    N, n = 7, 16
    VX, EToV = inputs.kuhn_cube_mesh(n)
    K = len(EToV)
    rho, kappa = inputs.materials_from_wavespeed(inputs.uniform_wavespeed(K))
    P = dg.make_problem(VX, EToV, N, rho, kappa)
    cbb = inputs.random_state(K, N)[0]
    want = nodal.to_nodal(N, dg.rhs(P, cbb))
    s = bb.Solver(VX, EToV, rho, kappa, N, basis=bb.BBDG_NODAL_TC, precision=bb.BBDG_F32)
    q = torch.tensor(inputs.abi_layout(nodal.to_nodal(N, cbb)[None]), device="cuda", dtype=torch.float32)
    r = torch.full_like(q, float("nan"))
    bb.bbdg_rhs(s.ctx, q, r)
    bb.bbdg_device_status(s.ctx)
    got = inputs.oracle_layout(r.cpu().numpy())[0].astype(np.float64)
    s.close()
    assert np.isfinite(got).all()
    assert rel(got, want) < TOL, rel(got, want)


def test_tc_needs_fp32(bb):
    VX, EToV, rho, kappa = problem(1, jitter=0.0)
    with pytest.raises(bb.BBDGError) as e:
        bb.Solver(VX, EToV, rho, kappa, 3, basis=bb.BBDG_NODAL_TC, precision=bb.BBDG_F64)
    assert e.value.code == -2


@pytest.mark.parametrize("N", range(1, 7))
def test_rows_form_rhs_matches_oracle(bb, N):
    """The element-row form (BBDG_FORM_ROWS: 32 elements x 4 fields on the MMA rows, the full
    operator [D^r D^s D^t L^0..L^3] streamed) against the oracle.  K = 162: 5.06 CTAs of 32
    elements, a ragged last one."""
    VX, EToV, rho, kappa = problem(3)
    K = len(EToV)
    P = dg.make_problem(VX, EToV, N, rho, kappa)
    cbb = inputs.random_state(K, N)[0]
    want = nodal.to_nodal(N, dg.rhs(P, cbb))
    s = bb.Solver(VX, EToV, rho, kappa, N, basis=bb.BBDG_NODAL_TC, precision=bb.BBDG_F32)
    bb.bbdg_set_stage_form(s.ctx, bb.BBDG_FORM_ROWS, 0)
    q = torch.tensor(inputs.abi_layout(nodal.to_nodal(N, cbb)[None]), device="cuda", dtype=torch.float32)
    r = torch.full_like(q, float("nan"))
    bb.bbdg_rhs(s.ctx, q, r)
    bb.bbdg_device_status(s.ctx)
    got = inputs.oracle_layout(r.cpu().numpy())[0].astype(np.float64)
    s.close()
    assert np.isfinite(got).all()
    assert rel(got, want) < TOL, rel(got, want)
    err = np.linalg.norm(got - want, axis=2) / np.linalg.norm(want, axis=(1, 2))[:, None]
    assert err.max() < 20 * TOL, err.max()


@pytest.mark.parametrize("bc", ["mirror", "absorbing"])
def test_rows_form_steps_with_shots(bb, bc):
    """Element-row form: S = 3 shots, 3 LSERK4 steps, both boundary conditions, against the
    node-row form (same operator, FP32 rounding apart) and finite; wrong forms refused."""
    N, S = 3, 3
    VX, EToV, rho, kappa = problem(3)
    K = len(EToV)
    q0 = torch.tensor(inputs.abi_layout(inputs.random_state(K, N, S=S, seed=12)), device="cuda", dtype=torch.float32)
    outs = []
    for form in (bb.BBDG_FORM_GROUP, bb.BBDG_FORM_ROWS):
        s = bb.Solver(VX, EToV, rho, kappa, N, basis=bb.BBDG_NODAL_TC, precision=bb.BBDG_F32)
        if bc == "absorbing":
            bb.bbdg_set_boundary(s.ctx, bb.BBDG_BC_ABSORBING)
        bb.bbdg_set_stage_form(s.ctx, form, 0)
        q, res = q0.clone(), torch.zeros_like(q0)
        bb.bbdg_step(s.ctx, q, res, torch.empty_like(q0), 0.0, 2e-3, 3)
        bb.bbdg_device_status(s.ctx)
        outs.append(q.cpu().numpy().astype(np.float64))
        s.close()
    assert np.isfinite(outs[1]).all()
    assert rel(outs[1], outs[0]) < 1e-5
    s = bb.Solver(VX, EToV, rho, kappa, 7, basis=bb.BBDG_NODAL_TC, precision=bb.BBDG_F32)
    with pytest.raises(bb.BBDGError):
        bb.bbdg_set_stage_form(s.ctx, bb.BBDG_FORM_ROWS, 0)          # N > 6
    s.close()
    s = bb.Solver(VX, EToV, rho, kappa, 3, precision=bb.BBDG_F32)
    with pytest.raises(bb.BBDGError):
        bb.bbdg_set_stage_form(s.ctx, bb.BBDG_FORM_ROWS, 0)          # BB basis
    s.close()
