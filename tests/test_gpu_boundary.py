"""GPU parity of the absorbing boundary option (zero exterior state on boundary faces,
bbdg_set_boundary) against the oracle, for the BB and both nodal paths; and the rebuild of
a captured graph after the device data it refers to are replaced."""
import numpy as np
import pytest

from oracle import dg, nodal
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


def make(n=3, seed=2):
    VX, EToV = inputs.kuhn_cube_mesh(n, jitter=0.1)
    K = len(EToV)
    c = inputs.uniform_wavespeed(K, seed=seed)
    rho = np.random.default_rng(seed + 10).uniform(0.5, 2.0, K)
    return VX, EToV, rho, rho * c * c


@pytest.mark.parametrize("N", range(1, 11))
def test_bb_rhs_absorbing_f64(bb, N):
    VX, EToV, rho, kappa = make(3 if N <= 6 else 2)
    K = len(EToV)
    P = dg.make_problem(VX, EToV, N, rho, kappa, bc="absorbing")
    q0 = inputs.random_state(K, N)[0]
    want = dg.rhs(P, q0)
    s = bb.Solver(VX, EToV, rho, kappa, N)
    bb.bbdg_set_boundary(s.ctx, bb.BBDG_BC_ABSORBING)
    q = torch.tensor(inputs.abi_layout(q0[None]), device="cuda")
    r = torch.empty_like(q)
    bb.bbdg_rhs(s.ctx, q, r)
    got = inputs.oracle_layout(r.cpu().numpy())[0]
    s.close()
    assert rel(got, want) < 1e-12, rel(got, want)


@pytest.mark.parametrize("basis", ["bb_f32", "nodal_f64", "nodal_tc"])
def test_absorbing_other_paths(bb, basis):
    N = 4
    VX, EToV, rho, kappa = make()
    K = len(EToV)
    P = dg.make_problem(VX, EToV, N, rho, kappa, bc="absorbing")
    cbb = inputs.random_state(K, N)[0]
    if basis == "bb_f32":
        cbb = cbb.astype(np.float32).astype(np.float64)
        want, q0 = dg.rhs(P, cbb), cbb
        s = bb.Solver(VX, EToV, rho, kappa, N, precision=bb.BBDG_F32)
        dt, tol = torch.float32, 1e-5
    else:
        want, q0 = nodal.to_nodal(N, dg.rhs(P, cbb)), nodal.to_nodal(N, cbb)
        if basis == "nodal_f64":
            s = bb.Solver(VX, EToV, rho, kappa, N, basis=bb.BBDG_NODAL)
            dt, tol = torch.float64, 1e-11
        else:
            q0 = q0.astype(np.float32).astype(np.float64)
            want = nodal.to_nodal(N, dg.rhs(P, nodal.from_nodal(N, q0)))
            s = bb.Solver(VX, EToV, rho, kappa, N, basis=bb.BBDG_NODAL_TC, precision=bb.BBDG_F32)
            dt, tol = torch.float32, 2e-5
    bb.bbdg_set_boundary(s.ctx, bb.BBDG_BC_ABSORBING)
    q = torch.tensor(inputs.abi_layout(q0[None]), device="cuda", dtype=dt)
    r = torch.empty_like(q)
    bb.bbdg_rhs(s.ctx, q, r)
    got = inputs.oracle_layout(r.cpu().numpy())[0].astype(np.float64)
    s.close()
    assert rel(got, want) < tol, rel(got, want)


def test_absorbing_steps_and_energy(bb):
    """Five LSERK4 steps with the absorbing boundary match the oracle, and the discrete
    energy decreases (outflow through the boundary)."""
    N, n = 3, 3
    VX, EToV, rho, kappa = make(n)
    K = len(EToV)
    P = dg.make_problem(VX, EToV, N, rho, kappa, bc="absorbing")
    q0 = inputs.random_state(K, N)[0]
    dt = 0.25 * (1.0 / n) / (N + 1) ** 2 / np.sqrt(kappa / rho).max()
    want, _, _ = dg.run(P, q0, 0.0, dt, 5)
    s = bb.Solver(VX, EToV, rho, kappa, N)
    bb.bbdg_set_boundary(s.ctx, bb.BBDG_BC_ABSORBING)
    q = torch.tensor(inputs.abi_layout(q0[None]), device="cuda")
    bb.bbdg_step(s.ctx, q, torch.zeros_like(q), torch.empty_like(q), 0.0, dt, 5)
    got = inputs.oracle_layout(q.cpu().numpy())[0]
    assert rel(got, want) < 1e-12, rel(got, want)
    assert dg.energy(P, got) < dg.energy(P, q0)
    # the adjoint is built for the mirror boundary
    with pytest.raises(bb.BBDGError):
        bb.bbdg_adjoint_rhs(s.ctx, q, torch.empty_like(q))
    s.close()


def test_graph_rebuilt_after_device_data_change(bb):
    """A graph captured before bbdg_set_materials (which replaces the geometry records) and
    bbdg_set_boundary is rebuilt: its replay equals stream-ordered steps with the new data."""
    N, n = 3, 2
    VX, EToV, rho, kappa = make(n)
    K = len(EToV)
    q0 = torch.tensor(inputs.abi_layout(inputs.random_state(K, N)), device="cuda")
    dt = 1e-3
    s = bb.Solver(VX, EToV, rho, kappa, N)
    q, res, scr = q0.clone(), torch.zeros_like(q0), torch.empty_like(q0)
    bb.bbdg_step_graph(s.ctx, q, res, scr, 0.0, dt, 2)                 # captured with the old data
    for change in ("materials", "boundary"):
        if change == "materials":
            bb.bbdg_set_materials(s.ctx, 2.0 * kappa, rho)
        else:
            bb.bbdg_set_boundary(s.ctx, bb.BBDG_BC_ABSORBING)
        q.copy_(q0)
        res.zero_()
        bb.bbdg_step_graph(s.ctx, q, res, scr, 0.0, dt, 2)
        q2, res2 = q0.clone(), torch.zeros_like(q0)
        bb.bbdg_step(s.ctx, q2, res2, torch.empty_like(q0), 0.0, dt, 2)
        torch.cuda.synchronize()
        assert torch.equal(q, q2) and torch.equal(res, res2), change
    s.close()
