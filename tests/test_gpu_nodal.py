"""GPU parity of the dense nodal (Warp & Blend) path against the oracle: the library's
nodes equal the oracle's, and the nodal right-hand side equals V_B A_BB V_B^{-1} applied to
nodal values (both bases span P^N, so the discrete operators agree; Section 4.1)."""
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


@pytest.mark.parametrize("N", range(1, 11))
def test_library_nodes_match_oracle(bb, N):
    np.testing.assert_allclose(bb.bbdg_nodal_nodes(N), nodal.warp_blend_barycentric(N), atol=1e-14)


@pytest.mark.parametrize("N", [1, 2, 4, 7, 10])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_nodal_rhs_matches_oracle(bb, N, prec):
    VX, EToV = inputs.kuhn_cube_mesh(2, jitter=0.1)
    K = len(EToV)
    c = inputs.uniform_wavespeed(K)
    rho = np.random.default_rng(5).uniform(0.5, 2.0, K)
    kappa = rho * c * c
    P = dg.make_problem(VX, EToV, N, rho, kappa)
    cbb = inputs.random_state(K, N)[0]
    want = nodal.to_nodal(N, dg.rhs(P, cbb))
    qn = nodal.to_nodal(N, cbb)
    p = bb.BBDG_F64 if prec == "f64" else bb.BBDG_F32
    dt = torch.float64 if prec == "f64" else torch.float32
    s = bb.Solver(VX, EToV, rho, kappa, N, basis=bb.BBDG_NODAL, precision=p)
    q = torch.tensor(inputs.abi_layout(qn[None]), device="cuda", dtype=dt)
    r = torch.empty_like(q)
    bb.bbdg_rhs(s.ctx, q, r)
    got = inputs.oracle_layout(r.cpu().numpy())[0].astype(np.float64)
    s.close()
    # FP64: the nodal operators carry the change-of-basis conditioning (cond(V_B) ~ 1e3 at N = 9)
    tol = 1e-11 if prec == "f64" else 2e-5
    assert rel(got, want) < tol, rel(got, want)


def test_nodal_step_matches_bb_step(bb):
    """Three LSERK4 steps in the nodal basis equal the BB steps mapped to nodal values."""
    N = 3
    VX, EToV = inputs.kuhn_cube_mesh(2)
    K = len(EToV)
    rho, kappa = np.ones(K), np.ones(K)
    cbb = inputs.random_state(K, N)
    dt = 0.25 * 0.5 / 16
    s_bb = bb.Solver(VX, EToV, rho, kappa, N)
    s_nd = bb.Solver(VX, EToV, rho, kappa, N, basis=bb.BBDG_NODAL)
    q1 = torch.tensor(inputs.abi_layout(cbb), device="cuda")
    q2 = torch.tensor(inputs.abi_layout(nodal.to_nodal(N, cbb)), device="cuda")
    for s, q in ((s_bb, q1), (s_nd, q2)):
        bb.bbdg_step(s.ctx, q, torch.zeros_like(q), torch.empty_like(q), 0.0, dt, 3)
    assert rel(inputs.oracle_layout(q2.cpu().numpy()),
               nodal.to_nodal(N, inputs.oracle_layout(q1.cpu().numpy()))) < 1e-12
    s_bb.close()
    s_nd.close()
