"""The first LSERK4 stage has a_1 = 0 (Carpenter & Kennedy's coefficients, as the oracle's
LSERK_A[0] states exactly), so a step overwrites the residual register without reading it:
every stage kernel must give the same state whether res holds zeros or NaN on entry."""
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


def test_first_coefficient_is_zero():
    assert dg.LSERK_A[0] == 0


@pytest.mark.parametrize("path", ["bb_f64", "bb_f32", "bb_warp_f32", "nodal_f32", "nodal_tc"])
def test_step_ignores_residual_on_entry(bb, path):
    N = 4
    VX, EToV = inputs.kuhn_cube_mesh(3, jitter=0.1)
    K = len(EToV)
    rho, kappa = inputs.materials_from_wavespeed(inputs.uniform_wavespeed(K))
    basis = {"nodal_f32": bb.BBDG_NODAL, "nodal_tc": bb.BBDG_NODAL_TC}.get(path, bb.BBDG_BB)
    prec = bb.BBDG_F64 if path == "bb_f64" else bb.BBDG_F32
    s = bb.Solver(VX, EToV, rho, kappa, N, basis=basis, precision=prec)
    if path == "bb_warp_f32":
        bb.bbdg_set_stage_form(s.ctx, bb.BBDG_FORM_WARP, 4)
    q0 = torch.tensor(inputs.abi_layout(inputs.random_state(K, N, S=2)), dtype=s.torch_dtype, device="cuda")
    dt = 0.25 / 3 / (N + 1) ** 2 / 3.0
    outs = []
    for fill in (0.0, float("nan")):
        q = q0.clone()
        res = torch.full_like(q, fill)
        bb.bbdg_step(s.ctx, q, res, torch.empty_like(q), 0.0, dt, 3)
        torch.cuda.synchronize()
        outs.append((q.cpu().numpy(), res.cpu().numpy()))
    s.close()
    assert np.isfinite(outs[1][0]).all() and np.isfinite(outs[1][1]).all()
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])
