"""Edge cases of the C ABI on the GPU: an empty batch (S = 0) and zero steps are no-ops for
every entry point that takes them; the shot count's upper limit is enforced before any
launch; a ragged last element group and a single all-boundary element are covered by
test_gpu_bb.py."""
import numpy as np
import pytest

from paper_1512_06025_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bb():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1512_06025_gb300 import bbdg
    return bbdg


@pytest.fixture(scope="module")
def solver(bb):
    VX, EToV = inputs.kuhn_cube_mesh(2)
    K = len(EToV)
    s = bb.Solver(VX, EToV, np.ones(K), np.ones(K), 3)
    yield s
    s.close()


def test_empty_batch_is_a_no_op(bb, solver):
    s = solver
    e = torch.empty((0, s.K, s.Np, 4), dtype=torch.float64, device="cuda")
    bb.bbdg_rhs(s.ctx, e, torch.empty_like(e))
    bb.bbdg_step(s.ctx, e, torch.empty_like(e), torch.empty_like(e), 0.0, 1e-3, 3)
    bb.bbdg_step_graph(s.ctx, e, torch.empty_like(e), torch.empty_like(e), 0.0, 1e-3, 3)
    bb.bbdg_rk_stage(s.ctx, e, torch.empty_like(e), torch.empty_like(e), 2, 0.0, 1e-3)
    bb.bbdg_step_noalloc(s.ctx, e, torch.empty_like(e), 0.0, 1e-3, 3)
    torch.cuda.synchronize()
    bb.bbdg_device_status(s.ctx)                 # raises if a kernel recorded an error


def test_zero_steps_leave_the_state(bb, solver):
    s = solver
    q0 = torch.tensor(inputs.abi_layout(inputs.random_state(s.K, 3, S=2)), device="cuda")
    for f in (bb.bbdg_step, bb.bbdg_step_graph):
        q, res = q0.clone(), torch.full_like(q0, 7.0)
        f(s.ctx, q, res, torch.empty_like(q0), 0.0, 1e-3, 0)
        torch.cuda.synchronize()
        assert torch.equal(q, q0) and bool((res == 7.0).all())
    q = q0.clone()
    bb.bbdg_step_noalloc(s.ctx, q, torch.zeros_like(q0), 0.0, 1e-3, 0)
    torch.cuda.synchronize()
    assert torch.equal(q, q0)


def test_shot_limit_and_negative_steps(bb, solver):
    s = solver
    q = torch.zeros((1, s.K, s.Np, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(bb.BBDGError):
        bb.bbdg_rhs(s.ctx, q, torch.empty_like(q), S=65536)
    with pytest.raises(bb.BBDGError):
        bb.bbdg_step(s.ctx, q, torch.zeros_like(q), torch.empty_like(q), 0.0, 1e-3, -1)
