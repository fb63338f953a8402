"""bbdg_step_noalloc: the allocation-free step (its ping-pong buffer is a static device
array of the library), for callers that cannot allocate device memory, e.g. plug-ins that
must not use their host's allocator.  Its results must equal bbdg_step's, including on a
second call that finds the array holding the first call's contents, for every basis.

This file is collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test."""
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


def rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("basis,prec", [("bb", "f64"), ("bb", "f32"), ("nodal", "f64"), ("nodal", "f32"),
                                        ("nodal_tc", "f32")])
def test_noalloc_matches_step_twice(bb, basis, prec):
    N = 3
    VX, EToV = inputs.kuhn_cube_mesh(3, jitter=0.1)
    K = len(EToV)
    c = inputs.uniform_wavespeed(K)
    rho, kappa = inputs.materials_from_wavespeed(c)
    p = bb.BBDG_F64 if prec == "f64" else bb.BBDG_F32
    dtype = torch.float64 if prec == "f64" else torch.float32
    tol = 1e-12 if prec == "f64" else 1e-5
    b = {"bb": bb.BBDG_BB, "nodal": bb.BBDG_NODAL, "nodal_tc": bb.BBDG_NODAL_TC}[basis]
    s = bb.Solver(VX, EToV, rho, kappa, N, basis=b, precision=p)
    dt = 0.25 * (1 / 3) / (N + 1) ** 2 / 3.0
    q0 = torch.tensor(inputs.abi_layout(inputs.random_state(K, N, S=2)), dtype=dtype, device="cuda")
    # reference: bbdg_step with a caller-provided scratch buffer
    q_ref, r_ref = q0.clone(), torch.zeros_like(q0)
    bb.bbdg_step(s.ctx, q_ref, r_ref, torch.empty_like(q0), 0.0, dt, 3)
    q_ref2, r_ref2 = q_ref.clone(), r_ref.clone()
    bb.bbdg_step(s.ctx, q_ref2, r_ref2, torch.empty_like(q0), 3 * dt, dt, 2)
    # two calls in a row of the allocation-free entry point (odd, then even step count)
    q, r = q0.clone(), torch.zeros_like(q0)
    bb.bbdg_step_noalloc(s.ctx, q, r, 0.0, dt, 3)
    torch.cuda.synchronize()
    assert rel(q, q_ref) <= tol and rel(r, r_ref) <= tol
    bb.bbdg_step_noalloc(s.ctx, q, r, 3 * dt, dt, 2)
    torch.cuda.synchronize()
    assert rel(q, q_ref2) <= tol and rel(r, r_ref2) <= tol
    s.close()


def test_noalloc_rejects_oversized_state(bb):
    """A state larger than the static array is refused with BBDG_EINVAL and a message."""
    N = 10
    VX, EToV = inputs.kuhn_cube_mesh(4)
    K = len(EToV)
    s = bb.Solver(VX, EToV, np.ones(K), np.ones(K), N, precision=bb.BBDG_F64)
    per_shot = K * 4 * bb.bbdg_num_nodes(N) * 8
    S = bb.bbdg_step_noalloc_max_bytes() // per_shot + 1
    q = torch.zeros((S, K, bb.bbdg_num_nodes(N), 4), dtype=torch.float64, device="cuda")
    with pytest.raises(bb.BBDGError) as ei:
        bb.bbdg_step_noalloc(s.ctx, q, torch.zeros_like(q), 0.0, 1e-4, 1)
    assert ei.value.code == -1 and "exceeds the static step buffer" in str(ei.value)
    s.close()


def test_noalloc_argument_order(bb):
    """The checks run in bbdg_step's order: an empty batch returns at once, bad pointers are
    refused before a zero step count is accepted."""
    VX, EToV = inputs.kuhn_cube_mesh(1)
    K = len(EToV)
    s = bb.Solver(VX, EToV, np.ones(K), np.ones(K), 2)
    q = torch.zeros((1, K, bb.bbdg_num_nodes(2), 4), dtype=torch.float64, device="cuda")
    bb.bbdg_step_noalloc(s.ctx, q, q, 0.0, 1e-3, 0, S=0)          # empty batch
    bb.bbdg_step_noalloc(s.ctx, q, torch.zeros_like(q), 0.0, 1e-3, 0)
    rc = bb.load().bbdg_step_noalloc(s.ctx, None, None, 1, 0.0, 1e-3, 0, None)
    assert rc == -1                                                # BBDG_EINVAL
    s.close()
