"""bbdg_step_host (state and receiver traces in host memory, caller-owned device work
buffer): equal bit for bit to bbdg_step on the same state, with pinned and pageable host
memory, several batches in flight on several streams, and the argument checks."""
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


def solver(bb, prec, n=3, N=4):
    VX, EToV = inputs.kuhn_cube_mesh(n, jitter=0.1)
    K = len(EToV)
    c = inputs.uniform_wavespeed(K)
    s = bb.Solver(VX, EToV, np.ones(K), c * c, N, precision=prec)
    bb.bbdg_set_sources(s.ctx, inputs.random_points(2, (-0.3, -0.3, -0.3), (0.3, 0.3, 0.3)),
                        np.array([0, 1], dtype=np.int64), 10.0, 0.05)
    bb.bbdg_set_receivers(s.ctx, inputs.receiver_plane(1.0 / n, 4))
    return s, K


@pytest.mark.parametrize("prec,pinned", [("f64", True), ("f32", True), ("f32", False)])
def test_step_host_equals_step(bb, prec, pinned):
    """S = 2 shots with sources, 3 steps (odd: the final state comes back from the ping-pong
    buffer), receiver traces: q and traces equal bbdg_step's bit for bit."""
    s, K = solver(bb, bb.BBDG_F64 if prec == "f64" else bb.BBDG_F32)
    dt = 1e-3
    q0 = torch.tensor(inputs.abi_layout(inputs.random_state(K, s.N, S=2)), dtype=s.torch_dtype)
    qd = q0.cuda()
    tr = torch.zeros((3, 2, 16), dtype=s.torch_dtype, device="cuda")
    bb.bbdg_step(s.ctx, qd, torch.zeros_like(qd), torch.empty_like(qd), 0.02, dt, 3, traces=tr)
    hq = q0.clone().pin_memory() if pinned else q0.clone()
    ht = torch.zeros((3, 2, 16), dtype=s.torch_dtype)
    ht = ht.pin_memory() if pinned else ht
    work = torch.empty(3 * q0.numel() + ht.numel(), dtype=s.torch_dtype, device="cuda")
    bb.bbdg_step_host(s.ctx, hq, work, 0.02, dt, 3, traces_host=ht)
    torch.cuda.synchronize()
    assert torch.equal(hq, qd.cpu())
    assert torch.equal(ht, tr.cpu())
    s.close()


def test_step_host_batches_in_flight(bb):
    """Three independent batches on three streams, two steps each, issued back to back and
    interleaved: each equals its own bbdg_step result."""
    s, K = solver(bb, bb.BBDG_F32, n=4, N=5)
    dt = 5e-4
    lanes = []
    for j in range(3):
        q0 = torch.tensor(inputs.abi_layout(inputs.random_state(K, s.N, S=1, seed=20 + j)), dtype=torch.float32)
        qd = q0.cuda()
        bb.bbdg_step(s.ctx, qd, torch.zeros_like(qd), torch.empty_like(qd), 0.0, dt, 2)
        lanes.append({"want": qd.cpu(), "hq": q0.pin_memory(),
                      "work": torch.empty((3,) + tuple(q0.shape), dtype=torch.float32, device="cuda"),
                      "st": torch.cuda.Stream()})
    torch.cuda.synchronize()
    for i in range(2):
        for L in lanes:
            bb.bbdg_step_host(s.ctx, L["hq"], L["work"], i * dt, dt, 1, stream=L["st"])
    torch.cuda.synchronize()
    for L in lanes:
        assert torch.equal(L["hq"], L["want"])
    s.close()


def test_step_host_argument_checks(bb):
    """A misaligned work pointer is rejected before anything is enqueued; S = 0 and
    nsteps = 0 leave the host state untouched."""
    s, K = solver(bb, bb.BBDG_F32)
    q0 = torch.tensor(inputs.abi_layout(inputs.random_state(K, s.N)), dtype=torch.float32)
    hq = q0.clone()
    work = torch.empty(3 * q0.numel() + 4, dtype=torch.float32, device="cuda")
    with pytest.raises(bb.BBDGError) as e:
        bb.bbdg_step_host(s.ctx, hq, work[1:], 0.0, 1e-3, 1)
    assert e.value.code == -1
    bb.bbdg_step_host(s.ctx, hq, work, 0.0, 1e-3, 0)
    bb.bbdg_step_host(s.ctx, hq, work, 0.0, 1e-3, 1, S=0)
    torch.cuda.synchronize()
    assert torch.equal(hq, q0)
    s.close()
