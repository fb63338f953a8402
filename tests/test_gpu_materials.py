"""GPU parity of bbdg_set_materials with device arrays and one medium per shot: every stage
form of the BB basis against the oracle shot by shot (each shot its own heterogeneous
kappa, rho), LSERK4 steps, the nodal bases against the same kernels run one medium at a
time, records formed on the device equal to the set-up ones, and the argument checks."""
import ctypes

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


def media(K, S, seed=40):
    """S seeded heterogeneous media: c ~ U[1, 3], rho ~ U[0.5, 2], kappa = rho c^2."""
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.5, 2.0, (S, K))
    c = rng.uniform(1.0, 3.0, (S, K))
    return rho * c * c, rho


def mesh(n=3):
    return inputs.kuhn_cube_mesh(n, jitter=0.1)


FORMS = [("group", 3, "f64"), ("group", 7, "f32"), ("warp", 3, "f64"), ("warp", 6, "f32"),
         ("pipe", 4, "f64"), ("pipe", 7, "f32"), ("thread", 2, "f64"), ("thread", 1, "f32")]


@pytest.mark.parametrize("form,N,prec", FORMS)
def test_per_shot_media_rhs_matches_oracle(bb, form, N, prec):
    """S = 3 shots, each with its own medium, through one bbdg_rhs call: shot s equals the
    oracle's right-hand side of medium s (FP64: 1e-12 in the 2-norm; FP32: 1e-5 element by
    element).  162 jittered tets: several element groups and a ragged tail."""
    VX, EToV = mesh()
    K, S = len(EToV), 3
    kap, rho = media(K, S)
    q0 = inputs.random_state(K, N, S=S)
    if prec == "f32":
        q0 = q0.astype(np.float32).astype(np.float64)
    s = bb.Solver(VX, EToV, np.ones(K), np.ones(K), N, precision=bb.BBDG_F64 if prec == "f64" else bb.BBDG_F32)
    bb.bbdg_set_stage_form(s.ctx, {"group": bb.BBDG_FORM_GROUP, "warp": bb.BBDG_FORM_WARP,
                                   "pipe": bb.BBDG_FORM_PIPE, "thread": bb.BBDG_FORM_THREAD}[form],
                           4 if form == "warp" else 0)
    s.set_materials(torch.tensor(kap, device="cuda"), torch.tensor(rho, device="cuda"))
    q = torch.tensor(inputs.abi_layout(q0), device="cuda", dtype=s.torch_dtype)
    r = torch.empty_like(q)
    bb.bbdg_rhs(s.ctx, q, r)
    got = inputs.oracle_layout(r.cpu().numpy()).astype(np.float64)
    bb.bbdg_device_status(s.ctx)
    s.close()
    for sh in range(S):
        want = dg.rhs(dg.make_problem(VX, EToV, N, rho[sh], kap[sh]), q0[sh])
        if prec == "f64":
            assert rel(got[sh], want) < 1e-12, (sh, rel(got[sh], want))
        else:
            assert elem_rel(got[sh][None], want[None]) < 1e-5, (sh, elem_rel(got[sh][None], want[None]))


def test_per_shot_media_steps_match_oracle(bb):
    """FP64, N = 3, S = 2 media, 4 LSERK4 steps from one random state per shot: each shot's
    trajectory equals the oracle's with its own medium to 1e-12."""
    VX, EToV = mesh()
    K, S, N = len(EToV), 2, 3
    kap, rho = media(K, S, seed=41)
    q0 = inputs.random_state(K, N, S=S, seed=7)
    dt = 2e-3
    s = bb.Solver(VX, EToV, rho[0], kap[0], N)
    s.set_materials(kap, rho)
    q = torch.tensor(inputs.abi_layout(q0), device="cuda")
    res = torch.zeros_like(q)
    bb.bbdg_step(s.ctx, q, res, torch.empty_like(q), 0.0, dt, 4)
    got = inputs.oracle_layout(q.cpu().numpy())
    s.close()
    for sh in range(S):
        P = dg.make_problem(VX, EToV, N, rho[sh], kap[sh])
        qo, ro = q0[sh].copy(), np.zeros_like(q0[sh])
        for i in range(4):
            qo, ro = dg.lserk4_step(lambda x, tt: dg.rhs(P, x), qo, ro, i * dt, dt)
        assert rel(got[sh], qo) < 1e-12, (sh, rel(got[sh], qo))


@pytest.mark.parametrize("basis", ["nodal", "nodal_tc"])
def test_per_shot_media_nodal_bases(bb, basis):
    """The nodal bases (FP32): shot s of an S = 2 call with per-shot media is bit-identical to
    an S = 1 call on shot s's state with medium s alone (the kernels read medium s for shot
    s and nothing else changes)."""
    VX, EToV = mesh()
    K, S, N = len(EToV), 2, 4
    kap, rho = media(K, S, seed=42)
    q0 = inputs.random_state(K, N, S=S, seed=8).astype(np.float32)
    s = bb.Solver(VX, EToV, np.ones(K), np.ones(K), N, precision=bb.BBDG_F32,
                  basis=bb.BBDG_NODAL if basis == "nodal" else bb.BBDG_NODAL_TC)
    q = torch.tensor(inputs.abi_layout(q0), device="cuda")
    s.set_materials(kap, rho)
    r = torch.empty_like(q)
    bb.bbdg_rhs(s.ctx, q, r)
    for sh in range(S):
        s.set_materials(kap[sh], rho[sh])
        r1 = torch.empty_like(q[sh:sh + 1])
        bb.bbdg_rhs(s.ctx, q[sh:sh + 1].clone(), r1)
        torch.cuda.synchronize()
        assert torch.equal(r[sh:sh + 1], r1), sh
    s.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_device_records_equal_setup_records(bb, prec):
    """Materials given at set-up (host arrays) and the same materials given later as device
    arrays give bit-identical right-hand sides (the records are formed by one routine)."""
    VX, EToV = mesh()
    K, N = len(EToV), 5
    kap, rho = media(K, 1, seed=43)
    q0 = inputs.random_state(K, N, seed=9)
    p = bb.BBDG_F64 if prec == "f64" else bb.BBDG_F32
    a = bb.Solver(VX, EToV, rho[0], kap[0], N, precision=p)
    b = bb.Solver(VX, EToV, np.ones(K), np.ones(K), N, precision=p)
    b.set_materials(torch.tensor(kap[0], device="cuda"), torch.tensor(rho[0], device="cuda"))
    q = torch.tensor(inputs.abi_layout(q0), device="cuda", dtype=a.torch_dtype)
    ra, rb = torch.empty_like(q), torch.empty_like(q)
    bb.bbdg_rhs(a.ctx, q, ra)
    bb.bbdg_rhs(b.ctx, q, rb)
    torch.cuda.synchronize()
    assert torch.equal(ra, rb)
    a.close()
    b.close()


def test_per_shot_media_graph_and_back_to_one_medium(bb):
    """bbdg_step_graph with per-shot media equals stream-ordered steps; returning to one
    medium gives the single-medium result again; the adjoint refuses per-shot media and
    works again after one medium is set."""
    VX, EToV = mesh(2)
    K, S, N = len(EToV), 2, 3
    kap, rho = media(K, S, seed=44)
    q0 = torch.tensor(inputs.abi_layout(inputs.random_state(K, N, S=S, seed=10)), device="cuda")
    s = bb.Solver(VX, EToV, rho[0], kap[0], N)
    ref = q0.clone()
    bb.bbdg_step(s.ctx, ref, torch.zeros_like(q0), torch.empty_like(q0), 0.0, 1e-3, 3)
    s.set_materials(kap, rho)
    q, res = q0.clone(), torch.zeros_like(q0)
    bb.bbdg_step_graph(s.ctx, q, res, torch.empty_like(q0), 0.0, 1e-3, 3)
    q2 = q0.clone()
    bb.bbdg_step(s.ctx, q2, torch.zeros_like(q0), torch.empty_like(q0), 0.0, 1e-3, 3)
    torch.cuda.synchronize()
    assert torch.equal(q, q2)
    assert not torch.equal(q[1], ref[1])          # shot 1 really ran in medium 1
    with pytest.raises(bb.BBDGError) as e:
        bb.bbdg_adjoint_rhs(s.ctx, q0[:1].clone(), torch.empty_like(q0[:1]), S=1)
    assert e.value.code == -2
    s.set_materials(kap[0], rho[0])
    q3 = q0.clone()
    bb.bbdg_step(s.ctx, q3, torch.zeros_like(q0), torch.empty_like(q0), 0.0, 1e-3, 3)
    torch.cuda.synchronize()
    assert torch.equal(q3, ref)
    bb.bbdg_adjoint_rhs(s.ctx, q0[:1].clone(), torch.empty_like(q0[:1]), S=1)
    s.close()


def test_set_materials_argument_checks(bb):
    """EINVAL, and nothing changes, for: a shot count other than the media's, a non-positive
    or non-finite entry, a host pointer, and S_or_1 < 1."""
    VX, EToV = mesh(2)
    K, N = len(EToV), 2
    kap, rho = media(K, 2, seed=45)
    s = bb.Solver(VX, EToV, rho[0], kap[0], N)
    q0 = torch.tensor(inputs.abi_layout(inputs.random_state(K, N, S=3, seed=11)), device="cuda")
    r0 = torch.empty_like(q0)
    bb.bbdg_rhs(s.ctx, q0, r0)
    bad = kap.copy()
    bad[1, 5] = -1.0
    with pytest.raises(bb.BBDGError) as e:
        s.set_materials(bad, rho)
    assert e.value.code == -1
    bad[1, 5] = np.nan
    with pytest.raises(bb.BBDGError):
        s.set_materials(bad, rho)
    host = np.ascontiguousarray(kap[0])
    hp = ctypes.c_void_p(host.ctypes.data)
    assert bb.load().bbdg_set_materials(s.ctx, hp, hp, 1) == -1
    kd = torch.tensor(kap[0], device="cuda")
    assert bb.load().bbdg_set_materials(s.ctx, bb._dev(kd), bb._dev(kd), 0) == -1
    r1 = torch.empty_like(q0)
    bb.bbdg_rhs(s.ctx, q0, r1)                     # the medium set up first is still in place
    torch.cuda.synchronize()
    assert torch.equal(r0, r1)
    s.set_materials(kap, rho)                      # two media ...
    with pytest.raises(bb.BBDGError) as e:
        bb.bbdg_rhs(s.ctx, q0, r1)                 # ... and three shots
    assert e.value.code == -1
    bb.bbdg_rhs(s.ctx, q0[:2].clone(), r1[:2])
    s.close()


def test_per_shot_media_set_before_operators(bb):
    """Materials set per shot on a context without operators are kept and used once the
    operators are built (records laid out per medium at set-up): FP64, N = 2, 2 shots."""
    VX, EToV = mesh()
    K, S, N = len(EToV), 2, 2
    kap, rho = media(K, S, seed=46)
    ctx = bb.bbdg_setup_mesh(VX, EToV, np.ones(K), np.ones(K))
    try:
        bb.bbdg_set_materials(ctx, kap, rho)
        bb.bbdg_setup_operators(ctx, N, bb.BBDG_BB, bb.BBDG_F64)
        q0 = inputs.random_state(K, N, S=S, seed=14)
        q = torch.tensor(inputs.abi_layout(q0), device="cuda")
        r = torch.empty_like(q)
        bb.bbdg_rhs(ctx, q, r)
        got = inputs.oracle_layout(r.cpu().numpy())
    finally:
        bb.bbdg_destroy(ctx)
    for sh in range(S):
        want = dg.rhs(dg.make_problem(VX, EToV, N, rho[sh], kap[sh]), q0[sh])
        assert rel(got[sh], want) < 1e-12, (sh, rel(got[sh], want))
