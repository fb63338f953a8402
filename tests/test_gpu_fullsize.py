"""Parity at the workloads' full sizes, in the launch configuration the benchmark uses
(autotuned elements per group and shots per tile), against the CPU oracle on outputs it
computes element by element (``dg.rhs(..., elements=...)``), or through identities that
hold at any size:

  C2  N = 7, 16^3 x 6 = 24 576 tets, unit medium, FP32 (the headline) and FP64: every
      element of the right-hand side and of one RK stage (residual and state);
  C3  24^3 x 6 = 82 944 jittered tets, c ~ U[1, 3], N = 1..10, FP32 and FP64: sampled
      elements (boundary and interior) of one RK stage;
  C4  32^3 x 6 = 196 608 tets, S = 64 shots, N = 5, FP32, layered c, one Ricker source per
      shot: sampled elements (the source elements among them) of two shots for one RK
      stage, and the CUDA-graph replay of two steps equal to stream-ordered steps;
  C5  N = 5, 16^3 x 6, c ~ U[1, 3], FP64, 8 sources, 256 receivers: the dot-product
      identity <A v, w> = <v, A^T w> at full size, and receiver traces of 3 steps against
      the oracle.

Tolerances: FP64 1e-12 relative (2-norm over the compared outputs); FP32 1e-5 relative,
the per-step FP32 bound the workloads set, against the oracle run on the FP32-rounded input.
"""
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


def sample_elements(P, count, seed, extra=()):
    """Boundary and interior elements (seeded), plus `extra`, sorted and unique."""
    rng = np.random.default_rng(seed)
    bnd = np.nonzero((P.mesh.nbr < 0).any(axis=1))[0]
    pick = np.concatenate([rng.choice(bnd, size=min(count // 4, len(bnd)), replace=False),
                           rng.choice(P.K, size=count, replace=False), np.asarray(extra, dtype=np.int64)])
    return np.unique(pick)


def tuned(bb, s, q, res, S=None):
    """The benchmark's launch shape: the autotuner over copies of the state."""
    from paper_1512_06025_gb300 import autotune
    autotune.tune(s, q.clone(), res.clone(), torch.empty_like(q), S=S, basis=bb.BBDG_BB, use_cache=False, reps=2)


def stage_reference(P, q, res, stage, t, dt, ks, src=None, shot=0):
    """Oracle residual and state of elements ks after RK stage `stage` of the step that
    starts at t (stage time t + c_s dt)."""
    ts = t + float(dg.LSERK_C[stage]) * dt
    r = dg.rhs(P, q, elements=ks)
    if src is not None:
        dg.add_sources(P, r, src, ts, shot, elements=ks)
    res_new = float(dg.LSERK_A[stage]) * res[ks] + dt * r
    return res_new, q[ks] + float(dg.LSERK_B[stage]) * res_new


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_c2_full_rhs_and_stage(bb, prec):
    N, n = 7, 16
    VX, EToV = inputs.kuhn_cube_mesh(n)
    K = len(EToV)
    rho, kappa = np.ones(K), np.ones(K)
    P = dg.make_problem(VX, EToV, N, rho, kappa)
    p = bb.BBDG_F32 if prec == "f32" else bb.BBDG_F64
    tdt = torch.float32 if prec == "f32" else torch.float64
    q0 = inputs.random_state(K, N)[0]
    r0 = inputs.random_state(K, N, seed=7)[0]
    if prec == "f32":
        q0, r0 = q0.astype(np.float32).astype(np.float64), r0.astype(np.float32).astype(np.float64)
    tol = 1e-5 if prec == "f32" else 1e-12
    s = bb.Solver(VX, EToV, rho, kappa, N, precision=p)
    q = torch.tensor(inputs.abi_layout(q0[None]), dtype=tdt, device="cuda")
    res = torch.tensor(inputs.abi_layout(r0[None]), dtype=tdt, device="cuda")
    tuned(bb, s, q, res)
    r = torch.empty_like(q)
    bb.bbdg_rhs(s.ctx, q, r)
    ks = np.arange(K)
    got = inputs.oracle_layout(r.cpu().numpy())[0].astype(np.float64)
    want = dg.rhs(P, q0)
    assert rel(got, want) < tol, rel(got, want)
    assert elem_rel(got, want) < 10 * tol, elem_rel(got, want)
    stage, t, dt = 2, 0.1, 0.25 / n / (N + 1) ** 2
    out = torch.empty_like(q)
    bb.bbdg_rk_stage(s.ctx, q, out, res, stage, t, dt)
    want_res, want_q = stage_reference(P, q0, r0, stage, t, dt, ks)
    got_res = inputs.oracle_layout(res.cpu().numpy())[0].astype(np.float64)
    got_q = inputs.oracle_layout(out.cpu().numpy())[0].astype(np.float64)
    s.close()
    assert rel(got_res, want_res) < tol, rel(got_res, want_res)
    assert rel(got_q, want_q) < tol, rel(got_q, want_q)
    assert elem_rel(got_res, want_res) < 10 * tol, elem_rel(got_res, want_res)
    assert elem_rel(got_q, want_q) < 10 * tol, elem_rel(got_q, want_q)


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("N", range(1, 11))
def test_c3_sampled_stage(bb, N, prec):
    c3_sampled_stage(bb, N, prec, warp_form=False)


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("N", [4, 7, 10])
def test_c3_sampled_stage_warp_form(bb, N, prec):
    """The element-per-warp kernel with its tuned warps per CTA (autotune.tune_warps)."""
    c3_sampled_stage(bb, N, prec, warp_form=True)


def test_c2_first_stage_ignores_residual(bb):
    """Stage 1 (a_1 = 0) of the C2 workload in FP32 with a NaN-filled residual register:
    every element against the oracle's stage from a zero residual."""
    N, n = 7, 16
    VX, EToV = inputs.kuhn_cube_mesh(n)
    K = len(EToV)
    rho, kappa = np.ones(K), np.ones(K)
    P = dg.make_problem(VX, EToV, N, rho, kappa)
    q0 = inputs.random_state(K, N)[0].astype(np.float32).astype(np.float64)
    s = bb.Solver(VX, EToV, rho, kappa, N, precision=bb.BBDG_F32)
    q = torch.tensor(inputs.abi_layout(q0[None]), dtype=torch.float32, device="cuda")
    tuned(bb, s, q, torch.zeros_like(q))
    res = torch.full_like(q, float("nan"))
    out = torch.empty_like(q)
    t, dt = 0.1, 0.25 / n / (N + 1) ** 2
    bb.bbdg_rk_stage(s.ctx, q, out, res, 0, t, dt)
    want_res, want_q = stage_reference(P, q0, np.zeros_like(q0), 0, t, dt, np.arange(K))
    got_res = inputs.oracle_layout(res.cpu().numpy())[0].astype(np.float64)
    got_q = inputs.oracle_layout(out.cpu().numpy())[0].astype(np.float64)
    s.close()
    assert rel(got_res, want_res) < 1e-5, rel(got_res, want_res)
    assert rel(got_q, want_q) < 1e-5, rel(got_q, want_q)
    assert elem_rel(got_res, want_res) < 1e-4, elem_rel(got_res, want_res)
    assert elem_rel(got_q, want_q) < 1e-4, elem_rel(got_q, want_q)


def c3_sampled_stage(bb, N, prec, warp_form):
    n = 24
    VX, EToV = inputs.kuhn_cube_mesh(n, jitter=0.1)
    K = len(EToV)
    c = inputs.uniform_wavespeed(K)
    rho, kappa = inputs.materials_from_wavespeed(c)
    P = dg.make_problem(VX, EToV, N, rho, kappa)
    p = bb.BBDG_F32 if prec == "f32" else bb.BBDG_F64
    tdt = torch.float32 if prec == "f32" else torch.float64
    q0 = inputs.random_state(K, N)[0]
    r0 = inputs.random_state(K, N, seed=7)[0]
    if prec == "f32":
        q0, r0 = q0.astype(np.float32).astype(np.float64), r0.astype(np.float32).astype(np.float64)
    s = bb.Solver(VX, EToV, rho, kappa, N, precision=p)
    q = torch.tensor(inputs.abi_layout(q0[None]), dtype=tdt, device="cuda")
    res = torch.tensor(inputs.abi_layout(r0[None]), dtype=tdt, device="cuda")
    if warp_form:
        from paper_1512_06025_gb300 import autotune
        autotune.tune_warps(s, q.clone(), res.clone(), torch.empty_like(q), reps=2)
    else:
        bb.bbdg_set_stage_form(s.ctx, bb.BBDG_FORM_GROUP, 0)
        tuned(bb, s, q, res)
    out = torch.empty_like(q)
    stage, t, dt = 4, 0.0, 0.25 / n / (N + 1) ** 2 / c.max()
    bb.bbdg_rk_stage(s.ctx, q, out, res, stage, t, dt)
    ks = sample_elements(P, 64, seed=N)
    want_res, want_q = stage_reference(P, q0, r0, stage, t, dt, ks)
    got_res = np.swapaxes(res[0, ks].cpu().numpy(), 1, 2).astype(np.float64)
    got_q = np.swapaxes(out[0, ks].cpu().numpy(), 1, 2).astype(np.float64)
    s.close()
    tol = 1e-5 if prec == "f32" else 1e-12
    assert rel(got_res, want_res) < tol, rel(got_res, want_res)
    assert rel(got_q, want_q) < tol, rel(got_q, want_q)
    assert elem_rel(got_res, want_res) < 10 * tol, elem_rel(got_res, want_res)
    assert elem_rel(got_q, want_q) < 10 * tol, elem_rel(got_q, want_q)


def test_c4_batched_shots(bb):
    N, n, S = 5, 32, 64
    VX, EToV = inputs.kuhn_cube_mesh(n)
    K = len(EToV)
    c = inputs.layered_wavespeed(VX, EToV)
    rho, kappa = inputs.materials_from_wavespeed(c)
    P = dg.make_problem(VX, EToV, N, rho, kappa)
    xs = inputs.random_points(S, -0.4, 0.4)
    shots = np.arange(S)
    src = dg.make_sources(P, xs, shot=shots)
    s = bb.Solver(VX, EToV, rho, kappa, N, precision=bb.BBDG_F32)
    bb.bbdg_set_sources(s.ctx, xs, shots, 10.0, 0.05)
    Np = s.Np
    q = torch.zeros((S, K, Np, 4), dtype=torch.float32, device="cuda")
    res = torch.zeros_like(q)
    checked = {0: 11, S - 1: 12}                     # shot -> seed of its random state
    host = {}
    for sh, seed in checked.items():
        q0 = inputs.random_state(K, N, seed=seed)[0].astype(np.float32).astype(np.float64)
        r0 = inputs.random_state(K, N, seed=seed + 100)[0].astype(np.float32).astype(np.float64)
        q[sh] = torch.tensor(inputs.abi_layout(q0), dtype=torch.float32, device="cuda")
        res[sh] = torch.tensor(inputs.abi_layout(r0), dtype=torch.float32, device="cuda")
        host[sh] = (q0, r0)
    tuned(bb, s, q, res, S=S)
    out = torch.empty_like(q)
    stage, t, dt = 1, 0.045, 0.25 / n / (N + 1) ** 2 / c.max()
    bb.bbdg_rk_stage(s.ctx, q, out, res, stage, t, dt)
    for sh, (q0, r0) in host.items():
        e_src = int(src.elem[sh])
        ks = sample_elements(P, 64, seed=sh, extra=[e_src, *P.mesh.nbr[e_src][P.mesh.nbr[e_src] >= 0]])
        want_res, want_q = stage_reference(P, q0, r0, stage, t, dt, ks, src=src, shot=sh)
        got_res = np.swapaxes(res[sh, ks].cpu().numpy(), 1, 2).astype(np.float64)
        got_q = np.swapaxes(out[sh, ks].cpu().numpy(), 1, 2).astype(np.float64)
        assert rel(got_res, want_res) < 1e-5, (sh, rel(got_res, want_res))
        assert rel(got_q, want_q) < 1e-5, (sh, rel(got_q, want_q))
        assert elem_rel(got_res, want_res) < 1e-4, (sh, elem_rel(got_res, want_res))
        assert elem_rel(got_q, want_q) < 1e-4, (sh, elem_rel(got_q, want_q))
    # the shots with a zero state and residual got exactly their source term (and nothing
    # leaked across shots): p at the source element only, u unchanged
    sh = 7
    e_src = int(src.elem[sh])
    ts = t + float(dg.LSERK_C[stage]) * dt
    want = dt * float(dg.LSERK_B[stage]) * kappa[e_src] * float(dg.ricker(ts)) * src.vec[sh]
    got = out[sh, e_src, :, 0].cpu().numpy().astype(np.float64)
    assert rel(got, want) < 1e-5
    others = out[sh].clone()
    others[e_src, :, 0] = 0
    assert float(others.abs().max()) == 0.0
    del out, others
    torch.cuda.empty_cache()
    # graph replay of two steps equals the stream-ordered steps, bit for bit
    q2, res2 = q.clone(), res.clone()
    scratch = torch.empty_like(q)
    bb.bbdg_step(s.ctx, q, res, scratch, 0.0, dt, 2)
    bb.bbdg_step_graph(s.ctx, q2, res2, scratch, 0.0, dt, 2)
    torch.cuda.synchronize()
    assert torch.equal(q, q2) and torch.equal(res, res2)
    assert bool(torch.isfinite(q).all())
    s.close()


def test_c5_adjoint_identity_and_traces(bb):
    N, n = 5, 16
    VX, EToV = inputs.kuhn_cube_mesh(n)
    K = len(EToV)
    c = inputs.uniform_wavespeed(K)
    rho, kappa = inputs.materials_from_wavespeed(c)
    s = bb.Solver(VX, EToV, rho, kappa, N, precision=bb.BBDG_F64)
    v = torch.tensor(inputs.abi_layout(inputs.random_state(K, N, seed=21)), device="cuda")
    w = torch.tensor(inputs.abi_layout(inputs.random_state(K, N, seed=22)), device="cuda")
    Av, ATw = torch.empty_like(v), torch.empty_like(w)
    bb.bbdg_rhs(s.ctx, v, Av)
    bb.bbdg_adjoint_rhs(s.ctx, w, ATw)
    lhs, rhs_ = float((Av * w).sum()), float((v * ATw).sum())
    scale = float(Av.abs().sum() * w.abs().max())
    assert abs(lhs - rhs_) <= 1e-13 * scale, (lhs, rhs_)
    # receiver traces of 3 steps from rest with 8 sources, against the oracle
    P = dg.make_problem(VX, EToV, N, rho, kappa)
    xs = inputs.random_points(8, (-0.4, -0.4, 0.0), (0.4, 0.4, 0.4))
    rec = inputs.receiver_plane(1.0 / n, 16)
    dt = 0.25 * (1.0 / n) / (N + 1) ** 2 / c.max()
    src, recs = dg.make_sources(P, xs), dg.make_receivers(P, rec)
    nsteps = 3
    _, _, want = dg.run(P, np.zeros((K, 4, P.Np)), 0.045, dt, nsteps, src, recs)
    bb.bbdg_set_sources(s.ctx, xs, np.zeros(8, dtype=np.int64), 10.0, 0.05)
    bb.bbdg_set_receivers(s.ctx, rec)
    q = torch.zeros((1, K, s.Np, 4), dtype=torch.float64, device="cuda")
    traces = torch.zeros((nsteps, 1, len(rec)), dtype=torch.float64, device="cuda")
    bb.bbdg_step(s.ctx, q, torch.zeros_like(q), torch.empty_like(q), 0.045, dt, nsteps, traces=traces)
    got = traces[:, 0, :].cpu().numpy()
    s.close()
    assert rel(got, want) < 1e-12, rel(got, want)
