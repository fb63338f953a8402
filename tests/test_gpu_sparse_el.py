"""GPU parity of the sparse lift-reduction surface variant (BBDG_LIFT_SPARSE_EL: L0
row-parallel, then each node's row of E_L, Algorithm 3 and the non-optimal surface kernel
of Section 4.2) against the oracle, whose lift is the factorised E_L^f L0 of Section 3.1.2;
and its agreement with the optimal variant (Algorithm 1)."""
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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def make(n, N, jitter=0.1, seed=2):
    VX, EToV = inputs.kuhn_cube_mesh(n, jitter=jitter)
    K = len(EToV)
    c = inputs.uniform_wavespeed(K, seed=seed)
    rho = np.random.default_rng(seed + 10).uniform(0.5, 2.0, K)
    return VX, EToV, rho, rho * c * c


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("N", range(1, 7))
def test_sparse_el_rhs_matches_oracle(bb, N, prec):
    VX, EToV, rho, kappa = make(3, N)          # K = 162: several groups and a ragged tail
    K = len(EToV)
    P = dg.make_problem(VX, EToV, N, rho, kappa)
    q0 = inputs.random_state(K, N, S=2)
    p = bb.BBDG_F64 if prec == "f64" else bb.BBDG_F32
    tdt = torch.float64 if prec == "f64" else torch.float32
    if prec == "f32":
        q0 = q0.astype(np.float32).astype(np.float64)
    want = np.stack([dg.rhs(P, q0[s]) for s in range(2)])
    s = bb.Solver(VX, EToV, rho, kappa, N, precision=p, lift_variant=bb.BBDG_LIFT_SPARSE_EL)
    for E in (1, 5):
        bb.bbdg_set_launch_shape(s.ctx, E, 1)
        q = torch.tensor(inputs.abi_layout(q0), dtype=tdt, device="cuda")
        r = torch.empty_like(q)
        bb.bbdg_rhs(s.ctx, q, r)
        got = inputs.oracle_layout(r.cpu().numpy()).astype(np.float64)
        tol = 1e-12 if prec == "f64" else 1e-5
        assert rel(got, want) < tol, (E, rel(got, want))
    s.close()


def test_sparse_el_steps_with_sources_equal_optimal(bb):
    """Two shots with Ricker sources, 4 LSERK4 steps: the two lift variants agree to FP64
    rounding, and the sparse one matches the oracle."""
    N, n, S = 4, 3, 2
    VX, EToV, rho, kappa = make(n, N)
    K = len(EToV)
    xs = np.array([[0.1, -0.05, 0.2], [-0.2, 0.15, -0.1]])
    shots = np.array([0, 1])
    dt = 0.25 * (1.0 / n) / (N + 1) ** 2 / np.sqrt(kappa / rho).max()
    q0 = inputs.random_state(K, N, S=S)
    outs = []
    for lv in (bb.BBDG_LIFT_OPTIMAL, bb.BBDG_LIFT_SPARSE_EL):
        s = bb.Solver(VX, EToV, rho, kappa, N, lift_variant=lv)
        bb.bbdg_set_sources(s.ctx, xs, shots, 10.0, 0.05)
        q = torch.tensor(inputs.abi_layout(q0), device="cuda")
        bb.bbdg_step(s.ctx, q, torch.zeros_like(q), torch.empty_like(q), 0.04, dt, 4)
        outs.append(inputs.oracle_layout(q.cpu().numpy()))
        s.close()
    assert rel(outs[1], outs[0]) < 1e-13
    P = dg.make_problem(VX, EToV, N, rho, kappa)
    src = dg.make_sources(P, xs, shot=shots)
    for sh in range(S):
        want, _, _ = dg.run(P, q0[sh], 0.04, dt, 4, src=src, shot=sh)
        assert rel(outs[1][sh], want) < 1e-12


def test_sparse_el_limits(bb):
    VX, EToV, rho, kappa = make(1, 1, jitter=0.0)
    with pytest.raises(bb.BBDGError) as e:
        bb.Solver(VX, EToV, rho, kappa, 7, lift_variant=bb.BBDG_LIFT_SPARSE_EL)
    assert e.value.code == -2
    # the nodal bases ignore the lift variant
    s = bb.Solver(VX, EToV, rho, kappa, 7, basis=bb.BBDG_NODAL, lift_variant=bb.BBDG_LIFT_SPARSE_EL)
    s.close()


def test_autotuner_chooses_a_lift_variant(bb):
    from paper_1512_06025_gb300 import autotune
    VX, EToV, rho, kappa = make(6, 3)
    K = len(EToV)
    s = bb.Solver(VX, EToV, rho, kappa, 3, precision=bb.BBDG_F32)
    q = torch.tensor(inputs.abi_layout(inputs.random_state(K, 3)), dtype=torch.float32, device="cuda")
    lv, times = autotune.tune_lift_variant(s, q.clone(), torch.zeros_like(q), torch.empty_like(q), reps=2)
    assert set(times) == {bb.BBDG_LIFT_OPTIMAL, bb.BBDG_LIFT_SPARSE_EL} and lv == min(times, key=times.get)
    assert s.lift_variant == lv
    r = torch.empty_like(q)
    bb.bbdg_rhs(s.ctx, q, r)
    assert bool(torch.isfinite(r).all())
    s.close()
