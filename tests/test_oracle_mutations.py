"""Planted mistakes: each plausible slip in the oracle's right-hand side must make one of
its pins fail.  The mistakes are planted in the oracle, on the CPU (monkeypatch)."""
import numpy as np
import pytest

from oracle import dg
from paper_1512_06025_gb300 import inputs


def problem(N=3):
    VX, EToV = inputs.kuhn_cube_mesh(2, jitter=0.1)
    K = len(EToV)
    c = inputs.uniform_wavespeed(K)
    rho = np.random.default_rng(11).uniform(0.5, 2.0, K)
    return dg.make_problem(VX, EToV, N, rho, rho * c * c)


def energy_pin_holds(P):
    q = inputs.random_state(P.K, P.N)[0]
    a, b = dg.energy_rate(P, q), dg.energy_dissipation(P, q)
    return abs(a - b) <= 1e-12 * abs(b)


def polynomial_pin_holds(P):
    """p = 0, u = global linear field: rhs_p = -kappa div u, rhs_u = 0."""
    q = np.zeros((P.K, 4, P.Np))
    q[:, 1] = dg.interpolate(P, lambda x, y, z: 1 + 2 * x - y)
    q[:, 2] = dg.interpolate(P, lambda x, y, z: 3 * y + z)
    q[:, 3] = dg.interpolate(P, lambda x, y, z: x - 0.5 * z)
    r = dg.rhs(P, q)
    ok_p = np.allclose(r[:, 0], -P.kappa[:, None] * 4.5, atol=1e-10 * P.kappa.max())
    return ok_p and np.abs(r[:, 1:]).max() < 1e-10


def pins_hold(P):
    return energy_pin_holds(P) and polynomial_pin_holds(P)


def test_unmutated_pins_hold():
    assert pins_hold(problem())


MUTATIONS = {
    "lift of the wrong face": lambda P: setattr(P, "lift", P.lift[[1, 0, 2, 3]]),
    "lift scaled by 2": lambda P: setattr(P, "lift", 2 * P.lift),
    "D^s replaced by D^r": lambda P: setattr(P, "Ds", P.Dr),
    "transposed G": lambda P: setattr(P.mesh, "G", np.transpose(P.mesh.G, (0, 2, 1)).copy()),
    "normal flipped on face 2": lambda P: P.mesh.normal.__setitem__((slice(None), 2), -P.mesh.normal[:, 2]),
    "J^f / J^k dropped": lambda P: setattr(P.mesh, "Jf", P.mesh.Jf / P.mesh.J[:, None] * 0.5),
    "neighbour nodes unpermuted": lambda P: setattr(P, "nbr_nodes", np.sort(P.nbr_nodes, axis=2)),
    "tau_u = tau_p": lambda P: setattr(P, "tau_u", P.tau_p.copy()),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(name):
    P = problem()
    MUTATIONS[name](P)
    assert not pins_hold(P), name


def test_flux_sign_mistake_is_caught(monkeypatch):
    P = problem()
    orig = dg.fluxes

    def bad(P, q, m, central=False, ks=None):
        Fp, Fu = orig(P, q, m, central, ks)
        return Fp, -Fu
    monkeypatch.setattr(dg, "fluxes", bad)
    assert not pins_hold(P)


def test_mirror_condition_mistake_is_caught(monkeypatch):
    """p^+ = +p^- instead of -p^- on the boundary breaks the energy pin."""
    P = problem()
    orig = dg.traces

    def bad(P, q, m, ks=None):
        ks = np.arange(P.K) if ks is None else np.asarray(ks)
        qm, qp = orig(P, q, m, ks)
        bs = P.mesh.nbr[ks, m] < 0
        qp[bs, 0] = qm[bs, 0]
        return qm, qp
    monkeypatch.setattr(dg, "traces", bad)
    assert not pins_hold(P)
