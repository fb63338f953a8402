"""Semi-discrete Bernstein-Bezier DG right-hand side, energy, LSERK4, sources, receivers.

TEST INFRASTRUCTURE ONLY (part of the CPU oracle; see ``oracle/__init__``).

The acoustic system (Section 2)
    (1/kappa) p_t + div u = f,      rho u_t + grad p = 0,
with upwind fluxes, on each element in strong form (eq. (discrete_var), Section 3):
    p_t   = kappa [ -div u + sum_f (J^f/J^k) L^f F_p ]
    u_i,t = (1/rho) [ -d_i p + sum_f (J^f/J^k) n_i L^f F_u ]
    F_p = 1/2 (tau_p [p] - n.[u]),   F_u = 1/2 (tau_u [u].n - [p]),
    [a] = a^+ - a^-,  tau_p = 1/{rho c},  tau_u = {rho c},  {a} = (a^+ + a^-)/2,
and the mirror conditions p^+ = -p^-, u^+ = u^- on the domain boundary (Section 2).

Readings of the printed eq. (discrete_var): the second "G_{i1} D^r" is G_{i1} D^s, "U_j"
is U_i, "i = 0..d" is i = 1..3, and the volume terms carry the minus signs of the
Section 2 weak form.

Layout: a state is q[K, 4, N_p] with fields (p, u, v, w) and BB coefficients in the node
order of ``oracle.operators``.  Everything is float64.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from fractions import Fraction

import numpy as np

from . import mesh as meshmod
from . import operators as ops


@dataclass
class Problem:
    """Mesh + order + materials, with the geometry and operators precomputed."""
    mesh: meshmod.Mesh
    N: int
    rho: np.ndarray
    kappa: np.ndarray
    Dr: np.ndarray = field(init=False)
    Ds: np.ndarray = field(init=False)
    Dt: np.ndarray = field(init=False)
    lift: np.ndarray = field(init=False)          # [4, Np, Nfp]
    fnodes: np.ndarray = field(init=False)        # [4, Nfp]
    nbr_nodes: np.ndarray = field(init=False)     # [K, 4, Nfp]
    tau_p: np.ndarray = field(init=False)         # [K, 4]
    tau_u: np.ndarray = field(init=False)         # [K, 4]
    bc: str = "mirror"    # boundary faces: "mirror" (Section 2) or "absorbing" (zero exterior state)

    def __post_init__(self):
        # kappa may be complex (complex-step differentiation of the misfit)
        self.rho = np.asarray(self.rho, dtype=np.result_type(self.rho, np.float64))
        self.kappa = np.asarray(self.kappa, dtype=np.result_type(self.kappa, np.float64))
        self.Dr, self.Ds, self.Dt = ops.reference_derivatives(self.N)
        self.lift = ops.lift_faces(self.N)
        self.fnodes = np.stack([ops.face_nodes(self.N, m) for m in range(4)])
        self.nbr_nodes = meshmod.neighbour_node_map(self.mesh, self.N)
        self.set_materials(self.rho, self.kappa)

    def set_materials(self, rho, kappa):
        """tau_p = 1/{rho c}, tau_u = {rho c} per face (Section 2); on a boundary face the
        average is taken with the element itself."""
        self.rho = np.asarray(rho, dtype=np.result_type(rho, np.float64))
        self.kappa = np.asarray(kappa, dtype=np.result_type(kappa, np.float64))
        z = self.rho * np.sqrt(self.kappa / self.rho)       # rho c
        zP = np.where(self.mesh.nbr >= 0, z[np.maximum(self.mesh.nbr, 0)], z[:, None])
        avg = 0.5 * (z[:, None] + zP)
        self.tau_p = 1.0 / avg
        self.tau_u = avg

    @property
    def K(self):
        return self.mesh.EToV.shape[0]

    @property
    def Np(self):
        return ops.num_nodes(self.N)


def make_problem(VX, EToV, N, rho, kappa, bc="mirror") -> Problem:
    return Problem(meshmod.build_mesh(VX, EToV), N, rho, kappa, bc=bc)


def traces(P: Problem, q: np.ndarray, m: int, ks=None):
    """Own (minus) and neighbour (plus) face coefficients of face m for the elements ks
    (default all): arrays [len(ks), 4, Nfp].  Boundary faces: the mirror conditions of
    Section 2, p^+ = -p^-, u^+ = u^-, or (P.bc == "absorbing") a zero exterior state,
    p^+ = 0, u^+ = 0, which the upwind flux turns into an outflow condition."""
    ks = np.arange(P.K) if ks is None else np.asarray(ks)
    qm = q[ks][:, :, P.fnodes[m]]
    nb = P.mesh.nbr[ks, m]
    interior = nb >= 0
    qp = np.empty_like(qm)
    ii = np.nonzero(interior)[0]
    qp[ii] = q[nb[ii][:, None, None], np.arange(4)[None, :, None], P.nbr_nodes[ks[ii], m][:, None, :]]
    bs = np.nonzero(~interior)[0]
    if P.bc == "absorbing":
        qp[bs] = 0.0
    else:
        qp[bs, 0] = -qm[bs, 0]
        qp[bs, 1:] = qm[bs, 1:]
    return qm, qp


def fluxes(P: Problem, q: np.ndarray, m: int, central: bool = False, ks=None):
    """F_p and F_u of face m (Section 2, 3) for the elements ks, each [len(ks), Nfp]."""
    ks = np.arange(P.K) if ks is None else np.asarray(ks)
    qm, qp = traces(P, q, m, ks)
    n = P.mesh.normal[ks, m]                                 # [k, 3]
    jp = qp[:, 0] - qm[:, 0]
    jun = np.einsum("ki,kin->kn", n, qp[:, 1:] - qm[:, 1:])
    tp = 0.0 if central else P.tau_p[ks, m][:, None]
    tu = 0.0 if central else P.tau_u[ks, m][:, None]
    Fp = 0.5 * (tp * jp - jun)
    Fu = 0.5 * (tu * jun - jp)
    return Fp, Fu


def volume_terms(P: Problem, q: np.ndarray, ks=None):
    """(-div u, -grad p) with d_i = sum_a G[i, a] D^a (Section 3), for the elements ks."""
    ks = np.arange(P.K) if ks is None else np.asarray(ks)
    qk = q[ks]
    G = P.mesh.G[ks]
    D = (P.Dr, P.Ds, P.Dt)
    dp = np.stack([qk[:, 0] @ Da.T for Da in D], axis=1)     # [k, 3(a), Np]
    grad = np.einsum("kia,kan->kin", G, dp)                  # [k, 3(i), Np]
    div = np.zeros((len(ks), P.Np), dtype=np.result_type(q, np.float64))
    for i in range(3):
        du = np.stack([qk[:, 1 + i] @ Da.T for Da in D], axis=1)
        div += np.einsum("ka,kan->kn", G[:, i, :], du)
    return -div, -grad


def rhs(P: Problem, q: np.ndarray, central: bool = False, elements=None) -> np.ndarray:
    """A(kappa, rho) q: the semi-discrete right-hand side without sources.  With
    `elements`, only those elements' rows (in that order), from the same formulas."""
    q = np.asarray(q)
    ks = np.arange(P.K) if elements is None else np.asarray(elements)
    dt_ = np.result_type(q, P.kappa, np.float64)
    mdiv, mgrad = volume_terms(P, q, ks)
    liftp = np.zeros((len(ks), P.Np), dtype=dt_)
    liftu = np.zeros((len(ks), 3, P.Np), dtype=dt_)
    for m in range(4):
        Fp, Fu = fluxes(P, q, m, central, ks)
        sJ = (P.mesh.Jf[ks, m] / P.mesh.J[ks])[:, None]
        lp = (sJ * Fp) @ P.lift[m].T                         # [k, Np]
        lu = (sJ * Fu) @ P.lift[m].T
        liftp += lp
        liftu += P.mesh.normal[ks, m][:, :, None] * lu[:, None, :]
    out = np.empty((len(ks),) + q.shape[1:], dtype=dt_)
    out[:, 0] = P.kappa[ks][:, None] * (mdiv + liftp)
    out[:, 1:] = (1.0 / P.rho[ks])[:, None, None] * (mgrad + liftu)
    return out


# ----------------------------------------------------------------------------------------
# energy (Section 2)
# ----------------------------------------------------------------------------------------
def energy(P: Problem, q: np.ndarray) -> float:
    """E = 1/2 sum_k int_{D^k} (p^2/kappa + rho |u|^2) with the exact BB mass matrix."""
    M = ops.mass_tet(P.N)
    quad = np.einsum("kfn,nm,kfm->kf", q, M, q)             # [K, 4]
    return 0.5 * float(np.sum(P.mesh.J * (quad[:, 0] / P.kappa + P.rho * quad[:, 1:].sum(axis=1))))


def energy_rate(P: Problem, q: np.ndarray, central: bool = False) -> float:
    """q^T W A q with W = blockdiag(J M / kappa, rho J M (x3)) = dE/dt."""
    M = ops.mass_tet(P.N)
    r = rhs(P, q, central)
    quad = np.einsum("kfn,nm,kfm->kf", q, M, r)
    return float(np.sum(P.mesh.J * (quad[:, 0] / P.kappa + P.rho * quad[:, 1:].sum(axis=1))))


def energy_dissipation(P: Problem, q: np.ndarray, central: bool = False) -> float:
    """The right side of the energy statement of Section 2, evaluated exactly for the
    discrete solution:
      -1/2 sum_{interior faces} int (tau_p [p]^2 + tau_u [u_n]^2)
      -    sum_{boundary faces} int tau_p (p^-)^2                      (mirror conditions)
      -1/2 sum_{boundary faces} int (tau_p (p^-)^2 + tau_u (u_n^-)^2)  (zero exterior state)
    with int_f a b = J^f a^T M2 b on face coefficients (face area 2).  The boundary terms
    are -p u_n + p F_p + u_n F_u on the face, with the fluxes of the boundary's exterior
    state."""
    if central:
        return 0.0
    M2 = ops.mass_tri(P.N)
    # tau recomputed here from rho and kappa, independently of the right-hand side's copy
    z = np.sqrt(P.kappa * P.rho)                              # rho c
    total = 0.0
    for m in range(4):
        nb = P.mesh.nbr[:, m]
        zavg = 0.5 * (z + np.where(nb >= 0, z[np.maximum(nb, 0)], z))
        tau_p, tau_u = 1.0 / zavg, zavg
        qm, qp = traces(P, q, m)
        n = P.mesh.normal[:, m]
        jp = qp[:, 0] - qm[:, 0]
        jun = np.einsum("ki,kin->kn", n, qp[:, 1:] - qm[:, 1:])
        interior = P.mesh.nbr[:, m] >= 0
        Jf = P.mesh.Jf[:, m]
        ip = np.einsum("kn,nm,km->k", jp, M2, jp)
        iu = np.einsum("kn,nm,km->k", jun, M2, jun)
        pm2 = np.einsum("kn,nm,km->k", qm[:, 0], M2, qm[:, 0])
        # each interior face is visited from both sides: weight 1/2 * 1/2
        total += np.sum(np.where(interior, -0.25 * Jf * (tau_p * ip + tau_u * iu), 0.0))
        if P.bc == "absorbing":
            un = np.einsum("ki,kin->kn", n, qm[:, 1:])
            un2 = np.einsum("kn,nm,km->k", un, M2, un)
            total += np.sum(np.where(interior, 0.0, -0.5 * Jf * (tau_p * pm2 + tau_u * un2)))
        else:
            total += np.sum(np.where(interior, 0.0, -Jf * tau_p * pm2))
    return float(total)


# ----------------------------------------------------------------------------------------
# low-storage RK4 (Carpenter & Kennedy 1994, five stages; Section 4.2)
# ----------------------------------------------------------------------------------------
LSERK_A = (Fraction(0), Fraction(-567301805773, 1357537059087), Fraction(-2404267990393, 2016746695238),
           Fraction(-3550918686646, 2091501179385), Fraction(-1275806237668, 842570457699))
LSERK_B = (Fraction(1432997174477, 9575080441755), Fraction(5161836677717, 13612068292357),
           Fraction(1720146321549, 2090206949498), Fraction(3134564353537, 4481467310338),
           Fraction(2277821191437, 14882151754819))
def _stage_times():
    """c_s = sum_j a_sj of the equivalent Butcher tableau, computed exactly from LSERK_A,
    LSERK_B (stage s evaluates q_0 + sum_j a_sj dt f_j).  Reading: the stage times are
    taken as these row sums, which makes the scheme consistent for time-dependent
    sources."""
    s = 5
    R = [Fraction(0)] * s      # coefficients of f_0..f_4 in res
    Q = [Fraction(0)] * s      # coefficients of f_0..f_4 in q - q_0
    c = []
    for i in range(s):
        c.append(sum(Q))
        R = [LSERK_A[i] * v for v in R]
        R[i] += 1
        Q = [qv + LSERK_B[i] * rv for qv, rv in zip(Q, R)]
    return tuple(c)


LSERK_C = _stage_times()


def lserk4_step(rhs_fn, q, res, t, dt):
    """One step: for s = 1..5, res = a_s res + dt rhs(q, t + c_s dt); q = q + b_s res."""
    for s in range(5):
        res = float(LSERK_A[s]) * res + dt * rhs_fn(q, t + float(LSERK_C[s]) * dt)
        q = q + float(LSERK_B[s]) * res
    return q, res


# ----------------------------------------------------------------------------------------
# point sources and receivers (not in the paper; workload definitions)
# ----------------------------------------------------------------------------------------
def ricker(t, f0=10.0, t0=0.05):
    a = (np.pi * f0 * (np.asarray(t) - t0)) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


@dataclass
class Sources:
    elem: np.ndarray      # [ns] element of each source
    vec: np.ndarray       # [ns, Np] M^{-1} b / J^e, b_alpha = B_alpha(lambda(x_s))
    shot: np.ndarray      # [ns] shot index
    f0: float = 10.0
    t0: float = 0.05


def make_sources(P: Problem, xyz, shot=None, f0=10.0, t0=0.05) -> Sources:
    """f = delta(x - x_s) r(t): adds kappa_e r(t) M^{-1} b / J^e to p_t of the element e
    that contains x_s (lowest index), b_alpha = B_alpha(lambda(x_s))."""
    xyz = np.atleast_2d(np.asarray(xyz, dtype=np.float64))
    e = meshmod.locate_points(P.mesh, xyz)
    lam = meshmod.barycentric_of_points(P.mesh, xyz, e)
    b = ops.bernstein_eval(P.N, lam)
    vec = (b @ ops.mass_inverse(P.N).T) / P.mesh.J[e][:, None]
    shot = np.zeros(len(xyz), dtype=np.int64) if shot is None else np.asarray(shot, dtype=np.int64)
    return Sources(elem=e, vec=vec, shot=shot, f0=f0, t0=t0)


def add_sources(P: Problem, out: np.ndarray, src: Sources, t: float, shot: int = 0, elements=None):
    """out += the point-source terms of `shot` at time t; with `elements`, out holds only
    those elements' rows (in that order)."""
    r = float(ricker(t, src.f0, src.t0))
    row = None if elements is None else {int(k): i for i, k in enumerate(np.asarray(elements))}
    for e, v, s in zip(src.elem, src.vec, src.shot):
        if s == shot:
            i = e if row is None else row.get(int(e))
            if i is not None:
                out[i, 0] += P.kappa[e] * r * v
    return out


@dataclass
class Receivers:
    elem: np.ndarray      # [nr]
    basis: np.ndarray     # [nr, Np]  B_alpha(lambda(x_r))


def make_receivers(P: Problem, xyz) -> Receivers:
    xyz = np.atleast_2d(np.asarray(xyz, dtype=np.float64))
    e = meshmod.locate_points(P.mesh, xyz)
    lam = meshmod.barycentric_of_points(P.mesh, xyz, e)
    return Receivers(elem=e, basis=ops.bernstein_eval(P.N, lam))


def sample(rec: Receivers, q: np.ndarray) -> np.ndarray:
    """p(x_r) = sum_alpha c_alpha B_alpha(lambda(x_r))."""
    return np.einsum("rn,rn->r", q[rec.elem, 0], rec.basis)


def run(P: Problem, q0, t0, dt, nsteps, src: Sources | None = None, rec: Receivers | None = None,
        shot: int = 0, central: bool = False):
    """nsteps LSERK4 steps from q0; returns (q, res, traces [nsteps, nr] or None).
    Receivers are sampled after every full step."""
    def f(q, t):
        r = rhs(P, q, central)
        if src is not None:
            add_sources(P, r, src, t, shot)
        return r
    q = np.array(q0, dtype=np.result_type(q0, P.kappa, np.float64))
    res = np.zeros_like(q)
    tr = [] if rec is not None else None
    t = t0
    for _ in range(nsteps):
        q, res = lserk4_step(f, q, res, t, dt)
        t += dt
        if rec is not None:
            tr.append(sample(rec, q))
    return q, res, (np.asarray(tr) if tr is not None else None)


# ----------------------------------------------------------------------------------------
# interpolation and quadrature (initial conditions and error norms; Section 4.1)
# ----------------------------------------------------------------------------------------
def element_points(P: Problem, lam: np.ndarray) -> np.ndarray:
    """Physical points [K, n, 3] of barycentric points lam[n, 4] in every element."""
    v = P.mesh.VX[P.mesh.EToV]                                # [K, 4, 3]
    return np.einsum("ni,kid->knd", lam, v)


def interpolate(P: Problem, fn) -> np.ndarray:
    """BB coefficients [K, Np] of the degree-N interpolant of fn(x, y, z) at the
    equispaced lattice lambda = alpha / N (exact for polynomials of degree <= N)."""
    lam = np.asarray(ops.tet_multi_indices(P.N), dtype=np.float64) / P.N
    X = element_points(P, lam)
    vals = fn(X[..., 0], X[..., 1], X[..., 2])                # [K, Np]
    V = ops.bernstein_eval(P.N, lam)                          # [Np, Np]
    return np.linalg.solve(V, vals.T).T


def tet_quadrature(n: int):
    """Collapsed (conical product) Gauss-Jacobi rule on the unit tetrahedron
    {x, y, z >= 0, x + y + z <= 1}; exact for degree <= 2n - 1.  Returns (lam[nq, 4], w[nq])
    with weights summing to 1/6."""
    from scipy.special import roots_jacobi
    tu, wu = roots_jacobi(n, 2.0, 0.0)
    tv, wv = roots_jacobi(n, 1.0, 0.0)
    tw, ww = roots_jacobi(n, 0.0, 0.0)
    u, v, w = (1 + tu) / 2, (1 + tv) / 2, (1 + tw) / 2
    wu, wv, ww = wu / 8, wv / 4, ww / 2
    U, Vv, W = np.meshgrid(u, v, w, indexing="ij")
    WU, WV, WW = np.meshgrid(wu, wv, ww, indexing="ij")
    x = U
    y = (1 - U) * Vv
    z = (1 - U) * (1 - Vv) * W
    lam = np.stack([1 - x - y - z, x, y, z], axis=-1).reshape(-1, 4)
    return lam, (WU * WV * WW).reshape(-1)


def l2_error(P: Problem, q: np.ndarray, exact, nquad: int | None = None) -> float:
    """sqrt(sum_k int_{D^k} sum_fields (q_h - exact)^2); exact(x, y, z) -> [..., 4]."""
    nquad = nquad or P.N + 3
    lam, w = tet_quadrature(nquad)
    X = element_points(P, lam)                                # [K, nq, 3]
    B = ops.bernstein_eval(P.N, lam)                          # [nq, Np]
    qh = np.einsum("qn,kfn->kqf", B, q)
    ex = exact(X[..., 0], X[..., 1], X[..., 2])
    vol = (4.0 / 3.0) * P.mesh.J                              # volume of D^k
    # int_{D^k} f = 6 vol(D^k) int_{unit tet} f(lambda)
    err2 = 6.0 * vol * np.einsum("q,kq->k", w, ((qh - ex) ** 2).sum(axis=-1))
    return float(np.sqrt(err2.sum()))


def standing_mode(t: float):
    """The cube solution of Section 4.1 with rho = kappa = 1 on [-1/2, 1/2]^3:
    p = cos(pi x) cos(pi y) cos(pi z) cos(sqrt(3) pi t); the velocity (not printed in the
    paper) follows from u_t = -grad p, u(0) = 0:
    u = sin(pi x) cos(pi y) cos(pi z) sin(sqrt(3) pi t) / sqrt(3), and cyclically."""
    w = np.sqrt(3.0) * np.pi
    def f(x, y, z):
        cx, cy, cz = np.cos(np.pi * x), np.cos(np.pi * y), np.cos(np.pi * z)
        sx, sy, sz = np.sin(np.pi * x), np.sin(np.pi * y), np.sin(np.pi * z)
        st = np.sin(w * t) / np.sqrt(3.0)
        return np.stack([cx * cy * cz * np.cos(w * t), sx * cy * cz * st, cx * sy * cz * st, cx * cy * sz * st], axis=-1)
    return f


def interpolate_state(P: Problem, fn4) -> np.ndarray:
    """[K, 4, Np] BB interpolant of a 4-field function fn4(x, y, z) -> [..., 4]."""
    return np.stack([interpolate(P, lambda x, y, z, i=i: fn4(x, y, z)[..., i]) for i in range(4)], axis=1)
