"""Misfit of receiver traces and its derivative with respect to the per-element bulk
modulus, for checking the discrete adjoint.

TEST INFRASTRUCTURE ONLY (part of the CPU oracle; see ``oracle/__init__``).

The paper is forward-only; the misfit is the workload's definition:
    J(kappa) = 1/2 sum_n sum_r (p_r(q^n) - d_r^n)^2,
q^n the fully discrete LSERK4 solution after step n (sources, receivers: ``oracle.dg``).
Its exact derivative is taken by complex-step differentiation of the same fully discrete
scheme: dJ/dkappa_k = Im J(kappa + i h e_k) / h, exact to roundoff for analytic J (no
subtractive cancellation), so it pins the discrete adjoint independently of any adjoint
code.
"""
from __future__ import annotations

import numpy as np

from . import dg


def traces(P: dg.Problem, src, rec, dt, nsteps, kappa=None):
    if kappa is not None:
        P.set_materials(P.rho, kappa)
    q0 = np.zeros((P.K, 4, P.Np))
    _, _, tr = dg.run(P, q0, 0.0, dt, nsteps, src=src, rec=rec)
    return tr


def misfit(P, src, rec, dt, nsteps, data, kappa=None):
    tr = traces(P, src, rec, dt, nsteps, kappa)
    return 0.5 * np.sum((tr - data) ** 2)


def gradient_complex_step(P, src, rec, dt, nsteps, data, kappa, h=1e-30, elements=None):
    """dJ/dkappa_k for k in elements (default: all) by complex steps of size h."""
    kappa = np.asarray(kappa, dtype=np.float64)
    elements = range(P.K) if elements is None else elements
    g = {}
    for k in elements:
        kc = kappa.astype(np.complex128)
        kc[k] += 1j * h
        g[k] = float(np.imag(misfit(P, src, rec, dt, nsteps, data, kc)) / h)
    P.set_materials(P.rho, kappa)
    return g
