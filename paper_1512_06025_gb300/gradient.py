"""Gradient of a receiver misfit with respect to the per-element bulk modulus kappa, by the
discrete adjoint of the LSERK4 scheme.

    J(kappa) = 1/2 sum_n sum_r (p_r(q^n) - d_r^n)^2

(q^n after step n, receivers of the context).  Two storage plans:

* whole trajectory (default when it fits the memory budget): the forward pass runs one
  bbdg_rk_stage per stage into consecutive slots of a (5 nsteps + 1)-state buffer, so slot
  5 i + s is the input of stage s of step i, and the reverse pass needs no recomputation.
  A GPU with hundreds of GB of HBM holds the trajectories of the workloads this is meant
  for (N = 5, 24 576 elements, 400 FP64 steps: 88 GB);
* uniform checkpoints every `checkpoint_every` steps: the forward pass (bbdg_step) keeps
  the state at segment starts and runs the last segment stage by stage into a (5 C + 1)-state
  buffer; the reverse pass walks that segment backwards at once, then reruns each earlier
  segment from its checkpoint into the same buffer and walks it backwards.

Either way the reverse pass calls bbdg_adjoint_step for each step, last first, injecting
the receiver residual of that step.  The residual r = p - d and the misfit J (compensated
FP64 sum) come from bbdg_misfit.  All arithmetic runs in the library's kernels; this module
only orders the calls and owns the buffers (torch tensors).  The paper is
forward-only; this is the differentiation form layered on it.
"""
from __future__ import annotations

import numpy as np

from . import bbdg


class MisfitGradient:
    def __init__(self, solver, dt, nsteps, data, checkpoint_every=None, stream=None, memory_budget=None):
        """solver: a bbdg.Solver (BB basis, FP64) with sources and receivers set.
        data: device tensor [nsteps][nrec] (FP64) of observed traces.
        checkpoint_every: None = keep the whole trajectory when its 5 nsteps + 1 states fit
        in memory_budget bytes (default: half of the device memory free now), else
        checkpoints every 20 steps; an integer C forces checkpoints every C steps."""
        import torch
        if solver.precision != bbdg.BBDG_F64:
            raise ValueError("the adjoint runs in FP64")
        self.s = solver
        self.dt = float(dt)
        self.nsteps = int(nsteps)
        self.data = data.contiguous()
        self.nrec = data.shape[1]
        self.stream = stream
        K, Np = solver.K, solver.Np
        dev = data.device
        self.shape = (1, K, Np, 4)
        state_bytes = K * Np * 4 * 8
        if checkpoint_every is None:
            if memory_budget is None:
                free, _ = torch.cuda.mem_get_info(dev)
                memory_budget = free // 2
            self.keep_all = (5 * self.nsteps + 1) * state_bytes <= memory_budget
            self.C = self.nsteps if self.keep_all else 20
        else:
            self.C = int(checkpoint_every)
            self.keep_all = False
        self.q = torch.zeros(self.shape, dtype=torch.float64, device=dev)
        self.res = torch.zeros_like(self.q)
        self.scratch = torch.empty_like(self.q)
        self.traces = torch.zeros((self.nsteps, 1, self.nrec), dtype=torch.float64, device=dev)
        self.ckpt = {}
        self.kept = None
        self.resid = torch.empty((self.nsteps, self.nrec), dtype=torch.float64, device=dev)
        self.J = torch.zeros(1, dtype=torch.float64, device=dev)
        nslots = 5 * (self.nsteps if self.keep_all else min(self.C, self.nsteps)) + 1
        self.stages = torch.empty((nslots,) + self.shape, dtype=torch.float64, device=dev)

    def set_kappa(self, rho, kappa):
        """kappa, rho: [K] FP64, CUDA tensors (passed by device pointer) or host arrays."""
        bbdg.bbdg_set_materials(self.s.ctx, kappa, rho)

    def forward(self):
        """Forward solve from rest, keeping the trajectory or checkpoints; returns J (python
        float) and the residuals r^n = p^n - d^n (device tensor [nsteps][nrec])."""
        if self.keep_all:
            return self._forward_keep_all()
        self.q.zero_()
        self.res.zero_()
        self.ckpt = {}
        starts = list(range(0, self.nsteps, self.C))
        for n0 in starts:
            m = min(self.C, self.nsteps - n0)
            self.ckpt[n0] = (self.q.clone(), self.res.clone())
            if n0 == starts[-1]:
                # the last segment runs stage by stage into the stage buffer: the reverse
                # sweep starts with it and needs no recomputation of it
                self.stages[0].copy_(self.q)
                self._run_segment(n0, m, self.res, traces=True)
                self.q.copy_(self.stages[5 * m])
            else:
                bbdg.bbdg_step(self.s.ctx, self.q, self.res, self.scratch, n0 * self.dt, self.dt, m,
                               traces=self.traces[n0:n0 + m], stream=self.stream)
        self.kept = starts[-1]
        return self._misfit()

    def _misfit(self):
        """r^n = p^n - d^n and J = 1/2 sum r^2, both by the library (compensated FP64 sum);
        J is read back to the host."""
        bbdg.bbdg_misfit(self.s.ctx, self.traces, self.data, self.resid, self.J, stream=self.stream)
        return float(self.J.item()), self.resid

    def _run_segment(self, n0, m, res, traces):
        """Steps n0 .. n0 + m - 1 from the state in stages[0] (residual register res), one
        bbdg_rk_stage per stage into consecutive slots of the stage buffer; with traces, the
        receivers are sampled after every step."""
        st_ = self.stages
        for i in range(m):
            t = (n0 + i) * self.dt
            for k in range(5):
                j = 5 * i + k
                bbdg.bbdg_rk_stage(self.s.ctx, st_[j], st_[j + 1], res, k, t, self.dt, stream=self.stream)
            if traces:
                bbdg.bbdg_sample_receivers(self.s.ctx, st_[5 * i + 5], self.traces[n0 + i], stream=self.stream)

    def _forward_keep_all(self):
        st = self.stages
        st[0].zero_()
        self.res.zero_()
        for i in range(self.nsteps):
            t = i * self.dt
            for k in range(5):
                j = 5 * i + k
                bbdg.bbdg_rk_stage(self.s.ctx, st[j], st[j + 1], self.res, k, t, self.dt, stream=self.stream)
            bbdg.bbdg_sample_receivers(self.s.ctx, st[5 * i + 5], self.traces[i], stream=self.stream)
        self.q.copy_(st[5 * self.nsteps])
        return self._misfit()

    def backward(self):
        """Reverse sweep; returns dJ/dkappa (device tensor [K], FP64)."""
        import torch
        K = self.s.K
        grad = torch.zeros(K, dtype=torch.float64, device=self.q.device)
        lq = torch.zeros(self.shape, dtype=torch.float64, device=self.q.device)
        lr = torch.zeros_like(lq)
        if self.keep_all:
            for n in reversed(range(self.nsteps)):
                bbdg.bbdg_adjoint_step(self.s.ctx, lq, lr, self.stages[5 * n:5 * n + 5], grad, n * self.dt, self.dt,
                                       rec_residual=self.resid[n], stream=self.stream)
            return grad
        res = torch.empty_like(lq)
        for n0 in sorted(self.ckpt, reverse=True):
            m = min(self.C, self.nsteps - n0)
            if n0 != self.kept:
                q0, r0 = self.ckpt[n0]
                res.copy_(r0)
                self.stages[0].copy_(q0)
                self._run_segment(n0, m, res, traces=False)
            for i in reversed(range(m)):
                n = n0 + i
                bbdg.bbdg_adjoint_step(self.s.ctx, lq, lr, self.stages[5 * i:5 * i + 5], grad, n * self.dt, self.dt,
                                       rec_residual=self.resid[n], stream=self.stream)
        return grad


def _autograd_function():
    import torch

    class KappaMisfit(torch.autograd.Function):
        """J(kappa) with the discrete-adjoint gradient: J = KappaMisfit.apply(kappa, driver, rho)."""

        @staticmethod
        def forward(ctx, kappa, driver, rho):
            driver.set_kappa(rho, kappa.detach().to(dtype=torch.float64))
            J, _ = driver.forward()
            ctx.driver = driver
            return torch.tensor(J, dtype=torch.float64, device=kappa.device)

        @staticmethod
        def backward(ctx, gJ):
            g = ctx.driver.backward()
            return gJ * g.to(gJ.device), None, None

    return KappaMisfit


def kappa_misfit(kappa, driver, rho):
    """torch.autograd entry: J(kappa) whose .backward() fills kappa.grad with dJ/dkappa."""
    return _autograd_function().apply(kappa, driver, rho)
