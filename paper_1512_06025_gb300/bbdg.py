"""Thin Python binding of libbbdg (include/bbdg.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does nothing but
convert arguments (numpy host arrays, torch CUDA tensors as raw device pointers, the
current CUDA stream) and raise on a non-zero status.  All arithmetic of the solver runs in
the library's CUDA kernels; there is no Python or CPU fallback: if the library cannot be
loaded, every call raises.

PyTorch is used only for device memory and streams (tensors are passed by data_ptr()).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbbdg.so")

BBDG_OK = 0
BBDG_BB, BBDG_NODAL, BBDG_NODAL_TC = 0, 1, 2
BBDG_ETIMEOUT = -7
BBDG_F64, BBDG_F32, BBDG_F32_LIFT64 = 0, 1, 2
BBDG_LIFT_OPTIMAL, BBDG_LIFT_SPARSE_EL = 0, 1
BBDG_FLUX_UPWIND, BBDG_FLUX_CENTRAL = 0, 1
BBDG_BC_MIRROR, BBDG_BC_ABSORBING = 0, 1
BBDG_FORM_GROUP, BBDG_FORM_WARP, BBDG_FORM_PIPE, BBDG_FORM_ROWS, BBDG_FORM_THREAD = 0, 1, 2, 3, 4

_lib = None


class BBDGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libbbdg error {code}: {msg}")
        self.code = code


def load(path: str | None = None):
    """Load libbbdg.so (built by paper_1512_06025_gb300.build); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise BBDGError(-100, f"{path} not found: build it with paper_1512_06025_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P, I, L, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    sig = {
        "bbdg_setup_mesh": (I, [ctypes.POINTER(P), L, P, L, P, P, P]),
        "bbdg_setup_operators": (I, [P, I, I, I, I]),
        "bbdg_set_materials": (I, [P, P, P, L]),
        "bbdg_set_flux": (I, [P, I]),
        "bbdg_set_boundary": (I, [P, I]),
        "bbdg_set_stage_form": (I, [P, I, I]),
        "bbdg_set_launch_shape": (I, [P, I, I]),
        "bbdg_step_graph": (I, [P, P, P, P, L, D, D, I, P, P]),
        "bbdg_step_noalloc": (I, [P, P, P, L, D, D, I, P]),
        "bbdg_step_host": (I, [P, P, P, L, D, D, I, P, P]),
        "bbdg_step_noalloc_max_bytes": (ctypes.c_size_t, []),
        "bbdg_set_sources": (I, [P, L, P, P, D, D]),
        "bbdg_set_receivers": (I, [P, L, P]),
        "bbdg_rhs": (I, [P, P, P, L, D, P]),
        "bbdg_step": (I, [P, P, P, P, L, D, D, I, P, P]),
        "bbdg_sample_receivers": (I, [P, P, P, L, P]),
        "bbdg_rk_stage": (I, [P, P, P, P, L, I, D, D, P]),
        "bbdg_adjoint_rhs": (I, [P, P, P, L, P]),
        "bbdg_adjoint_step": (I, [P, P, P, P, P, L, D, D, P, P]),
        "bbdg_last_error": (ctypes.c_char_p, [P]),
        "bbdg_device_status": (I, [P]),
        "bbdg_destroy": (None, [P]),
        "bbdg_num_nodes": (I, [I]),
        "bbdg_nodal_nodes": (I, [I, P]),
        "bbdg_measure_fma_peak": (I, [I, ctypes.POINTER(D)]),
        "bbdg_misfit": (I, [P, P, P, L, P, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return [n for n in dir(load()) if n.startswith("bbdg_")]


def _check(rc, ctx=None):
    if rc != BBDG_OK:
        msg = load().bbdg_last_error(ctx)
        raise BBDGError(rc, msg.decode() if msg else "")


def _host(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def _dev(t):
    """Raw device pointer of a CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("state tensors must be contiguous CUDA tensors")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


# ---------------------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ---------------------------------------------------------------------------------------
def bbdg_setup_mesh(vxyz, EToV, rho, kappa):
    lib = load()
    v, vp = _host(vxyz, np.float64)
    e, ep = _host(EToV, np.int32)
    r, rp = _host(rho, np.float64)
    k, kp = _host(kappa, np.float64)
    ctx = ctypes.c_void_p()
    rc = lib.bbdg_setup_mesh(ctypes.byref(ctx), v.shape[0], vp, e.shape[0], ep, rp, kp)
    _check(rc, None)
    return ctx


def bbdg_setup_operators(ctx, N, basis=BBDG_BB, precision=BBDG_F64, lift_variant=BBDG_LIFT_OPTIMAL):
    _check(load().bbdg_setup_operators(ctx, N, basis, precision, lift_variant), ctx)


def bbdg_set_materials(ctx, kappa, rho, S_or_1=None):
    """kappa, rho: FP64 arrays [K] (one medium) or [S][K] (one per shot).  CUDA tensors are
    passed by pointer; anything else is first copied to a CUDA tensor (marshalling only)."""
    import torch

    def dev(a):
        t = a if isinstance(a, torch.Tensor) else torch.as_tensor(np.asarray(a, dtype=np.float64))
        if not t.is_cuda:
            t = t.to(device="cuda", dtype=torch.float64)
        if t.dtype != torch.float64:
            raise ValueError("kappa and rho must be float64")
        return t.contiguous()

    k, r = dev(kappa), dev(rho)
    if k.shape != r.shape or k.dim() not in (1, 2):
        raise ValueError("kappa and rho must both be [K] or [S][K]")
    if S_or_1 is None:
        S_or_1 = k.shape[0] if k.dim() == 2 else 1
    _check(load().bbdg_set_materials(ctx, _dev(k), _dev(r), int(S_or_1)), ctx)


def bbdg_set_flux(ctx, flux):
    _check(load().bbdg_set_flux(ctx, flux), ctx)


def bbdg_set_boundary(ctx, bc):
    _check(load().bbdg_set_boundary(ctx, bc), ctx)


def bbdg_set_stage_form(ctx, form, warps_per_cta=8):
    _check(load().bbdg_set_stage_form(ctx, form, warps_per_cta), ctx)


def bbdg_set_launch_shape(ctx, E, shots_per_tile=1):
    _check(load().bbdg_set_launch_shape(ctx, E, shots_per_tile), ctx)


def bbdg_set_sources(ctx, xyz, shot=None, f0=10.0, t0=0.05):
    x, xp = _host(np.atleast_2d(xyz), np.float64)
    n = x.shape[0]
    s, sp = _host(np.zeros(n) if shot is None else shot, np.int64)
    _check(load().bbdg_set_sources(ctx, n, xp, sp, f0, t0), ctx)


def bbdg_set_receivers(ctx, xyz):
    x, xp = _host(np.atleast_2d(xyz), np.float64)
    _check(load().bbdg_set_receivers(ctx, x.shape[0], xp), ctx)


def bbdg_rhs(ctx, q, rhs, S=None, t=0.0, stream=None):
    S = q.shape[0] if S is None else S
    _check(load().bbdg_rhs(ctx, _dev(q), _dev(rhs), S, t, _stream(stream)), ctx)


def bbdg_step(ctx, q, res, scratch, t0, dt, nsteps, traces=None, S=None, stream=None):
    S = q.shape[0] if S is None else S
    _check(load().bbdg_step(ctx, _dev(q), _dev(res), _dev(scratch), S, t0, dt, nsteps, _dev(traces),
                            _stream(stream)), ctx)


def bbdg_step_host(ctx, q_host, work, t0, dt, nsteps, traces_host=None, S=None, stream=None):
    """q_host (and traces_host): CPU tensors, pinned for asynchronous copies; work: a CUDA
    buffer of at least 3 state arrays (+ the traces)."""
    if q_host.is_cuda or not q_host.is_contiguous():
        raise ValueError("q_host must be a contiguous CPU tensor")
    if traces_host is not None and (traces_host.is_cuda or not traces_host.is_contiguous()):
        raise ValueError("traces_host must be a contiguous CPU tensor")
    S = q_host.shape[0] if S is None else S
    th = None if traces_host is None else ctypes.c_void_p(traces_host.data_ptr())
    _check(load().bbdg_step_host(ctx, ctypes.c_void_p(q_host.data_ptr()), _dev(work), S, t0, dt, nsteps, th,
                                 _stream(stream)), ctx)


def bbdg_step_graph(ctx, q, res, scratch, t0, dt, nsteps, traces=None, S=None, stream=None):
    S = q.shape[0] if S is None else S
    _check(load().bbdg_step_graph(ctx, _dev(q), _dev(res), _dev(scratch), S, t0, dt, nsteps, _dev(traces),
                                  _stream(stream)), ctx)


def bbdg_step_noalloc(ctx, q, res, t0, dt, nsteps, S=None, stream=None):
    """bbdg_step without a caller-provided ping-pong buffer (the library's static array is
    used instead); for callers that cannot allocate device memory."""
    S = q.shape[0] if S is None else S
    _check(load().bbdg_step_noalloc(ctx, _dev(q), _dev(res), S, t0, dt, nsteps, _stream(stream)), ctx)


def bbdg_step_noalloc_max_bytes():
    return int(load().bbdg_step_noalloc_max_bytes())


def bbdg_rk_stage(ctx, q_in, q_out, res, stage, t, dt, S=None, stream=None):
    S = q_in.shape[0] if S is None else S
    _check(load().bbdg_rk_stage(ctx, _dev(q_in), _dev(q_out), _dev(res), S, stage, t, dt, _stream(stream)), ctx)


def bbdg_adjoint_rhs(ctx, mu, out, S=None, stream=None):
    S = mu.shape[0] if S is None else S
    _check(load().bbdg_adjoint_rhs(ctx, _dev(mu), _dev(out), S, _stream(stream)), ctx)


def bbdg_adjoint_step(ctx, lam_q, lam_res, q_stages, grad_kappa, t, dt, rec_residual=None, S=None, stream=None):
    S = lam_q.shape[0] if S is None else S
    _check(load().bbdg_adjoint_step(ctx, _dev(lam_q), _dev(lam_res), _dev(q_stages), _dev(grad_kappa), S, t, dt,
                                    _dev(rec_residual), _stream(stream)), ctx)


def bbdg_sample_receivers(ctx, q, traces, S=None, stream=None):
    S = q.shape[0] if S is None else S
    _check(load().bbdg_sample_receivers(ctx, _dev(q), _dev(traces), S, _stream(stream)), ctx)


def bbdg_device_status(ctx):
    _check(load().bbdg_device_status(ctx), ctx)


def bbdg_destroy(ctx):
    load().bbdg_destroy(ctx)


def bbdg_num_nodes(N):
    return load().bbdg_num_nodes(N)


def bbdg_misfit(ctx, traces, data, resid, J, stream=None):
    """resid = traces - data and J[0] = 1/2 sum resid^2 (FP64, compensated), on the device."""
    _check(load().bbdg_misfit(ctx, _dev(traces), _dev(data), int(traces.numel()), _dev(resid), _dev(J),
                              _stream(stream)), ctx)


def bbdg_measure_fma_peak(precision):
    """Measured FMA rate of the current device in TFLOP/s (BBDG_F64 or BBDG_F32)."""
    out = ctypes.c_double(0.0)
    _check(load().bbdg_measure_fma_peak(precision, ctypes.byref(out)), None)
    return float(out.value)


def bbdg_nodal_nodes(N):
    out = np.zeros((bbdg_num_nodes(N), 4))
    _check(load().bbdg_nodal_nodes(N, out.ctypes.data_as(ctypes.c_void_p)), None)
    return out


class Solver:
    """Owns one context: mesh + operators (+ sources/receivers).  Convenience wrapper over
    the entry points above; the caller owns the state tensors."""

    def __init__(self, VX, EToV, rho, kappa, N, basis=BBDG_BB, precision=BBDG_F64, lift_variant=BBDG_LIFT_OPTIMAL):
        self.ctx = bbdg_setup_mesh(VX, EToV, rho, kappa)
        self.K = int(np.asarray(EToV).shape[0])
        self.N = N
        self.basis = basis
        self.precision = precision
        self.lift_variant = lift_variant
        bbdg_setup_operators(self.ctx, N, basis, precision, lift_variant)

    def set_lift_variant(self, lift_variant):
        """Rebuild the operators with another lift variant (sources and receivers stay)."""
        bbdg_setup_operators(self.ctx, self.N, self.basis, self.precision, lift_variant)
        self.lift_variant = lift_variant

    def set_materials(self, kappa, rho):
        """kappa, rho: [K] (one medium) or [S][K] (one per shot), FP64."""
        shape = tuple(np.shape(kappa))
        if shape != tuple(np.shape(rho)) or shape[-1:] != (self.K,) or len(shape) not in (1, 2):
            raise ValueError(f"kappa and rho must both be [{self.K}] or [S][{self.K}]")
        bbdg_set_materials(self.ctx, kappa, rho)

    @property
    def Np(self):
        return bbdg_num_nodes(self.N)

    @property
    def torch_dtype(self):
        import torch
        return torch.float64 if self.precision == BBDG_F64 else torch.float32

    def close(self):
        if self.ctx:
            bbdg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
