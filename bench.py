"""Benchmark of the Bernstein-Bezier DG stage kernels on one GB300 (or N replicas).

Workload (the per-stage right-hand side + LSERK4 update of the paper, Sections 3-4.2):
  N = 7, unit cube [-1/2, 1/2]^3 split into 16^3 hexahedra x 6 = 24576 affine tetrahedra,
  unit wavespeed, upwind flux, dt = 0.25 h / (N+1)^2; seeded random BB coefficients of the
  standing-mode problem's size (the coefficient values do not change the work).
A timed step is one LSERK4 step = 5 fused stage kernels (trace gather, upwind flux, volume
derivatives, L0 + reduction chain, update) through the C ABI (bbdg_rk_stage), ping-pong
buffers, inputs resident in HBM.  L2 is flushed (a 512 MB write) between timed steps.

Metric: GDOF/s per RK stage = 4 fields x K x N_p / (time of one stage) / 1e9.

--impl reference times the CPU oracle (test infrastructure) on the same metric.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BB-DG GDOF/s per RK stage vs nodal, N=1–10, FP32/FP64; gradient/forward ratio"
UNIT = "GDOF/s"
N_ORDER = 7
N_HEX = 16
FORM_NAMES = {0: "group", 1: "warp", 2: "pipe", 3: "rows", 4: "thread"}
# kernel of each BB stage form (roofline key and name in the report)
FORM_KERNELS = {"group": "bb_stage_kernel", "pipe": "bb_pipe_kernel", "warp": "bb_stage_warp_kernel",
                "thread": "bb_thread_kernel"}


def workload_config():
    K = 6 * N_HEX ** 3
    return {"workload": f"C2: N={N_ORDER}, {N_HEX}^3x6={K} tets, unit cube, unit wavespeed, upwind, LSERK4",
            "N": N_ORDER, "K": K, "dof_per_stage": 4 * K * (N_ORDER + 1) * (N_ORDER + 2) * (N_ORDER + 3) // 6,
            "l2": "flushed between timed steps (512 MB write)", "inputs": "resident in HBM"}


def np_of(N):
    return (N + 1) * (N + 2) * (N + 3) // 6


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def reduce_max(x, world, device):
    """The maximum of x over the ranks (the slowest replica's time); x itself when alone."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(world, dof_per_rank, stage_ms_max):
    """Whole-job GDOF/s of `world` replicas that each advance dof_per_rank unknowns per stage,
    timed by the slowest rank."""
    return world * dof_per_rank / (stage_ms_max * 1e-3) / 1e9


# ---------------------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"bbdg_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "50"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        loaded = [r for r in rows if r[0] > 0.5 * r[1]] or rows
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for _, _, p in loaded:
            for n, v in zip(names[1:], p[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": sorted(reasons), "samples": len(loaded)}


# ---------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------
def stage_bytes_per_element(N, tsize):
    """Algorithmic HBM bytes of one fused stage per element, averaged over the five stages
    of a step: read q and res, write q_new and res (16 N_p words) in stages 2-5; stage 1
    (LSERK a_1 = 0) does not read res (12 N_p words); the geometry record (20 words), 4
    neighbour ids and the face code word (20 bytes).  Neighbour traces are counted as L2
    re-reads (0 bytes)."""
    return (4 * 16 + 12) * np_of(N) * tsize / 5 + 20 * tsize + 20


def stage_flops_per_element(N):
    """Floating-point operations of one fused stage per element, counted from the kernel
    (FMA = 2): fluxes 14 per face node; L0 14 per output (7 FMA); reduction chain 6 per
    output; degree N-1 gradient/divergence coefficients 44 per coefficient; per node 94
    (gradient 21, divergence 7, lift gather 34, residual 8, update 24)."""
    Np, Nfp, Np1 = np_of(N), (N + 1) * (N + 2) // 2, np_of(N - 1)
    return 4 * Nfp * 14 + 8 * Nfp * 14 + 8 * (Np - Nfp) * 6 + Np1 * 44 + Np * 94


def nodal_tc_flops_per_element(N, rows=False):
    """Tensor-core FLOPs a nodal tensor-core kernel issues per element (FMA = 2), three TF32
    passes (hi.hi, hi.lo, lo.hi).  Node-row kernel: rows padded to 128-row tiles, [D^r | L^0]
    K-slices padded to 8, two columns per derivative region (3) and per face (4).  Element-row
    kernel (rows=True): 4 rows (fields) per element, N = N_p padded to a multiple of 16, K =
    3 N_p + 4 N^f_p padded to 8."""
    Np, Nfp = np_of(N), (N + 1) * (N + 2) // 2
    if rows:
        NN = 16 if Np <= 16 else (Np + 15) // 16 * 16
        return 3 * 2 * 4 * NN * ((3 * Np + 4 * Nfp + 7) // 8 * 8)
    Mpad = (Np + 127) // 128 * 128
    Kd, Kf = (Np + 7) // 8 * 8, (Nfp + 7) // 8 * 8
    return 3 * 2 * Mpad * (Kd * 6 + Kf * 8)


# source file of each BB stage form's kernel (the digest ties a recorded ncu traffic figure
# to the source it was taken on)
FORM_SOURCES = {"group": "bb_stage.cuh", "pipe": "bb_pipe.cuh", "warp": "bb_stage_warp.cuh",
                "thread": "bb_stage_thread.cuh"}


def source_digest(form="group"):
    h = hashlib.sha256()
    with open(os.path.join(ROOT, "paper_1512_06025_gb300", "csrc", FORM_SOURCES[form]), "rb") as f:
        h.update(f.read())
    return h.hexdigest()


def recorded_traffic(kernel_key, form="group"):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current
    kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
        rec = d.get(kernel_key)
        if rec and rec.get("source_sha256") == source_digest(form):
            return rec.get("dram_bytes_per_launch")
    except Exception:
        return None
    return None


def run_gpu(args, rank, world, local_rank):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1512_06025_gb300 import bbdg, inputs

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    N, n = N_ORDER, N_HEX
    VX, EToV = inputs.kuhn_cube_mesh(n)
    K = len(EToV)
    Np = np_of(N)
    rho, kappa = np.ones(K), np.ones(K)
    dt = 0.25 * (1.0 / n) / (N + 1) ** 2
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    out = {}

    def measure(precision, steps, warmup, basis=None, tune=True):
        from paper_1512_06025_gb300 import autotune
        basis = bbdg.BBDG_BB if basis is None else basis
        s = bbdg.Solver(VX, EToV, rho, kappa, N, basis=basis, precision=precision)
        dtype = s.torch_dtype
        q0 = torch.tensor(inputs.abi_layout(inputs.random_state(K, N)), dtype=dtype, device=dev)
        E, form, forms = None, None, {}
        if tune and basis in (bbdg.BBDG_BB, bbdg.BBDG_NODAL_TC):
            form, forms = autotune.tune_form(s, q0.clone(), torch.zeros_like(q0), torch.empty_like(q0))
            E = s.tuned.get("E")
        elif tune:
            E, _ = autotune.tune(s, q0.clone(), torch.zeros_like(q0), torch.empty_like(q0), basis=basis)
        qa, qb = q0.clone(), torch.empty_like(q0)
        res = torch.zeros_like(q0)
        t = 0.0

        def one_step(events=None):
            nonlocal qa, qb, t
            for st in range(5):
                if events is not None:
                    events[st].record(stream)
                bbdg.bbdg_rk_stage(s.ctx, qa, qb, res, st, t, dt, stream=stream)
                qa, qb = qb, qa
            if events is not None:
                events[5].record(stream)
            t += dt

        for _ in range(warmup):
            one_step()
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(steps)]
        for i in range(steps):
            flush.fill_(float(i))            # evict L2 between timed steps (outside the events)
            one_step(evs[i])
        torch.cuda.synchronize()
        barrier()
        step_ms = [e[0].elapsed_time(e[5]) for e in evs]
        stage_ms = [e[j].elapsed_time(e[j + 1]) for e in evs for j in range(5)]
        finite = bool(torch.isfinite(qa).all().item())
        s.close()
        return {"step_ms": sum(step_ms) / steps, "stage_ms": sum(stage_ms) / len(stage_ms),
                "total_ms": sum(step_ms), "finite": finite, "E": E, "form": FORM_NAMES.get(form),
                "forms_ms_per_stage": {k: round(v, 5) for k, v in forms.items()}}

    # measured FMA rates of this GPU (the FP64 path's arithmetic roofline denominator)
    fma_peaks = {"f64": bbdg.bbdg_measure_fma_peak(bbdg.BBDG_F64), "f32": bbdg.bbdg_measure_fma_peak(bbdg.BBDG_F32)}
    with ClockSampler(local_rank) as clk:
        f32 = measure(bbdg.BBDG_F32, args.steps, args.warmup)
        f64 = measure(bbdg.BBDG_F64, max(4, args.steps // 10), max(3, args.warmup // 2)) if not args.fp32_only else None
        nod32 = nod64 = nodtc = None
        if not args.fp32_only and not args.no_nodal:
            nod32 = measure(bbdg.BBDG_F32, max(4, args.steps // 10), 3, basis=bbdg.BBDG_NODAL)
            nod64 = measure(bbdg.BBDG_F64, 4, 3, basis=bbdg.BBDG_NODAL)
            nodtc = measure(bbdg.BBDG_F32, max(4, args.steps // 10), 3, basis=bbdg.BBDG_NODAL_TC)
    clocks = clk.summary()

    # end to end through the public API (bbdg_step_host: the library copies the pinned host
    # state in, steps it and copies it back out, every step).  Serving loop over P independent state batches, one stream each: the upload of
    # batch k+1, the step of batch k and the download of batch k-1 overlap (copy engines and
    # SMs run concurrently); every step moves its own q both ways.  A step's state is q
    # alone: its first stage has a_1 = 0 and overwrites the residual register without
    # reading it, so res stays on the device as scratch.  The one-batch loop (copies and
    # step strictly in sequence) is reported beside it.
    e2e = None
    if not args.no_e2e:
        s = bbdg.Solver(VX, EToV, rho, kappa, N, precision=bbdg.BBDG_F32)
        P = 3
        lanes = []
        for j in range(P):
            hq = torch.tensor(inputs.abi_layout(inputs.random_state(K, N, seed=inputs.SEED_STATE + j)),
                              dtype=torch.float32).pin_memory()
            lanes.append({"hq": hq, "work": torch.empty((3,) + tuple(hq.shape), dtype=torch.float32, device=dev),
                          "st": torch.cuda.Stream(device=dev)})
        e2e_steps = max(3 * P, (args.steps // 10) // P * P)

        def e2e_step(L, t):
            # the library's host-buffer entry point: upload, step, download on the lane's stream
            bbdg.bbdg_step_host(s.ctx, L["hq"], L["work"], t, dt, 1, stream=L["st"])

        def timed(nlanes, nsteps):
            for i in range(nlanes):
                e2e_step(lanes[i], 0.0)
            torch.cuda.synchronize()
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for L in lanes[:nlanes]:
                L["st"].wait_event(e0)
            for i in range(nsteps):
                e2e_step(lanes[i % nlanes], i * dt)
            for L in lanes[:nlanes]:
                ev = torch.cuda.Event()
                ev.record(L["st"])
                stream.wait_event(ev)
            e1.record(stream)
            torch.cuda.synchronize()
            barrier()
            return e0.elapsed_time(e1) / nsteps

        ms = timed(P, e2e_steps)
        ms_serial = timed(1, max(3, e2e_steps // P))
        nbytes = lanes[0]["hq"].numel() * 4
        e2e = {"step_ms": ms, "serial_step_ms": ms_serial, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "launches_per_step": 6, "batches_in_flight": P}
        s.close()

    # max over ranks
    def allmax(x):
        return reduce_max(x, world, dev)

    f32_stage = allmax(f32["stage_ms"])
    f32_step = allmax(f32["step_ms"])
    dof = 4 * K * Np
    value = weak_value(world, dof, f32_stage)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    bytes_launch = stage_bytes_per_element(N, 4) * K
    achieved = bytes_launch / (f32["stage_ms"] * 1e-3) / 1e9
    result = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(f32_step, 5), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded random BB coefficients, Kuhn cube mesh)",
        "config": {**workload_config(), "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
                     "frac": round(achieved / hbm_peak, 4),
                     "traffic": recorded_traffic(f"{f32['form']}_f32_N7", f32["form"]),
                     "kernel": f"{FORM_KERNELS[f32['form']]}<float,7>", "peak_source": peak_src,
                     "algorithmic_bytes_per_launch": bytes_launch},
        "clocks": clocks,
        "gpu_launches": 5 * args.steps,
        "finite": f32["finite"],
    }
    if f64 is not None:
        f64_stage = allmax(f64["stage_ms"])
        flops = stage_flops_per_element(N) * K
        fp64_peak = fma_peaks["f64"]
        result["fp64"] = {"value": round(world * dof / (f64_stage * 1e-3) / 1e9, 3), "unit": UNIT,
                          "stage_ms": round(f64_stage, 5), "dtype": "f64", "form": f64["form"],
                          "roofline": {"bound": "alu", "achieved": round(flops / (f64["stage_ms"] * 1e-3) / 1e12, 4),
                                       "peak": round(fp64_peak, 4), "unit": "TFLOP/s",
                                       "frac": round(flops / (f64["stage_ms"] * 1e-3) / 1e12 / fp64_peak, 4),
                                       "peak_source": "measured in this run (bbdg_measure_fma_peak, FP64 FMA chains)"}}
    result["config"]["elements_per_group"] = f32["E"]
    result["config"]["stage_form"] = f32["form"]
    result["stage_forms_ms"] = f32["forms_ms_per_stage"]
    result["fma_peaks_tflops"] = {k: round(v, 3) for k, v in fma_peaks.items()}
    if nod32 is not None:
        n32, n64 = allmax(nod32["stage_ms"]), allmax(nod64["stage_ms"])
        result["nodal"] = {"f32": {"value": round(world * dof / (n32 * 1e-3) / 1e9, 3), "unit": UNIT,
                                   "stage_ms": round(n32, 5)},
                           "f64": {"value": round(world * dof / (n64 * 1e-3) / 1e9, 3), "unit": UNIT,
                                   "stage_ms": round(n64, 5)},
                           "bb_over_nodal_f32": round(n32 / f32_stage, 3),
                           "kernel": "nodal_stage_kernel (dense Warp & Blend, node per thread, SIMT)"}
        ntc = allmax(nodtc["stage_ms"])
        tc_rows = nodtc.get("form") == "rows"
        tc_flops = nodal_tc_flops_per_element(N, tc_rows) * K
        tf32_peak = float(peaks.get("bf16_tflops", 1900.0)) / 2.0
        result["nodal"]["tc_f32"] = {
            "value": round(world * dof / (ntc * 1e-3) / 1e9, 3), "unit": UNIT, "stage_ms": round(ntc, 5),
            "kernel": ("nodal_tcr_kernel (tcgen05 kind::tf32, 3xTF32 split, element rows x node columns)" if tc_rows else
                       "nodal_tc_kernel (tcgen05 kind::tf32, 3xTF32 split, [D^r | L^0] with vertex symmetry)"),
            "forms_ms": nodtc.get("forms_ms_per_stage"),
            "roofline": {"bound": "tensor", "achieved": round(tc_flops / (nodtc["stage_ms"] * 1e-3) / 1e12, 2),
                         "peak": round(tf32_peak, 1), "unit": "TFLOP/s",
                         "frac": round(tc_flops / (nodtc["stage_ms"] * 1e-3) / 1e12 / tf32_peak, 4),
                         "peak_source": "measured bf16 burst x 1/2 (nominal TF32 : BF16 dense ratio)"}}
        result["nodal"]["bb_over_nodal_tc_f32"] = round(ntc / f32_stage, 3)
        if f64 is not None:
            result["nodal"]["bb_over_nodal_f64"] = round(n64 / allmax(f64["stage_ms"]), 3)
    if e2e is not None:
        e2e_ms = allmax(e2e["step_ms"])
        e2e_serial = allmax(e2e["serial_step_ms"])
        result["e2e"] = {"value": round(weak_value(world, dof, e2e_ms / 5), 3), "unit": UNIT,
                         "h2d_bytes_per_step": e2e["h2d_bytes_per_step"], "d2h_bytes_per_step": e2e["d2h_bytes_per_step"],
                         "ms_per_step": round(e2e_ms, 4),
                         "mode": f"bbdg_step_host, {e2e['batches_in_flight']} independent state batches on as many "
                                 "streams: upload of q, step, download of q of consecutive batches overlap (res is "
                                 "device scratch: LSERK a_1 = 0)",
                         "serial": {"value": round(weak_value(world, dof, e2e_serial / 5), 3),
                                    "ms_per_step": round(e2e_serial, 4),
                                    "mode": "one batch: upload, step, download in sequence"}}
    if not args.fp32_only and not args.no_batched:
        result["batched"] = batched_shots(bbdg, inputs, torch, dev, stream, world, reduce_max, hbm_peak)
    if not args.no_adjoint:
        adj = adjoint_ratio(bbdg, inputs, torch, dev, stream)
        result["adjoint"] = adj
        result["gradient_over_forward"] = adj["ratio"]
    if not args.no_sweep:
        pk = {"hbm_gbs": hbm_peak, "f64_tflops": fma_peaks["f64"], "f32_tflops": fma_peaks["f32"],
              "tf32_tflops": float(peaks.get("bf16_tflops", 1900.0)) / 2.0}
        result["sweep"] = sweep(bbdg, inputs, torch, dev, stream, flush, pk, full=args.sweep)
        result["sweep"]["large_mesh"] = sweep_large(
            bbdg, inputs, torch, dev, stream, flush, pk, orders=tuple(LARGE_MESH_N) if args.sweep else (7,),
            precisions=("f32", "f64") if args.sweep else ("f32",))
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return result


def batched_shots(bbdg, inputs, torch, dev, stream, world, reduce_max, hbm_peak, nsteps=500):
    """C4 as configured: S = 64 shots on a 32^3 x 6 = 196 608-tet mesh, N = 5, FP32, layered
    wavespeed, one Ricker source per shot, zero initial state, all shots advanced together
    for nsteps LSERK4 steps captured in ONE CUDA graph (bbdg_step_graph from t0 = 0, so every
    source fires at its real stage times); stage form and launch shape (elements per group,
    shots per tile) from the autotuner.  The timed region is that one graph launch (its
    capture, a few ms of host work, included).  11.3 GB per state array (far larger than
    L2)."""
    from paper_1512_06025_gb300 import autotune
    N, n, S = 5, 32, 64
    VX, EToV = inputs.kuhn_cube_mesh(n)
    K = len(EToV)
    c = inputs.layered_wavespeed(VX, EToV)
    rho, kappa = inputs.materials_from_wavespeed(c)
    dt = 0.25 * (1.0 / n) / (N + 1) ** 2 / c.max()
    s = bbdg.Solver(VX, EToV, rho, kappa, N, precision=bbdg.BBDG_F32)
    f0, t0 = 10.0, 0.05
    bbdg.bbdg_set_sources(s.ctx, inputs.random_points(S, -0.4, 0.4), np.arange(S, dtype=np.int64), f0, t0)
    q = torch.zeros((S, K, s.Np, 4), dtype=torch.float32, device=dev)
    res, scr = torch.zeros_like(q), torch.empty_like(q)
    form, _ = autotune.tune_form(s, q, res, scr, S=S, reps=2)
    q.zero_()
    res.zero_()
    bbdg.bbdg_step(s.ctx, q, res, scr, 0.0, dt, 2, stream=stream)           # warm
    q.zero_()
    res.zero_()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    bbdg.bbdg_step_graph(s.ctx, q, res, scr, 0.0, dt, nsteps, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    stage_ms = reduce_max(e0.elapsed_time(e1) / (nsteps * 5), world, dev)
    finite = bool(torch.isfinite(q).all().item())
    pmax = float(q[..., 0].abs().max().item())
    dof = 4 * K * s.Np * S
    E = s.tuned["E"]
    s.close()
    del q, res, scr
    torch.cuda.empty_cache()
    return {"workload": f"C4: {n}^3x6={K} tets, S={S} shots, N={N}, FP32, layered c, one Ricker source per shot, "
                        f"{nsteps} steps",
            "value": round(world * dof / (stage_ms * 1e-3) / 1e9, 3), "unit": UNIT, "stage_ms": round(stage_ms, 4),
            "graph": f"{nsteps} steps ({5 * nsteps} stage launches) captured in one bbdg_step_graph from t0 = 0",
            "stage_form": FORM_NAMES[form], "elements_per_group": E,
            "roofline": bb_roofline(N, 4, stage_ms, K * S, {"hbm_gbs": hbm_peak}),
            "finite": finite, "max_abs_p": pmax,
            "final_time": round(nsteps * dt, 6), "ricker": {"f0": f0, "t0": t0},
            "dt": dt}


def adjoint_ratio(bbdg, inputs, torch, dev, stream, nsteps=400, C=20):
    """C5: N = 5, 16^3 x 6 tets, c ~ U[1, 3], 8 Ricker sources, 256 receivers, FP64,
    nsteps LSERK4 steps; misfit to synthetic data from a 5 % perturbed c.  Wall times of a
    plain forward solve and of forward + reverse sweep, for MisfitGradient's automatic storage
    plan (the whole trajectory when it fits half of the free HBM) and for checkpoints every
    C steps with recomputation."""
    from paper_1512_06025_gb300.gradient import MisfitGradient
    N, n = 5, 16
    VX, EToV = inputs.kuhn_cube_mesh(n)
    K = len(EToV)
    c = inputs.uniform_wavespeed(K)
    rho, kappa = inputs.materials_from_wavespeed(c)
    xs = inputs.random_points(8, (-0.4, -0.4, 0.0), (0.4, 0.4, 0.4))
    rec = inputs.receiver_plane(1.0 / n, 16)
    dt = 0.25 * (1.0 / n) / (N + 1) ** 2 / c.max()
    s = bbdg.Solver(VX, EToV, rho, kappa, N, precision=bbdg.BBDG_F64)
    bbdg.bbdg_set_sources(s.ctx, xs, np.zeros(8, dtype=np.int64), 10.0, 0.05)
    bbdg.bbdg_set_receivers(s.ctx, rec)
    ctrue = c * (1 + 0.05 * np.random.default_rng(inputs.SEED_CTRUE).uniform(-1, 1, K))
    data = torch.zeros((nsteps, len(rec)), dtype=torch.float64, device=dev)
    q, res, scr = (torch.zeros((1, K, s.Np, 4), dtype=torch.float64, device=dev) for _ in range(3))
    traces = torch.zeros((nsteps, 1, len(rec)), dtype=torch.float64, device=dev)
    bbdg.bbdg_set_materials(s.ctx, ctrue ** 2, rho)
    bbdg.bbdg_step(s.ctx, q, res, scr, 0.0, dt, nsteps, traces=traces, stream=stream)
    data.copy_(traces[:, 0, :])
    bbdg.bbdg_set_materials(s.ctx, kappa, rho)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    bbdg.bbdg_step(s.ctx, q, res, scr, 0.0, dt, 5, stream=stream)      # warm
    torch.cuda.synchronize()
    e[0].record(stream)
    q.zero_()
    res.zero_()
    bbdg.bbdg_step(s.ctx, q, res, scr, 0.0, dt, nsteps, traces=traces, stream=stream)
    e[1].record(stream)
    torch.cuda.synchronize()
    fwd = e[0].elapsed_time(e[1])
    del q, res, scr
    out = {"workload": f"C5: N=5, 16^3x6={K} tets, c~U[1,3], 8 sources, 256 receivers, FP64, {nsteps} steps",
           "forward_ms": round(fwd, 2)}
    for name, ce in (("auto", None), ("checkpoints", C)):
        drv = MisfitGradient(s, dt, nsteps, data, checkpoint_every=ce, stream=stream)
        drv.forward()
        drv.backward()                                                   # warm
        torch.cuda.synchronize()
        t = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        t[0].record(stream)
        J, _ = drv.forward()
        g = drv.backward()
        t[1].record(stream)
        torch.cuda.synchronize()
        grad = t[0].elapsed_time(t[1])
        out[name] = {"plan": "whole trajectory (5 nsteps + 1 states)" if drv.keep_all else f"checkpoints every {drv.C} steps",
                     "stored_states": int(drv.stages.shape[0]), "gradient_ms": round(grad, 2),
                     "ratio": round(grad / fwd, 3), "misfit": J, "finite": bool(torch.isfinite(g).all().item())}
        del drv
        torch.cuda.empty_cache()
    s.close()
    # the configured plan (checkpoints every C steps, segments recomputed) is the headline;
    # the whole-trajectory plan is reported beside it
    out["ratio"] = out["checkpoints"]["ratio"]
    out["ratio_plan"] = out["checkpoints"]["plan"]
    return out


def time_stages(bbdg, torch, s, q0, dt, stream, flush, steps):
    """Median ms per RK stage over `steps` timed LSERK4 steps (5 bbdg_rk_stage launches each,
    CUDA events on the launching stream, L2 flushed before each step), after one warm step."""
    qa, qb, res = q0.clone(), torch.empty_like(q0), torch.zeros_like(q0)
    ms = []
    for it in range(steps + 1):
        flush.fill_(float(it))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for st in range(5):
            bbdg.bbdg_rk_stage(s.ctx, qa, qb, res, st, 0.0, dt, stream=stream)
            qa, qb = qb, qa
        e1.record(stream)
        torch.cuda.synchronize()
        if it >= 1:
            ms.append(e0.elapsed_time(e1) / 5)
    finite = bool(torch.isfinite(qa).all().item())
    del qa, qb, res
    return sorted(ms)[len(ms) // 2], finite


def bb_roofline(N, tsize, stage_ms, K, peaks):
    """HBM roofline of a BB stage in FP32 (algorithmic bytes over the measured copy peak), or
    the FP64 pipe roofline in FP64 (algorithmic FLOPs over the measured FP64 FMA rate)."""
    if tsize == 4:
        gbs = stage_bytes_per_element(N, 4) * K / (stage_ms * 1e-3) / 1e9
        return {"bound": "hbm", "achieved_gbs": round(gbs, 1), "frac": round(gbs / peaks["hbm_gbs"], 4)}
    tf = stage_flops_per_element(N) * K / (stage_ms * 1e-3) / 1e12
    return {"bound": "alu", "achieved_tflops": round(tf, 4), "frac": round(tf / peaks["f64_tflops"], 4)}


def sweep(bbdg, inputs, torch, dev, stream, flush, peaks, steps=3, full=False):
    """C3: N = 1..10 on a 24^3 x 6 = 82 944-tet jittered cube, c ~ U[1, 3]: GDOF/s per stage
    and roofline fraction of the BB path (FP32: HBM bound; FP64: FP64-pipe bound), each with
    its fastest stage form and launch shape (autotune.tune_form), and of the nodal path
    (FP32: SIMT, and tensor cores with its TF32 roofline), L2 flushed between steps.
    full=True adds the element-per-warp kernel in both precisions as separate lines."""
    from paper_1512_06025_gb300 import autotune
    n = 24
    VX, EToV = inputs.kuhn_cube_mesh(n, jitter=0.1)
    K = len(EToV)
    c = inputs.uniform_wavespeed(K)
    rho, kappa = inputs.materials_from_wavespeed(c)
    paths = [("bb_f32", bbdg.BBDG_BB, bbdg.BBDG_F32), ("bb_f64", bbdg.BBDG_BB, bbdg.BBDG_F64),
             ("nodal_f32", bbdg.BBDG_NODAL, bbdg.BBDG_F32), ("nodal_tc_f32", bbdg.BBDG_NODAL_TC, bbdg.BBDG_F32)]
    if full:
        paths += [("bb_warp_f32", bbdg.BBDG_BB, bbdg.BBDG_F32), ("bb_warp_f64", bbdg.BBDG_BB, bbdg.BBDG_F64)]
    out = {}
    for N in range(1, 11):
        dt = 0.25 * (1.0 / n) / (N + 1) ** 2 / c.max()
        dof = 4 * K * np_of(N)
        row = {}
        for name, basis, prec in paths:
            s = bbdg.Solver(VX, EToV, rho, kappa, N, basis=basis, precision=prec)
            q0 = torch.tensor(inputs.abi_layout(inputs.random_state(K, N)), dtype=s.torch_dtype, device=dev)
            z, w = torch.zeros_like(q0), torch.empty_like(q0)
            if name.startswith("bb_warp"):
                W, _ = autotune.tune_warps(s, q0.clone(), z, w, reps=2)
                row[name + "_warps_per_cta"] = W
            elif basis in (bbdg.BBDG_BB, bbdg.BBDG_NODAL_TC):
                form, _ = autotune.tune_form(s, q0.clone(), z, w, reps=2)
                row[name + "_form"] = FORM_NAMES[form]
            else:
                autotune.tune(s, q0.clone(), z, w, basis=basis, reps=2)
            del z, w
            stage, finite = time_stages(bbdg, torch, s, q0, dt, stream, flush, steps)
            row[name] = round(dof / (stage * 1e-3) / 1e9, 3)
            if name in ("bb_f32", "bb_f64"):
                row[name + "_roofline"] = bb_roofline(N, 4 if prec == bbdg.BBDG_F32 else 8, stage, K, peaks)
            if name == "nodal_f32":
                # dense products: 6 N_p^2 + 8 N_p N^f_p multiply-adds per element, FP32 FMA pipe
                Np, Nfp = np_of(N), (N + 1) * (N + 2) // 2
                tf = 2.0 * (6 * Np * Np + 8 * Np * Nfp) * K / (stage * 1e-3) / 1e12
                row[name + "_roofline"] = {"bound": "alu", "achieved_tflops": round(tf, 2),
                                           "frac": round(tf / peaks["f32_tflops"], 4)}
            if name == "nodal_tc_f32":
                tf = nodal_tc_flops_per_element(N, row.get(name + "_form") == "rows") * K / (stage * 1e-3) / 1e12
                row[name + "_roofline"] = {"bound": "tensor", "achieved_tflops": round(tf, 2),
                                           "frac": round(tf / peaks["tf32_tflops"], 4)}
            row[name + "_finite"] = finite
            s.close()
            del q0
        row["bb_over_nodal_f32"] = round(row["bb_f32"] / row["nodal_f32"], 3)
        row["bb_over_nodal_tc_f32"] = round(row["bb_f32"] / row["nodal_tc_f32"], 3)
        row["working_set_mb_f32"] = round(3 * 4 * K * np_of(N) * 4 / 1e6, 1)
        out[N] = row
    return {"workload": f"C3: {n}^3x6={K} tets jittered 10% h, c~U[1,3], N=1..10", "unit": UNIT,
            "steps_timed": steps, "by_N": out}


# meshes whose three FP32 state arrays (q, q_out, res) exceed 4x the 129 MB L2
LARGE_MESH_N = {1: 80, 2: 58, 3: 48, 4: 40, 5: 34, 6: 30, 7: 26}


def sweep_large(bbdg, inputs, torch, dev, stream, flush, peaks, orders=(7,), precisions=("f32",), steps=3):
    """BB path with its fastest stage form at the given orders on unit-wavespeed Kuhn meshes
    sized so that a stage's FP32 working set is at least 4x the L2, with the roofline
    fraction (the C2 headline mesh and C3 at low N are partly L2-resident)."""
    from paper_1512_06025_gb300 import autotune
    out = {}
    for N in orders:
        n = LARGE_MESH_N[N]
        VX, EToV = inputs.kuhn_cube_mesh(n)
        K = len(EToV)
        dt = 0.25 * (1.0 / n) / (N + 1) ** 2
        row = {"mesh": f"{n}^3x6={K} tets", "working_set_mb_f32": round(3 * 4 * K * np_of(N) * 4 / 1e6, 1)}
        for name in precisions:
            prec = bbdg.BBDG_F32 if name == "f32" else bbdg.BBDG_F64
            s = bbdg.Solver(VX, EToV, np.ones(K), np.ones(K), N, precision=prec)
            q0 = torch.tensor(inputs.abi_layout(inputs.random_state(K, N)), dtype=s.torch_dtype, device=dev)
            z, w = torch.zeros_like(q0), torch.empty_like(q0)
            form, _ = autotune.tune_form(s, q0.clone(), z, w, reps=2)
            del z, w
            stage, finite = time_stages(bbdg, torch, s, q0, dt, stream, flush, steps)
            row["bb_" + name] = round(4 * K * s.Np / (stage * 1e-3) / 1e9, 3)
            row["bb_" + name + "_form"] = FORM_NAMES[form]
            row["bb_" + name + "_roofline"] = bb_roofline(N, 4 if name == "f32" else 8, stage, K, peaks)
            row["bb_" + name + "_finite"] = finite
            s.close()
            del q0
        out[N] = row
    return out


# ---------------------------------------------------------------------------------------
# CPU oracle (baseline / reference arm)
# ---------------------------------------------------------------------------------------
def _oracle_stage_timer(n):
    from oracle import dg
    from paper_1512_06025_gb300 import inputs
    VX, EToV = inputs.kuhn_cube_mesh(n)
    K = len(EToV)
    P = dg.make_problem(VX, EToV, N_ORDER, np.ones(K), np.ones(K))
    q = inputs.random_state(K, N_ORDER)[0]
    res = np.zeros_like(q)
    dt = 0.25 * (1.0 / n) / (N_ORDER + 1) ** 2
    a, b = float(dg.LSERK_A[1]), float(dg.LSERK_B[1])

    def stage():
        nonlocal q, res
        res = a * res + dt * dg.rhs(P, q)
        q = q + b * res
    return K, stage


def cpu_threads():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        if info:
            return max(int(i.get("num_threads", 1)) for i in info)
    except Exception:
        pass
    return os.cpu_count()


def cpu_baseline():
    """The oracle as it stands on the host cores: one LSERK4 step (5 stages) of the full
    workload mesh, FP64, numpy."""
    K, stage = _oracle_stage_timer(N_HEX)
    stage()                                  # warm (first-call allocations)
    t0 = time.perf_counter()
    for _ in range(5):
        stage()
    dt = (time.perf_counter() - t0) / 5
    dof = 4 * K * np_of(N_ORDER)
    out = {"value": round(dof / dt / 1e9, 5), "unit": UNIT, "cores": cpu_threads(), "kind": "oracle",
           "sample": f"5 RK stages (1 LSERK4 step) of the full {K}-tet N={N_ORDER} mesh, FP64 numpy",
           "stage_s": round(dt, 4)}
    single = cpu_baseline_single_core()
    if single is not None:
        out["single_core"] = single
    return out


def cpu_baseline_single_core(n=8):
    """The oracle with every BLAS / OpenMP pool held to one thread (a child process, so the
    setting applies before numpy loads): one RK stage of an n^3 x 6 mesh, scaled per DOF."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               BLIS_NUM_THREADS="1", VECLIB_MAXIMUM_THREADS="1")
    code = ("import sys, time, json; sys.path.insert(0, %r); import bench; K, st = bench._oracle_stage_timer(%d); "
            "st(); t = time.perf_counter(); st(); st(); dt = (time.perf_counter() - t) / 2; "
            "print(json.dumps({'K': K, 'stage_s': dt}))") % (ROOT, n)
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
        d = json.loads(r.stdout.strip().splitlines()[-1])
    except Exception:
        return None
    dof = 4 * d["K"] * np_of(N_ORDER)
    return {"value": round(dof / d["stage_s"] / 1e9, 5), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"1 RK stage of a {n}^3x6={d['K']}-tet N={N_ORDER} mesh, FP64 numpy, one thread",
            "stage_s": round(d["stage_s"], 4)}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    # size the per-step sample so that warmup + steps stays within about two minutes
    budget = 120.0
    K8, st8 = _oracle_stage_timer(8)
    st8()
    t0 = time.perf_counter()
    st8()
    t8 = time.perf_counter() - t0
    n = 8
    for cand in (16, 12, 10, 8, 6, 4):
        if t8 * (cand / 8) ** 3 * (args.steps + args.warmup) <= budget:
            n = cand
            break
    else:
        n = 4
    K, stage = _oracle_stage_timer(n)
    for _ in range(args.warmup):
        stage()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        stage()
    el = time.perf_counter() - t0
    dof = 4 * K * np_of(N_ORDER)
    value = dof / (el / args.steps) / 1e9
    cb = {"value": round(value, 5), "unit": UNIT, "cores": cpu_threads(), "kind": "oracle",
          "sample": f"each step = 1 RK stage (RHS + update) of a {n}^3x6={K}-tet N={N_ORDER} mesh, FP64 numpy"}
    return {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(el / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded random BB coefficients, Kuhn cube mesh)",
            "config": {**workload_config(), "parallelism": "CPU oracle on rank 0"},
            "cpu_baseline": cb,
            "e2e": {"value": round(value, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def profile_case(case, steps):
    """A short single-path run for profilers (no timing, small device footprint): `case`
    is bb_f32 / bb_f64 (C2 stages, default stage form), bb_f32_pipe (C2 stages, pipelined
    form), bb_f32_thread (element-per-thread form, N = 1 on a 64^3 x 6 mesh, 100 MB per
    state array), nodal_tc (C2 tensor-core nodal stages, node-row kernel), nodal_tc_rows (the
    C2 mesh at N = 4, element-row kernel) or adjoint (C5,
    a few steps of forward + reverse with the whole trajectory kept)."""
    import torch
    from paper_1512_06025_gb300 import bbdg, inputs
    torch.cuda.set_device(0)
    if case == "adjoint":
        from paper_1512_06025_gb300.gradient import MisfitGradient
        N, n = 5, 16
        VX, EToV = inputs.kuhn_cube_mesh(n)
        K = len(EToV)
        c = inputs.uniform_wavespeed(K)
        rho, kappa = inputs.materials_from_wavespeed(c)
        s = bbdg.Solver(VX, EToV, rho, kappa, N, precision=bbdg.BBDG_F64)
        bbdg.bbdg_set_sources(s.ctx, inputs.random_points(8, (-0.4, -0.4, 0.0), (0.4, 0.4, 0.4)),
                              np.zeros(8, dtype=np.int64), 10.0, 0.05)
        bbdg.bbdg_set_receivers(s.ctx, inputs.receiver_plane(1.0 / n, 16))
        dt = 0.25 * (1.0 / n) / (N + 1) ** 2 / c.max()
        drv = MisfitGradient(s, dt, steps, torch.zeros((steps, 256), dtype=torch.float64, device="cuda"))
        drv.forward()
        g = drv.backward()
        torch.cuda.synchronize()
        out = {"case": case, "steps": steps, "finite": bool(torch.isfinite(g).all().item())}
        s.close()
        return out
    basis = {"bb_f32": bbdg.BBDG_BB, "bb_f32_pipe": bbdg.BBDG_BB, "bb_f64": bbdg.BBDG_BB,
             "bb_f32_thread": bbdg.BBDG_BB, "nodal_tc": bbdg.BBDG_NODAL_TC, "nodal_tc_rows": bbdg.BBDG_NODAL_TC}[case]
    prec = bbdg.BBDG_F64 if case == "bb_f64" else bbdg.BBDG_F32
    N, n = {"nodal_tc_rows": (4, 16), "bb_f32_thread": (1, 64)}.get(case, (7, 16))
    VX, EToV = inputs.kuhn_cube_mesh(n)
    K = len(EToV)
    s = bbdg.Solver(VX, EToV, np.ones(K), np.ones(K), N, basis=basis, precision=prec)
    if case == "bb_f32_pipe":
        bbdg.bbdg_set_stage_form(s.ctx, bbdg.BBDG_FORM_PIPE, 0)
    elif case == "nodal_tc":
        bbdg.bbdg_set_stage_form(s.ctx, bbdg.BBDG_FORM_GROUP, 0)
    elif case == "nodal_tc_rows":
        bbdg.bbdg_set_stage_form(s.ctx, bbdg.BBDG_FORM_ROWS, 0)
    elif case == "bb_f32_thread":
        bbdg.bbdg_set_stage_form(s.ctx, bbdg.BBDG_FORM_THREAD, 0)
    q = torch.tensor(inputs.abi_layout(inputs.random_state(K, N)), dtype=s.torch_dtype, device="cuda")
    res, scr = torch.zeros_like(q), torch.empty_like(q)
    bbdg.bbdg_step(s.ctx, q, res, scr, 0.0, 0.25 / n / (N + 1) ** 2, steps)
    torch.cuda.synchronize()
    bbdg.bbdg_device_status(s.ctx)
    out = {"case": case, "steps": steps, "finite": bool(torch.isfinite(q).all().item())}
    s.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp32-only", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-nodal", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--sweep", action="store_true",
                    help="widen the N = 1..10 sweep: element-per-warp lines, large meshes at every N <= 7")
    ap.add_argument("--no-sweep", action="store_true", help="skip the N = 1..10 sweep")
    ap.add_argument("--profile-case", choices=["bb_f32", "bb_f32_pipe", "bb_f32_thread", "bb_f64", "nodal_tc", "nodal_tc_rows",
                                                "adjoint"],
                    help="run a few steps of one path for a profiler and exit (no timing)")
    args = ap.parse_args()
    if args.profile_case:
        print(json.dumps(profile_case(args.profile_case, min(args.steps, 4))), flush=True)
        return
    if args.warmup < 3:
        args.warmup = 3
    rank, world, local_rank = dist_env()
    if args.impl == "reference":
        r = run_reference(args, rank, world)
    else:
        r = run_gpu(args, rank, world, local_rank)
    if rank == 0 and r is not None:
        print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
