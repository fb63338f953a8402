"""Autotuner for the launch shape of the stage kernels.

The paper tunes the number of elements per thread block of each kernel (K_V, K_S, K_U,
Section 4.2).  The fused stage kernel has two launch parameters: E, the elements per group
(one group per CTA iteration), and, for batched runs, the shots per tile (the order in
which concurrently running CTAs visit (element group, shot) pairs).  This module times
candidates through the C ABI (bbdg_set_launch_shape + bbdg_rk_stage; CUDA events on the
launching stream; L2 flushed between repetitions), keeps the fastest, and caches it per
(GPU, basis, precision, N, shots, K bucket) in a JSON file next to the library
(git-ignored).  `tune_lift_variant` also chooses between the two BB surface variants
(Algorithm 1 and the sparse E_L of Algorithm 3, N <= 6), as the paper compares them, and
`tune_stage_form` between the group kernel and the element-per-warp kernel, and
`tune_form` among every stage form built for the context (group, warp-specialised
pipelined, element per warp), each with its own launch parameters tuned.
"""
from __future__ import annotations

import json
import os

from . import bbdg

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_autotune.json")

BB_CANDIDATES = (1, 2, 3, 4, 6, 8, 12, 16, 24)
NODAL_CANDIDATES = (4, 8, 12, 16, 24, 32)
SHOT_TILES = (1, 2, 4, 8, 16)
WARP_CANDIDATES = (2, 4, 8, 16)


def _key(basis, precision, N, S, K):
    import torch
    name = torch.cuda.get_device_name().replace(" ", "_")
    kb = 1 << max(0, int(K).bit_length() - 1)      # K bucket (power of two)
    return f"{name}|b{basis}|p{precision}|N{N}|S{S}|K{kb}"


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(d):
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def _time_shape(solver, q, res, scratch, S, E, ST, reps, flush, stream):
    import torch
    if E is not None:
        bbdg.bbdg_set_launch_shape(solver.ctx, E, ST)
    a, b = q, scratch
    ms = []
    for r in range(reps + 1):
        flush.fill_(float(r))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for st in range(5):
            bbdg.bbdg_rk_stage(solver.ctx, a, b, res, st, 0.0, 1e-6, S=S, stream=stream)
            a, b = b, a
        e1.record(stream)
        torch.cuda.synchronize()
        if r > 0:
            ms.append(e0.elapsed_time(e1) / 5)
    return sorted(ms)[len(ms) // 2]


def tune(solver, q, res, scratch, S=None, basis=bbdg.BBDG_BB, reps=6, use_cache=True, flush_mb=512):
    """Pick (E, shots per tile) for solver's context; sets it and returns
    (E, {"E=..,ST=..": ms_per_stage}).  q, res, scratch: device tensors shaped like the
    workload's state (their contents are overwritten)."""
    import torch
    S = q.shape[0] if S is None else S
    key = _key(basis, solver.precision, solver.N, S, solver.K)
    cache = _load() if use_cache else {}
    if key in cache:
        bbdg.bbdg_set_launch_shape(solver.ctx, int(cache[key]["E"]), int(cache[key].get("ST", 1)))
        return int(cache[key]["E"]), cache[key]["ms"]
    # the tensor-core nodal kernel's element tile is fixed by its MMA shape
    cands = BB_CANDIDATES if basis == bbdg.BBDG_BB else ([0] if basis == bbdg.BBDG_NODAL_TC else NODAL_CANDIDATES)
    flush = torch.empty(flush_mb * 1024 * 1024 // 4, dtype=torch.float32, device=q.device)
    stream = torch.cuda.current_stream()
    timings = {}
    for E in cands:
        try:
            timings[(E, 1)] = _time_shape(solver, q, res, scratch, S, E, 1, reps, flush, stream)
        except bbdg.BBDGError:
            continue
    bestE = min(timings, key=timings.get)[0]
    if S > 1:
        for ST in SHOT_TILES[1:]:
            if S % ST == 0:
                try:
                    timings[(bestE, ST)] = _time_shape(solver, q, res, scratch, S, bestE, ST, reps, flush, stream)
                except bbdg.BBDGError:
                    continue
    bestE, bestST = min(timings, key=timings.get)
    bbdg.bbdg_set_launch_shape(solver.ctx, bestE, bestST)
    table = {f"E={e},ST={t}": v for (e, t), v in timings.items()}
    if use_cache:
        cache = _load()
        cache[key] = {"E": bestE, "ST": bestST, "ms": table}
        _store(cache)
    return bestE, table


def tune_lift_variant(solver, q, res, scratch, S=None, reps=6):
    """BB basis: time both lift variants (each with its own tuned launch shape) for
    N <= 6 and keep the faster one on `solver`.  Returns (variant, {variant: ms_per_stage})."""
    import torch
    if solver.basis != bbdg.BBDG_BB or solver.N > 6:
        tune(solver, q, res, scratch, S=S, basis=solver.basis, reps=reps)
        return solver.lift_variant, {}
    best = {}
    for lv in (bbdg.BBDG_LIFT_OPTIMAL, bbdg.BBDG_LIFT_SPARSE_EL):
        solver.set_lift_variant(lv)
        E, table = tune(solver, q, res, scratch, S=S, basis=bbdg.BBDG_BB, reps=reps, use_cache=False)
        best[lv] = min(table.values())
    lv = min(best, key=best.get)
    solver.set_lift_variant(lv)
    tune(solver, q, res, scratch, S=S, basis=bbdg.BBDG_BB, reps=reps, use_cache=False)
    torch.cuda.synchronize()
    return lv, best


def tune_warps(solver, q, res, scratch, S=None, reps=6):
    """Element-per-warp form: time each warps-per-CTA candidate and keep the fastest on
    `solver` (form left at BBDG_FORM_WARP).  Returns (W, {W: ms_per_stage})."""
    import torch
    stream = torch.cuda.current_stream()
    flush = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device=q.device)
    table = {}
    for W in WARP_CANDIDATES:
        try:
            bbdg.bbdg_set_stage_form(solver.ctx, bbdg.BBDG_FORM_WARP, W)
        except bbdg.BBDGError:
            continue
        table[W] = _time_shape(solver, q, res, scratch, S, None, 1, reps, flush, stream)
    best = min(table, key=table.get)
    bbdg.bbdg_set_stage_form(solver.ctx, bbdg.BBDG_FORM_WARP, best)
    return best, table


def tune_stage_form(solver, q, res, scratch, S=None, reps=6):
    """BB basis, Algorithm 1, FP32 or FP64: time the group kernel (its launch shape tuned)
    and the element-per-warp kernel (its warps per CTA tuned) and keep the faster form on
    `solver`.  Returns (form, {"group": ms, "warp": ms})."""
    if (solver.basis != bbdg.BBDG_BB or solver.lift_variant != bbdg.BBDG_LIFT_OPTIMAL
            or solver.precision == bbdg.BBDG_F32_LIFT64):
        tune(solver, q, res, scratch, S=S, basis=solver.basis, reps=reps)
        return bbdg.BBDG_FORM_GROUP, {}
    bbdg.bbdg_set_stage_form(solver.ctx, bbdg.BBDG_FORM_GROUP, 0)
    _, gtable = tune(solver, q, res, scratch, S=S, basis=bbdg.BBDG_BB, reps=reps, use_cache=False)
    W, wtable = tune_warps(solver, q, res, scratch, S=S, reps=reps)
    best = {"group": min(gtable.values()), "warp": min(wtable.values())}
    if best["group"] <= best["warp"]:
        bbdg.bbdg_set_stage_form(solver.ctx, bbdg.BBDG_FORM_GROUP, 0)
        return bbdg.BBDG_FORM_GROUP, best
    return bbdg.BBDG_FORM_WARP, best


def _tune_tc_form(solver, q, res, scratch, S=None, reps=6):
    """Tensor-core nodal basis: time the node-row kernel (BBDG_FORM_GROUP) and, for N <= 6,
    the element-row kernel (BBDG_FORM_ROWS); keep the faster.  Returns (form, {name: ms})."""
    import torch
    S = q.shape[0] if S is None else S
    stream = torch.cuda.current_stream()
    flush = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device=q.device)
    names = {bbdg.BBDG_FORM_GROUP: "node_rows", bbdg.BBDG_FORM_ROWS: "element_rows"}
    best = {}
    for form in (bbdg.BBDG_FORM_GROUP, bbdg.BBDG_FORM_ROWS):
        try:
            bbdg.bbdg_set_stage_form(solver.ctx, form, 0)
        except bbdg.BBDGError:
            continue
        best[form] = _time_shape(solver, q, res, scratch, S, None, 1, reps, flush, stream)
    form = min(best, key=best.get)
    bbdg.bbdg_set_stage_form(solver.ctx, form, 0)
    solver.tuned = {"form": form}
    return form, {names[f]: v for f, v in best.items()}


def tune_form(solver, q, res, scratch, S=None, reps=6, use_cache=True, forms=None):
    """BB basis with Algorithm 1, FP32 or FP64: time the group kernel (elements per group and
    shots per tile tuned), the warp-specialised pipelined kernel (N <= 8) and the
    element-per-warp kernel (warps per CTA tuned) and the element-per-thread kernel (N <= 2),
    and keep the fastest on `solver`.  Tensor-core nodal basis: the node-row or the element-row kernel, whichever is faster.
    Other contexts fall back to `tune`.  Returns (form, {form name: ms per stage}); cached
    per (GPU, precision, N, shots, K bucket) like `tune`."""
    import torch
    if solver.basis == bbdg.BBDG_NODAL_TC:
        return _tune_tc_form(solver, q, res, scratch, S=S, reps=reps)
    if (solver.basis != bbdg.BBDG_BB or solver.lift_variant != bbdg.BBDG_LIFT_OPTIMAL
            or solver.precision == bbdg.BBDG_F32_LIFT64):
        tune(solver, q, res, scratch, S=S, basis=solver.basis, reps=reps, use_cache=use_cache)
        return bbdg.BBDG_FORM_GROUP, {}
    S = q.shape[0] if S is None else S
    key = "form|" + _key(solver.basis, solver.precision, solver.N, S, solver.K)
    cache = _load() if use_cache else {}
    names = {bbdg.BBDG_FORM_GROUP: "group", bbdg.BBDG_FORM_PIPE: "pipe", bbdg.BBDG_FORM_WARP: "warp",
             bbdg.BBDG_FORM_THREAD: "thread"}
    if key in cache:
        c = cache[key]
        bbdg.bbdg_set_launch_shape(solver.ctx, int(c["E"]), int(c.get("ST", 1)))
        bbdg.bbdg_set_stage_form(solver.ctx, int(c["form"]), int(c.get("W", 8)))
        solver.tuned = {"form": int(c["form"]), "E": int(c["E"]), "ST": int(c.get("ST", 1)), "W": int(c.get("W", 8))}
        return int(c["form"]), c["ms"]
    forms = forms or (bbdg.BBDG_FORM_GROUP, bbdg.BBDG_FORM_PIPE, bbdg.BBDG_FORM_WARP, bbdg.BBDG_FORM_THREAD)
    stream = torch.cuda.current_stream()
    flush = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device=q.device)
    best = {}
    bbdg.bbdg_set_stage_form(solver.ctx, bbdg.BBDG_FORM_GROUP, 0)
    E, gtable = tune(solver, q, res, scratch, S=S, basis=bbdg.BBDG_BB, reps=reps, use_cache=False)
    gbest = min(gtable, key=gtable.get)
    ST = int(gbest.split("ST=")[1])
    best[bbdg.BBDG_FORM_GROUP] = (gtable[gbest], 8)
    if bbdg.BBDG_FORM_PIPE in forms:
        try:
            bbdg.bbdg_set_stage_form(solver.ctx, bbdg.BBDG_FORM_PIPE, 0)
            best[bbdg.BBDG_FORM_PIPE] = (_time_shape(solver, q, res, scratch, S, None, 1, reps, flush, stream), 8)
        except bbdg.BBDGError:
            pass
    if bbdg.BBDG_FORM_THREAD in forms:
        try:
            bbdg.bbdg_set_stage_form(solver.ctx, bbdg.BBDG_FORM_THREAD, 0)
            best[bbdg.BBDG_FORM_THREAD] = (_time_shape(solver, q, res, scratch, S, None, 1, reps, flush, stream), 8)
        except bbdg.BBDGError:
            pass
    if bbdg.BBDG_FORM_WARP in forms:
        try:
            W, wtable = tune_warps(solver, q, res, scratch, S=S, reps=reps)
            best[bbdg.BBDG_FORM_WARP] = (min(wtable.values()), W)
        except bbdg.BBDGError:
            pass
    form = min(best, key=lambda f: best[f][0])
    bbdg.bbdg_set_launch_shape(solver.ctx, E, ST)
    bbdg.bbdg_set_stage_form(solver.ctx, form, best[form][1])
    table = {names[f]: v[0] for f, v in best.items()}
    solver.tuned = {"form": form, "E": E, "ST": ST, "W": best[form][1]}
    if use_cache:
        cache = _load()
        cache[key] = {"form": form, "E": E, "ST": ST, "W": best[form][1], "ms": table}
        _store(cache)
    return form, table
