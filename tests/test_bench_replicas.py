"""Host logic of the multi-GPU path (replicas only: every rank runs the whole workload on
its own GPU, no data-path collective): the max-over-ranks reduction of the stage time and
the whole-job value, run as two gloo ranks on the CPU; and the reference arm, which rank 0
alone runs."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        stage_ms = [0.080, 0.095][rank]          # rank 1 is the slower replica
        mx = bench.reduce_max(stage_ms, world, torch.device("cpu"))
        out[rank] = (mx, bench.weak_value(world, 11796480, mx))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    world, port = 2, _free_port()
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0] == res[1]
    mx, value = res[0]
    assert mx == pytest.approx(0.095)
    assert value == pytest.approx(2 * 11796480 / 0.095e-3 / 1e9)


def test_single_rank_value():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(0.5, 1, None) == 0.5
    assert bench.weak_value(1, 1e9, 1000.0) == pytest.approx(1.0)


def test_reference_arm_runs_on_rank_zero_only():
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    args = argparse.Namespace(steps=1, warmup=0)
    assert bench.run_reference(args, rank=1, world=2) is None
