"""bench.py with N replicas (one process per GPU, no data-path collective):
the host logic -- max-over-ranks timing and the whole-job aggregate -- on
two gloo ranks on the CPU."""
import importlib.util
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import torch.distributed as dist

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    b = _bench()
    t = b.reduce_max(times[rank], dist, "cpu")
    dist.barrier()
    out[rank] = (t, b.replica_mlups(world, 1000, 10, t))
    dist.destroy_process_group()


def test_replica_timing_and_aggregate_two_gloo_ranks():
    import torch.multiprocessing as mp

    world, times = 2, [0.25, 0.5]
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank, args=(r, world, port, times, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    # every rank sees the slowest rank's time; the value counts all ranks' updates
    assert [out[r][0] for r in range(world)] == [0.5, 0.5]
    assert out[0][1] == pytest.approx(world * 1000 * 10 / 0.5 / 1e6)


def test_single_process_needs_no_group():
    b = _bench()
    assert b.reduce_max(0.3) == 0.3
    assert b.replica_mlups(1, 16777216, 2000, 1.0) == pytest.approx(33554.432)
