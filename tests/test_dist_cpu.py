"""The multi-rank host path of bench.py on CPU: two gloo ranks on 127.0.0.1 exchange the
per-rank times and solve counts exactly as the GPU ranks do (one process per GPU, weak
scaling: value = all ranks' solves / the slowest rank's time)."""
import importlib.util
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import torch.distributed as dist
    b = _bench()
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 100.0 + 50.0 * rank          # this rank's timed region
        solves = 20 * (rank + 1)          # this rank's solves
        b.barrier(world)
        out[rank] = (b.all_max(ms, world), b.all_sum(solves, world))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_reduce_time_and_solves():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(90)
    assert all(p.exitcode == 0 for p in procs)
    # every rank sees the slowest time and the total solve count
    assert dict(out) == {0: (150.0, 60.0), 1: (150.0, 60.0)}


def test_single_rank_passthrough():
    b = _bench()
    assert b.all_max(3.5, 1) == 3.5 and b.all_sum(7, 1) == 7
